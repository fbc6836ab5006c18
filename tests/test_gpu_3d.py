"""Near-coplanar (3-D) mode through the C ABI against the FP64 oracle on the
same seeded non-coplanar inputs (antenna heights): the selected plan
(N_slab and K exactly, Phi_max, alpha_slab, r3 range, t3max), the tilted and
final images, the coplanar limit against the 2-D mode, and the moment cap."""
from dataclasses import replace

import numpy as np
import pytest
import torch

import paper_2512_06254_gb300 as toi
from oracle import toi_oracle as O
from paper_2512_06254_gb300 import synth

from gpu_helpers import gpu_image, rel_err, to_dev, to_np

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5


def _workload(height, n_pol=1, flag_frac=0.0, cell=40.0):
    return replace(synth.tiny_workload(), n_ant=12, n_chan=16, f_lo_hz=150e6, f_hi_hz=160.5e6,
                   n_pol=n_pol, image_size=128, cell_arcsec=cell, height_sigma_m=height,
                   flag_frac=flag_frac)


def _plan(w, **kw):
    return toi.Plan(w.image_size, w.cell_arcsec, w.n_bl, w.n_chan, w.n_pol, mode=3, **kw)


@pytest.mark.parametrize("height,n_pol,weights", [
    (300.0, 1, False),      # Phi_max ~ 10.6: two slabs, K = 16
    (100.0, 4, True),       # one slab, K = 8; flags and weights
])
def test_mode3_matches_oracle(height, n_pol, weights):
    w = _workload(height, n_pol, 0.1 if weights else 0.0)
    sn = synth.make_snapshot(w, 2, with_weights=weights)
    h = to_np(sn)
    ref = O.image_snapshot_3d(h["uvw"], h["freq"], h["vis"], h["flag"], h["weight"],
                              w.image_size, w.cell_arcsec)
    plan = _plan(w)
    out = gpu_image(plan, to_dev(sn))
    assert out["status"] == toi.TOI_OK
    info = plan.mode3_info()
    rp = ref["plan"]
    assert (info["n_slab"], info["K"]) == (rp["n_slab"], rp["K"])
    assert info["phi_max"] == pytest.approx(rp["phi_max"], rel=1e-9)
    assert info["alpha_slab"] == pytest.approx(rp["alpha_slab"], rel=1e-9)
    assert info["t3max"] == pytest.approx(ref["t3max"], rel=1e-9)
    assert info["r3min"] == pytest.approx(float(ref["r"][:, 2].min()), rel=1e-9, abs=1e-9)
    assert info["r3max"] == pytest.approx(float(ref["r"][:, 2].max()), rel=1e-9, abs=1e-9)
    tilted = plan.buffer(toi.BUF_TILTED).cpu().numpy()
    et, ei = rel_err(tilted, ref["tilted"]), rel_err(out["image"], ref["image"])
    print(f"height {height}: n_slab {info['n_slab']} K {info['K']} tilted {et:.2e} image {ei:.2e}")
    assert et < IMG_TOL and ei < IMG_TOL
    plan.close()


def test_mode3_tracks_the_exact_3d_image():
    """Sampled pixels of the GPU's 3-D tilted image against the brute-force
    I_D^(3) (the Chebyshev truncation at K = 16 is far below the ES error
    here), and clearly closer to it than the 2-D image."""
    w = _workload(300.0)
    sn = synth.make_snapshot(w, 5)
    h = to_np(sn)
    p = O.prepare(h["uvw"], h["freq"], h["vis"], h["flag"], None)
    N = w.image_size
    rows = np.arange(0, N, 9)
    cols = np.arange(3, N, 11)
    exact = O.dirty_image_3d_dft(p["r"], p["c"], N, w.cell_arcsec, p["V"], p["omega"],
                                 p["sumw"], rows, cols)
    plan3 = _plan(w)
    gpu_image(plan3, to_dev(sn))
    t3 = plan3.buffer(toi.BUF_TILTED).cpu().numpy()[np.ix_(rows, cols)]
    plan3.close()
    plan2 = toi.Plan(N, w.cell_arcsec, w.n_bl, w.n_chan, w.n_pol)
    gpu_image(plan2, to_dev(sn))
    t2 = plan2.buffer(toi.BUF_TILTED).cpu().numpy()[np.ix_(rows, cols)]
    plan2.close()
    peak = np.abs(exact).max()
    e3, e2 = np.abs(t3 - exact).max() / peak, np.abs(t2 - exact).max() / peak
    print(f"sampled vs exact I_D^(3): 3-D {e3:.2e}, 2-D {e2:.2e}")
    assert e3 < IMG_TOL
    assert e2 > 10 * e3


def _coplanar(sn):
    """The snapshot with its uvw projected onto their best-fit plane, so r3
    vanishes to rounding."""
    uvw = sn["uvw"].clone()
    _, _, vt = torch.linalg.svd(uvw - uvw.mean(0), full_matrices=False)
    n = vt[2]
    out = dict(sn)
    out["uvw"] = (uvw - (uvw @ n)[:, None] * n[None, :]).contiguous()
    return out


def test_mode3_coplanar_equals_2d():
    w = _workload(0.0)
    sn = _coplanar(synth.make_snapshot(w, 1))
    plan3 = _plan(w)
    o3 = gpu_image(plan3, to_dev(sn))
    info = plan3.mode3_info()
    plan3.close()
    plan2 = toi.Plan(w.image_size, w.cell_arcsec, w.n_bl, w.n_chan, w.n_pol)
    o2 = gpu_image(plan2, to_dev(sn))
    plan2.close()
    assert info["n_slab"] == 1 and info["K"] == 8
    assert rel_err(o3["image"], o2["image"]) < IMG_TOL


def test_mode3_moment_cap_and_unsupported_paths():
    w = _workload(300.0)                 # needs N_slab K = 32
    sn = synth.make_snapshot(w, 2)
    d = to_dev(sn)
    plan = _plan(w, max_moments=16)
    with pytest.raises(toi.ToiError) as e:
        plan.grid(d["uvw"], d["freq"], d["vis"], flag=d["flag"])
    assert e.value.status == toi.TOI_ERR_UNSUPPORTED and "max_moments" in str(e.value)
    plan.close()
    plan = _plan(w)
    plan.grid(d["uvw"], d["freq"], d["vis"], flag=d["flag"])
    img = torch.empty(w.image_size, w.image_size, device="cuda")
    plan.image(0, img)
    g = torch.zeros_like(img)
    gs = torch.empty(w.n_bl, w.n_chan, dtype=torch.complex64, device="cuda")
    with pytest.raises(toi.ToiError) as e:
        plan.degrid_backward(g, grad_sample=gs)
    assert e.value.status == toi.TOI_ERR_UNSUPPORTED
    plan.close()
    with pytest.raises(toi.ToiError) as e:
        _plan(w, batch_max=4)
    assert e.value.status == toi.TOI_ERR_UNSUPPORTED
