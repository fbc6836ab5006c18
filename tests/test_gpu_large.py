"""Image sizes of the paper's size sweep (Section 5: N = 2048 ... 10240 over
fields of 1-3 degrees) and the mixed-radix transform lengths they need
(G = 2N = 2^a, 3 2^a, 5 2^a), through the C ABI against the FP64 oracle.

Small mixed-radix sizes are compared whole (tilted image, final image, the
reverse pass); the large ones on sampled pixels that the oracle evaluates one
by one: the tilted image against the exact dirty image of Section 3.2, and
the final image against the bilinear interpolation of that exact image at
the oracle's re-projection source positions (Section 3.3)."""
from dataclasses import replace

import numpy as np
import pytest
import torch

import paper_2512_06254_gb300 as toi
from oracle import toi_oracle as O
from paper_2512_06254_gb300 import synth

from gpu_helpers import gpu_image, plan_for, rel_err, to_dev, to_np

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5


def _small(n_ant, n_chan, N, n_pol, flag_frac=0.0):
    w = synth.tiny_workload()
    return replace(w, n_ant=n_ant, n_chan=n_chan, image_size=N, n_pol=n_pol,
                   flag_frac=flag_frac, cell_arcsec=2.0 * 128 / N)


@pytest.mark.parametrize("n_ant,n_chan,N,n_pol,weights", [
    (9, 40, 96, 1, False),       # G = 192 = 3 2^6
    (12, 33, 160, 4, True),      # G = 320 = 5 2^6, ragged channels, flags, weights
    (16, 64, 384, 2, False),     # G = 768 = 3 2^8
    (14, 50, 640, 1, True),      # G = 1280 = 5 2^8
])
def test_mixed_radix_sizes_match_oracle(n_ant, n_chan, N, n_pol, weights):
    w = _small(n_ant, n_chan, N, n_pol, 0.2 if weights else 0.0)
    sn = synth.make_snapshot(w, 1, with_weights=weights)
    s = to_np(sn)
    r = O.image_snapshot(s["uvw"], s["freq"], s["vis"], s["flag"], s["weight"], N,
                         w.cell_arcsec)
    plan = plan_for(w)
    out = gpu_image(plan, to_dev(sn))
    assert out["status"] == toi.TOI_OK
    et = rel_err(plan.buffer(toi.BUF_TILTED).cpu().numpy(), r["tilted"])
    ei = rel_err(out["image"], r["image"])
    print(f"N {N}: tilted {et:.2e} image {ei:.2e}")
    assert et < IMG_TOL and ei < IMG_TOL
    plan.close()


@pytest.mark.parametrize("N", [96, 160])
def test_mixed_radix_reverse_pass(N):
    """toi_degrid_backward at G = 3 2^a and 5 2^a against the oracle's
    adjoint (sample cotangents to 2e-5 of their peak)."""
    w = _small(10, 29, N, 2, 0.1)
    sn = synth.make_snapshot(w, 2, with_weights=True)
    h = to_np(sn)
    gimg = np.random.default_rng(4).normal(size=(N, N))
    ref = O.image_snapshot_adjoint(h["uvw"], h["freq"], h["vis"], h["flag"], h["weight"], N,
                                   w.cell_arcsec, gimg)
    plan = plan_for(w)
    d = to_dev(sn)
    img = torch.empty(N, N, dtype=torch.float32, device="cuda")
    plan.grid(d["uvw"], d["freq"], d["vis"], flag=d["flag"], weight=d["weight"])
    plan.image(0, img)
    gs = torch.empty(w.n_bl, w.n_chan, dtype=torch.complex64, device="cuda")
    plan.degrid_backward(torch.from_numpy(gimg.astype(np.float32)).cuda(), grad_sample=gs)
    assert plan.sync_status() == toi.TOI_OK
    assert rel_err(gs.cpu().numpy(), ref["g"]) < 2e-5
    plan.close()


def test_mixed_radix_batch():
    """The batched engine at N = 160 (G = 320): three uneven snapshots equal
    the oracle's images."""
    base = replace(synth.tiny_workload(), n_ant=12, n_chan=48, n_pol=2, image_size=160,
                   cell_arcsec=1.6)
    ws = synth.uneven_stream(base, 3, seed=3, channel_choices=(12, 24, 48), flag_max=0.4,
                             image_sizes=(160,))
    snaps = [synth.make_snapshot(w, s) for s, w in enumerate(ws)]
    plan = toi.Plan(160, base.cell_arcsec, base.n_bl, base.n_chan, base.n_pol, tlisi_tile=32,
                    batch_max=4)
    ds = []
    for sn in snaps:
        d = {k: (v.cuda() if v is not None else None) for k, v in sn.items()}
        d["image"] = torch.empty(160, 160, device="cuda")
        ds.append(d)
    rows = torch.empty(3, 5, 5, device="cuda")
    plan.batch(ds, rows)
    assert plan.sync_status() == toi.TOI_OK
    for w, sn, d in zip(ws, snaps, ds):
        h = to_np(sn)
        ref = O.image_snapshot(h["uvw"], h["freq"], h["vis"], h["flag"], h["weight"], 160,
                               w.cell_arcsec)["image"]
        assert rel_err(d["image"].cpu().numpy(), ref) < IMG_TOL
    plan.close()


# ------------------------------------------------ the paper's large sizes --

def _exact_block(p, N, cell, j2, j1):
    """Exact tilted image on the 2 x 2 block with corner (j2, j1) (rows,
    cols; entries past the last row or column are 0, as in the oracle's
    bilinear interpolation)."""
    rows = [j2, j2 + 1] if j2 + 1 < N else [j2]
    cols = [j1, j1 + 1] if j1 + 1 < N else [j1]
    blk = np.zeros((2, 2))
    blk[:len(rows), :len(cols)] = O.dirty_image_dft(p["r"][:, 0], p["r"][:, 1], p["c"], N, cell,
                                                    p["omega"], p["sumw"], rows, cols)
    return blk


@pytest.mark.parametrize("N,fov_deg", [
    (6144, 2.0),      # G = 12288 = 3 2^12
    (8192, 2.0),      # G = 16384
    (10240, 3.0),     # G = 20480 = 5 2^12, the paper's largest image and field
])
def test_paper_sizes_sampled_pixels(N, fov_deg):
    cell = fov_deg * 3600.0 / N
    w = synth.meerkat_workload(n_snap=8, n_chan=1024, image_size=N, cell_arcsec=cell)
    sn = synth.make_snapshot(w, 5)
    s = to_np(sn)
    p = O.prepare(s["uvw"], s["freq"], s["vis"], s["flag"], None)
    plan = plan_for(w)
    out = gpu_image(plan, to_dev(sn))
    assert out["status"] == toi.TOI_OK
    assert abs(out["info"][10] - p["xi"]) < 1e-9 and abs(out["info"][11] - p["eta"]) < 1e-9
    tilted = plan.buffer(toi.BUF_TILTED).cpu().numpy()
    image = out["image"]
    plan.close()
    rng = np.random.default_rng(N)
    pk = tuple(int(a) for a in np.unravel_index(np.argmax(np.abs(tilted)), tilted.shape))
    pix = [(int(a), int(b)) for a, b in rng.integers(0, N, size=(30, 2))] + [pk, (N // 2, N // 2)]
    rows = np.array([a for a, _ in pix])
    cols = np.array([b for _, b in pix])
    exact = np.array([O.dirty_image_dft(p["r"][:, 0], p["r"][:, 1], p["c"], N, cell, p["omega"],
                                        p["sumw"], [a], [b])[0, 0] for a, b in pix])
    peak = np.abs(tilted).max()
    et = np.abs(tilted[rows, cols] - exact).max() / peak
    # final image: output pixels away from the border, so that every source
    # position lies on the image (the largest shift is ~100 px here)
    out_pix = [(int(a), int(b)) for a, b in rng.integers(N // 16, N - N // 16, size=(16, 2))]
    fa2, fa1 = (int(a) for a in np.unravel_index(np.argmax(np.abs(image)), image.shape))
    out_pix += [(fa2 + d2, fa1 + d1) for d2, d1 in ((0, 0), (1, 0), (0, 1), (-2, 3))
                if N // 16 <= fa2 + d2 < N - N // 16 and N // 16 <= fa1 + d1 < N - N // 16]
    j2o = np.array([a for a, _ in out_pix], dtype=np.float64)
    j1o = np.array([b for _, b in out_pix], dtype=np.float64)
    j1, j2 = O.reproject_source_at(j1o, j2o, N, cell / 3600.0, p["xi"], p["eta"])
    want = []
    for a1, a2 in zip(j1, j2):
        b0, a0 = int(np.floor(a2)), int(np.floor(a1))
        fb, fa = a2 - b0, a1 - a0
        blk = _exact_block(p, N, cell, b0, a0)
        want.append((1 - fb) * ((1 - fa) * blk[0, 0] + fa * blk[0, 1]) +
                    fb * ((1 - fa) * blk[1, 0] + fa * blk[1, 1]))
    got = image[j2o.astype(int), j1o.astype(int)]
    ei = np.abs(got - np.array(want)).max() / peak
    shift = np.hypot(j1 - j1o, j2 - j2o).max()
    print(f"N {N} fov {fov_deg}: tilted {et:.2e}, final {ei:.2e}, largest shift {shift:.1f} px")
    assert et < IMG_TOL and ei < IMG_TOL
