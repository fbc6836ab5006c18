"""FP16 visibility storage (half pairs with a per-channel FP32 scale, decoded
in the gridder, FP32 accumulation) through the C ABI.

Parity: the GPU path on the stored values against the FP64 oracle fed the
decoded values (scale x half, what the kernel reads) at the tolerance of the
complex64 path.  Quantisation error: the imaging map of Section 3.2 is linear
in the weighted sample values c_q, with |exp(i phase)| = 1, and bilinear
re-projection is a convex combination, so every pixel of the image made from
the quantised samples differs from the unquantised one by at most
sum_q |delta c_q| / (omega sum w) (plus the gridding error of both);
that bound is evaluated on the data and asserted, and the error printed."""
import numpy as np
import pytest
import torch

import paper_2512_06254_gb300 as toi
from oracle import toi_oracle as O
from paper_2512_06254_gb300 import synth

from gpu_helpers import gpu_image, plan_for, rel_err, to_dev, to_np

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5


def _decoded(q, scale):
    """The complex128 values the kernel reads from a half pair + scale."""
    qd = q.double()
    return torch.complex(qd[..., 0], qd[..., 1]) * scale.double()[None, :, None]


def _quant_bound(vis, dec, flag, n_pol, omega, sumw):
    """sum_q |delta c_q| / (omega sum w) over the parallel hands (unit
    weights, flags zero the weight of their polarisation)."""
    pa, pb = O.parallel_hands(n_pol)
    d = (dec - vis.to(torch.complex128))
    keep = (flag == 0).double()
    if pa == pb:
        dc = d[..., pa] * keep[..., pa]
    else:
        dc = d[..., pa] * keep[..., pa] + d[..., pb] * keep[..., pb]
    return float(dc.abs().sum()) / (omega * sumw)


def _plan16(w, **kw):
    return plan_for(w, vis_dtype=toi.TOI_VIS_C16_CHANSCALE, **kw)


def test_fp16_tiny_parity_and_quantisation_error():
    w = synth.tiny_workload()
    plan = _plan16(w)
    for s in range(w.n_snap):
        sn = synth.make_snapshot(w, s)
        q, scale = synth.to_fp16_channel_scaled(sn["vis"])
        dec = _decoded(q, scale)
        h = to_np(sn)
        ref_dec = O.image_snapshot(h["uvw"], h["freq"], dec.numpy(), h["flag"], None,
                                   w.image_size, w.cell_arcsec)
        ref = O.image_snapshot(h["uvw"], h["freq"], h["vis"], h["flag"], None,
                               w.image_size, w.cell_arcsec)
        d = to_dev(sn)
        d["vis"] = q.cuda()
        d["chan_scale"] = scale.cuda()
        out = gpu_image(plan, d)
        assert out["status"] == toi.TOI_OK
        assert rel_err(out["image"], ref_dec["image"]) < IMG_TOL
        bound = _quant_bound(sn["vis"], dec, sn["flag"], w.n_pol, ref["omega"], ref["sumw"])
        err = np.abs(out["image"] - ref["image"]).max()
        peak = np.abs(ref["image"]).max()
        print(f"tiny snapshot {s}: fp16 image error {err:.3e} (peak {peak:.3e}, "
              f"bound {bound:.3e}, relative {err / peak:.2e})")
        assert err <= bound + 2 * IMG_TOL * peak
    plan.close()


@pytest.fixture(scope="module")
def meerkat16():
    w = synth.meerkat_workload()
    sn = synth.make_snapshot(w, 5, device="cuda", uvw_index=5)
    q, scale = synth.to_fp16_channel_scaled(sn["vis"])
    return w, sn, q, scale


def test_fp16_meerkat_sampled_pixels_and_full_image_error(meerkat16):
    """2016 x 4096 x 4 MeerKAT-shaped snapshot stored as FP16: sampled tilted
    pixels match the exact Section 3.2 image of the decoded values; the whole
    image differs from the complex64 path's by less than the quantisation
    bound."""
    w, sn, q, scale = meerkat16
    N = w.image_size
    plan16 = _plan16(w)
    d = dict(sn)
    d["vis"] = q
    d["chan_scale"] = scale
    out16 = gpu_image(plan16, d)
    assert out16["status"] == toi.TOI_OK
    tilted16 = plan16.buffer(toi.BUF_TILTED).cpu().numpy()
    plan16.close()

    dec = _decoded(q, scale)
    s = {k: (v.cpu().numpy() if v is not None else None) for k, v in sn.items()}
    p = O.prepare(s["uvw"], s["freq"], dec.cpu().numpy(), s["flag"], None)
    rng = np.random.default_rng(11)
    pk = np.unravel_index(np.argmax(np.abs(tilted16)), tilted16.shape)
    pix = [(int(a), int(b)) for a, b in rng.integers(0, N, size=(30, 2))] + [pk]
    beta = w.cell_arcsec * O.ARCSEC
    vals, exact = [], []
    for (j2, j1) in pix:
        t1 = -beta * (j1 - N // 2)
        t2 = beta * (j2 - N // 2)
        ph = 2 * np.pi * (p["r"][:, 0] * t1 + p["r"][:, 1] * t2)
        exact.append((p["c"] * np.exp(1j * ph)).sum().real / (p["omega"] * p["sumw"]))
        vals.append(tilted16[j2, j1])
    peak = np.abs(tilted16).max()
    assert np.abs(np.array(vals) - np.array(exact)).max() < IMG_TOL * peak

    plan32 = plan_for(w)
    out32 = gpu_image(plan32, sn)
    plan32.close()
    bound = _quant_bound(sn["vis"], dec, sn["flag"], w.n_pol, p["omega"], p["sumw"])
    err = np.abs(out16["image"] - out32["image"]).max()
    print(f"meerkat snapshot 5: fp16 vs complex64 image max diff {err:.3e} "
          f"(peak {peak:.3e}, bound {bound:.3e}, relative {err / peak:.2e})")
    assert err <= bound + 2 * IMG_TOL * peak
