"""Reverse mode of the snapshot image on the GPU (toi_degrid_backward and the
autograd wrapper) against the FP64 oracle's adjoint on the same seeded
inputs.

Tolerances: the GPU chain is float32 (bilinear gather, two FFT passes of
length G, 64-tap degridding); each stage adds rounding of a few 1e-7 of the
largest magnitude it carries, so the sample cotangents are compared at
2e-5 of max |g|.  grad_weight subtracts <dL/dI, I> / sum w from
Re(conj(g) V), and the float32 forward image enters that term, so it is
compared at 1e-4 of max |grad_weight|."""
from dataclasses import replace

import numpy as np
import pytest
import torch

import paper_2512_06254_gb300 as toi
from oracle import toi_oracle as O
from paper_2512_06254_gb300 import synth
from paper_2512_06254_gb300.autograd import image_snapshot

from gpu_helpers import plan_for, rel_err, to_dev, to_np

pytestmark = pytest.mark.gpu

G_TOL = 2e-5
GW_TOL = 1e-4


def _workload(n_ant, n_chan, N, n_pol, flag_frac):
    w = synth.tiny_workload()
    return replace(w, n_ant=n_ant, n_chan=n_chan, image_size=N, n_pol=n_pol,
                   flag_frac=flag_frac, cell_arcsec=2.0 * 128 / N)


def _gpu_backward(plan, d, gimg, n_pol):
    N = plan.N
    img = torch.empty(N, N, dtype=torch.float32, device="cuda")
    plan.grid(d["uvw"], d["freq"], d["vis"], flag=d["flag"], weight=d.get("weight"))
    plan.image(0, img)
    nbl, nch = d["vis"].shape[:2]
    gs = torch.empty(nbl, nch, dtype=torch.complex64, device="cuda")
    gv = torch.empty(nbl, nch, n_pol, dtype=torch.complex64, device="cuda")
    gw = torch.empty(nbl, nch, n_pol, dtype=torch.float32, device="cuda")
    g_dev = torch.from_numpy(gimg.astype(np.float32)).cuda()
    plan.degrid_backward(g_dev, image=img, grad_sample=gs, grad_vis=gv, grad_weight=gw)
    assert plan.sync_status() == toi.TOI_OK
    return dict(image=img.cpu().numpy(), g=gs.cpu().numpy(), grad_vis=gv.cpu().numpy(),
                grad_weight=gw.cpu().numpy())


@pytest.mark.parametrize("n_ant,n_chan,N,n_pol,weights", [
    (16, 64, 128, 1, False),
    (11, 70, 256, 4, True),      # ragged channels, flags, weights
    (5, 37, 64, 2, True),
])
def test_backward_matches_oracle_adjoint(n_ant, n_chan, N, n_pol, weights):
    w = _workload(n_ant, n_chan, N, n_pol, 0.2 if weights else 0.0)
    sn = synth.make_snapshot(w, 2, with_weights=weights)
    h = to_np(sn)
    rng = np.random.default_rng(21)
    gimg = rng.normal(size=(N, N))
    ref = O.image_snapshot_adjoint(h["uvw"], h["freq"], h["vis"], h["flag"], h["weight"], N,
                                   w.cell_arcsec, gimg)
    plan = plan_for(w)
    out = _gpu_backward(plan, to_dev(sn), gimg, n_pol)
    eg = rel_err(out["g"], ref["g"])
    ev = rel_err(out["grad_vis"], ref["grad_vis"])
    ew = rel_err(out["grad_weight"], ref["grad_weight"])
    print(f"n_pol {n_pol} N {N}: g {eg:.2e}, grad_vis {ev:.2e}, grad_weight {ew:.2e}")
    assert eg < G_TOL and ev < G_TOL and ew < GW_TOL
    # zero exactly where the definition says so
    assert np.all(out["g"][ref["g"] == 0] == 0)
    assert np.all(out["grad_weight"][ref["grad_weight"] == 0] == 0)
    # the adjoint identity on the GPU's own forward and reverse passes
    L = float((gimg * out["image"]).sum())
    via = float((np.conj(out["grad_vis"].astype(np.complex128)) * h["vis"]).real.sum())
    assert abs(via - L) <= 1e-5 * np.abs(gimg).sum() * np.abs(out["image"]).max()
    # the slot is clear again: the next snapshot images correctly
    sn2 = synth.make_snapshot(w, 3, with_weights=weights)
    h2 = to_np(sn2)
    r2 = O.image_snapshot(h2["uvw"], h2["freq"], h2["vis"], h2["flag"], h2["weight"], N,
                          w.cell_arcsec)
    d2 = to_dev(sn2)
    img2 = torch.empty(N, N, dtype=torch.float32, device="cuda")
    plan.grid(d2["uvw"], d2["freq"], d2["vis"], flag=d2["flag"], weight=d2.get("weight"))
    plan.image(0, img2)
    assert rel_err(img2.cpu().numpy(), r2["image"]) < 1e-5
    plan.close()


def test_backward_meerkat_sampled_samples():
    """2016 x 4096 x 4 MeerKAT-shaped snapshot: the GPU sample cotangents at
    4096 sampled selected samples equal the oracle's ES degridding of the
    oracle's grid cotangent there."""
    w = synth.meerkat_workload()
    sn = synth.make_snapshot(w, 4, device="cuda", uvw_index=4)
    N = w.image_size
    rng = np.random.default_rng(8)
    gimg = rng.normal(size=(N, N))
    plan = plan_for(w)
    img = torch.empty(N, N, dtype=torch.float32, device="cuda")
    plan.grid(sn["uvw"], sn["freq"], sn["vis"], flag=sn["flag"])
    plan.image(0, img)
    gs = torch.empty(w.n_bl, w.n_chan, dtype=torch.complex64, device="cuda")
    plan.degrid_backward(torch.from_numpy(gimg.astype(np.float32)).cuda(), grad_sample=gs)
    assert plan.sync_status() == toi.TOI_OK
    g_gpu = gs.cpu().numpy()
    plan.close()

    s = {k: (v.cpu().numpy() if v is not None else None) for k, v in sn.items()}
    p = O.prepare(s["uvw"], s["freq"], s["vis"], s["flag"], None)
    W, G = 8, 2 * N
    beta = O.es_beta(W)
    gt = O.reproject_adjoint(gimg, w.cell_arcsec, p["xi"], p["eta"])
    H = O.tilted_image_adjoint(gt, G, W, beta, p["omega"], p["sumw"])
    sel_flat = np.flatnonzero(p["sel"].ravel())
    pick = rng.choice(len(sel_flat), 4096, replace=False)
    g1, g2 = O.grid_coords(p["r"][pick, 0], p["r"][pick, 1], N, w.cell_arcsec)
    g_ref = O.degrid_es(H, g1, g2, W, beta)
    got = g_gpu.ravel()[sel_flat[pick]]
    err = np.abs(got - g_ref).max() / np.abs(g_ref).max()
    print(f"meerkat sampled g relative error {err:.2e}")
    assert err < G_TOL
    assert np.all(g_gpu.ravel()[np.flatnonzero(~p["sel"].ravel())] == 0)


def test_autograd_point_source_and_weights():
    """A localisation-style loss sum (I - target)^2 through the autograd
    wrapper with a torch point-source model: d/d(l, m, S) and d/dw equal the
    oracle's adjoint and chain rule on the same loss."""
    w = _workload(12, 48, 128, 4, 0.1)
    sn = synth.make_snapshot(w, 1, with_weights=True)
    h = to_np(sn)
    N = w.image_size
    cell = w.cell_arcsec * O.ARCSEC
    l0, m0, S0 = 5.2 * cell, -3.7 * cell, 1.3
    target = O.image_snapshot(h["uvw"], h["freq"],
                              O.point_source_vis(h["uvw"], h["freq"], 4, l0 + 0.4 * cell,
                                                 m0 - 0.3 * cell, 1.1),
                              h["flag"], h["weight"], N, w.cell_arcsec)["image"]

    d = to_dev(sn)
    lt = torch.tensor(l0, dtype=torch.float64, device="cuda", requires_grad=True)
    mt = torch.tensor(m0, dtype=torch.float64, device="cuda", requires_grad=True)
    St = torch.tensor(S0, dtype=torch.float64, device="cuda", requires_grad=True)
    wt = d["weight"].clone().requires_grad_(True)
    k = d["freq"] / O.C_LIGHT
    u, v, ww = d["uvw"][:, 0:1], d["uvw"][:, 1:2], d["uvw"][:, 2:3]
    n = torch.sqrt(1 - lt * lt - mt * mt)
    ph = (u * lt + v * mt + ww * (n - 1)) * k[None, :]
    V = St * torch.exp(-2j * np.pi * ph)
    zero = torch.zeros_like(V)
    vis = torch.stack([V, zero, zero, V], dim=2).to(torch.complex64)
    plan = plan_for(w)
    img = image_snapshot(plan, d["uvw"], d["freq"], vis, flag=d["flag"], weight=wt)
    tgt = torch.from_numpy(target.astype(np.float32)).cuda()
    loss = ((img - tgt) ** 2).sum()
    loss.backward()
    plan.close()

    vis_np = O.point_source_vis(h["uvw"], h["freq"], 4, l0, m0, S0)
    r = O.image_snapshot(h["uvw"], h["freq"], vis_np, h["flag"], h["weight"], N, w.cell_arcsec)
    a = O.image_snapshot_adjoint(h["uvw"], h["freq"], vis_np, h["flag"], h["weight"], N,
                                 w.cell_arcsec, 2.0 * (r["image"] - target))
    gr = O.point_source_gradient(h["uvw"], h["freq"], a["grad_vis"], l0, m0, S0)
    got = dict(l=lt.grad.item(), m=mt.grad.item(), flux=St.grad.item())
    print("point-source gradient gpu", got, "oracle", gr)
    for key in ("l", "m", "flux"):
        assert abs(got[key] - gr[key]) <= 1e-4 * abs(gr[key]), key
    assert rel_err(wt.grad.cpu().numpy(), a["grad_weight"]) < GW_TOL


def test_backward_argument_errors():
    w = _workload(6, 16, 64, 4, 0.0)
    sn = synth.make_snapshot(w, 0)
    d = to_dev(sn)
    plan = plan_for(w)
    g = torch.zeros(64, 64, dtype=torch.float32, device="cuda")
    gs = torch.empty(w.n_bl, 16, dtype=torch.complex64, device="cuda")
    gw = torch.empty(w.n_bl, 16, 4, dtype=torch.float32, device="cuda")
    with pytest.raises(toi.ToiError) as e:
        plan.degrid_backward(g, grad_sample=gs)          # slot never gridded
    assert e.value.status == toi.TOI_ERR_ARG
    plan.grid(d["uvw"], d["freq"], d["vis"], flag=d["flag"])
    with pytest.raises(toi.ToiError) as e:
        plan.degrid_backward(g)                           # no output
    assert e.value.status == toi.TOI_ERR_ARG
    with pytest.raises(toi.ToiError) as e:
        plan.degrid_backward(g, grad_weight=gw)           # grad_weight without image
    assert e.value.status == toi.TOI_ERR_ARG
    plan.close()
