"""Windowed point-source localisation (toi_localise_seed, toi_localise and
the autograd wrapper) through the C ABI against the FP64 oracle on the same
seeded inputs, and against central finite differences of the GPU's own loss
(steps 1e-3 pixel in l and m, 1e-3 relative in S).

Tolerances: the model windows come from faceted ES gridding in float32
(1e-5 of the window peak, as the images); the loss and gradients combine
the GPU tilted image and the model, each within ~1e-6 of the peak, so they
are compared at 1e-4 relative (grad_weight: 1e-4 of its largest value)."""
from dataclasses import replace

import numpy as np
import pytest
import torch

import paper_2512_06254_gb300 as toi
from oracle import toi_oracle as O
from paper_2512_06254_gb300 import synth
from paper_2512_06254_gb300.autograd import localise_loss

from gpu_helpers import gpu_image, plan_for, rel_err, to_dev, to_np

pytestmark = pytest.mark.gpu

WIN = O.LOC_WINDOW


def _workload(n_ant=12, n_chan=48, N=128, n_pol=4, flag_frac=0.1):
    w = synth.tiny_workload()
    return replace(w, n_ant=n_ant, n_chan=n_chan, image_size=N, n_pol=n_pol,
                   flag_frac=flag_frac)


def _sources(h, w, windows, offsets):
    """A source near each window's centre, off the pixel grid."""
    p = O.prepare(h["uvw"], h["freq"], h["vis"], h["flag"], h["weight"])
    cell = w.cell_arcsec * O.ARCSEC
    N = w.image_size
    out = []
    for (j2c, j1c), (d2, d1, S) in zip(windows, offsets):
        t1 = -cell * (j1c + WIN // 2 + d1 - N // 2)
        t2 = cell * (j2c + WIN // 2 + d2 - N // 2)
        l, m = O.source_of_pixel(t1, t2, p["V"])
        out.append((l, m, S))
    return np.array(out)


def _setup(weights=True):
    w = _workload()
    sn = synth.make_snapshot(w, 3, with_weights=weights)
    h = to_np(sn)
    windows = np.array([[10, 70], [60, 20], [75, 30], [96, 96]])   # windows 1, 2 overlap
    src = _sources(h, w, windows, [(0.3, -0.4, 1.2), (-0.2, 0.1, 2.5), (1.3, 0.6, 0.7),
                                   (0.0, 0.0, 1.0)])
    plan = plan_for(w, max_windows=8)
    d = to_dev(sn)
    gpu_image(plan, d, out=False)
    return w, sn, h, d, windows, src, plan


def _run(plan, windows, src, weight_like=None, model=True):
    n = len(windows)
    win = torch.from_numpy(windows.astype(np.int32)).cuda()
    s = torch.from_numpy(src).cuda()
    out = dict(loss=torch.empty(n, dtype=torch.float64, device="cuda"),
               grad_src=torch.empty(n, 3, dtype=torch.float64, device="cuda"))
    if model:
        out["model"] = torch.empty(n, WIN, WIN, device="cuda")
    if weight_like is not None:
        out["grad_weight"] = torch.empty_like(weight_like)
    plan.localise(win, s, **out)
    assert plan.sync_status() == toi.TOI_OK
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_localise_matches_oracle():
    w, sn, h, d, windows, src, plan = _setup()
    got = _run(plan, windows, src, weight_like=d["weight"])
    plan.close()
    ref = O.localise(h["uvw"], h["freq"], h["vis"], h["flag"], h["weight"], w.image_size,
                     w.cell_arcsec, windows, src, WIN)
    em = max(rel_err(got["model"][i], ref["model"][i]) for i in range(len(windows)))
    el = np.abs(got["loss"] - ref["loss"]).max() / np.abs(ref["loss"]).max()
    eg = np.abs(got["grad_src"] - ref["grad_src"]) / np.abs(ref["grad_src"])
    ew = rel_err(got["grad_weight"], ref["grad_weight"])
    print(f"model {em:.2e} loss {el:.2e} grad_src {eg.max():.2e} grad_weight {ew:.2e}")
    assert em < 1e-5 and el < 1e-4 and eg.max() < 1e-4 and ew < 1e-4
    assert np.all(got["grad_weight"][ref["grad_weight"] == 0] == 0)


def test_gradients_match_gpu_finite_differences():
    w, sn, h, d, windows, src, plan = _setup()
    base = _run(plan, windows, src, model=False)
    cell = w.cell_arcsec * O.ARCSEC
    for i in (0, 2):
        for k, step in ((0, 1e-3 * cell), (1, 1e-3 * cell), (2, 1e-3 * src[i, 2])):
            sp, sm = src.copy(), src.copy()
            sp[i, k] += step
            sm[i, k] -= step
            Lp = _run(plan, windows, sp, model=False)["loss"].sum()
            Lm = _run(plan, windows, sm, model=False)["loss"].sum()
            fd = (Lp - Lm) / (2 * step)
            g = base["grad_src"][i, k]
            print(f"window {i} param {k}: analytic {g:.6e} central difference {fd:.6e}")
            assert abs(fd - g) <= 1e-2 * abs(g), (i, k)
    plan.close()


def test_true_source_gives_near_zero_loss():
    """Data that are the model's own visibilities: the GPU tilted image and
    the faceted model both equal the exact window image (1e-5 of its peak),
    so the loss is at rounding level."""
    w = _workload(flag_frac=0.0)
    sn = synth.make_snapshot(w, 3)
    h = to_np(sn)
    windows = np.array([[40, 50]])
    src = _sources(h, w, windows, [(0.25, -0.35, 1.7)])
    vis = O.point_source_vis(h["uvw"], h["freq"], w.n_pol, *src[0])
    sn = dict(sn, vis=torch.from_numpy(vis.astype(np.complex64)))
    plan = plan_for(w, max_windows=1)
    d = to_dev(sn)                # toi_localise reads the gridded inputs again
    gpu_image(plan, d, out=False)
    tilted = plan.buffer(toi.BUF_TILTED).cpu().numpy()
    got = _run(plan, windows, src)
    plan.close()
    pm = O.prepare(h["uvw"], h["freq"], vis, h["flag"], None)
    exact = O.window_image_exact(pm, w.image_size, w.cell_arcsec, windows[0], WIN)
    j2c, j1c = windows[0]
    D = tilted[j2c:j2c + WIN, j1c:j1c + WIN]
    peak = np.abs(exact).max()
    eD = np.abs(D - exact).max() / peak
    eM = np.abs(got["model"][0] - exact).max() / peak
    scale = (got["model"][0] ** 2).sum()
    print(f"true source: data {eD:.2e}, model {eM:.2e}, relative loss {got['loss'][0] / scale:.2e}")
    assert eD < 1e-5 and eM < 1e-5
    assert got["loss"][0] < 1e-9 * scale


def test_seed_picks_smallest_tlisi_tiles():
    w, sn, h, d, windows, src, plan = _setup(weights=False)
    nt = w.image_size // 32
    rng = np.random.default_rng(6)
    tl = rng.uniform(0.5, 1.0, size=(nt, nt)).astype(np.float32)
    tl[1, 2], tl[3, 0], tl[2, 2] = 0.1, 0.2, 0.2          # tie broken by tile index
    tl[0, 0] = np.nan
    n_win = 3
    win, s = plan.localise_seed(torch.from_numpy(tl).cuda(), n_win)
    win, s = win.cpu().numpy(), s.cpu().numpy()
    tilted = plan.buffer(toi.BUF_TILTED).cpu().numpy()
    plan.close()
    keys = sorted(range(nt * nt), key=lambda t: (np.inf if np.isnan(tl.flat[t]) else tl.flat[t], t))
    p = O.prepare(h["uvw"], h["freq"], h["vis"], h["flag"], None)
    N = w.image_size
    cell = w.cell_arcsec * O.ARCSEC
    for i, t in enumerate(keys[:n_win]):
        ty, tx = divmod(t, nt)
        c2 = min(max(ty * 32 + 16 - WIN // 2, 0), N - WIN)
        c1 = min(max(tx * 32 + 16 - WIN // 2, 0), N - WIN)
        assert tuple(win[i]) == (c2, c1)
        blk = tilted[c2:c2 + WIN, c1:c1 + WIN]
        j2, j1 = np.unravel_index(np.argmax(blk), blk.shape)
        l, m = O.source_of_pixel(-cell * (c1 + j1 - N // 2), cell * (c2 + j2 - N // 2), p["V"])
        # V from the GPU plane fit agrees with the oracle's to ~1e-9
        assert s[i, 0] == pytest.approx(l, rel=1e-8, abs=1e-13)
        assert s[i, 1] == pytest.approx(m, rel=1e-8, abs=1e-13)
        assert s[i, 2] == pytest.approx(p["omega"] * float(blk[j2, j1]), rel=1e-6)


def test_autograd_wrapper_and_argument_errors():
    w, sn, h, d, windows, src, plan = _setup()
    direct = _run(plan, windows, src, model=False)
    gpu_image(plan, d, out=False)                # the image again (tilted kept)
    win = torch.from_numpy(windows.astype(np.int32)).cuda()
    s = torch.from_numpy(src).cuda().requires_grad_(True)
    wt = d["weight"].clone().requires_grad_(True)
    plan.grid(d["uvw"], d["freq"], d["vis"], flag=d["flag"], weight=wt.detach())
    plan.image(0, None)
    L = localise_loss(plan, win, s, weight=wt)
    (3.0 * L).backward()
    assert float(L.detach()) == pytest.approx(direct["loss"].sum(), rel=1e-6)
    assert np.abs(s.grad.cpu().numpy() - 3.0 * direct["grad_src"]).max() <= \
        1e-5 * np.abs(direct["grad_src"]).max()
    assert wt.grad is not None and torch.isfinite(wt.grad).all()
    # the tilted image was used as workspace: another call is refused
    with pytest.raises(toi.ToiError) as e:
        plan.localise(win, s.detach())
    assert e.value.status == toi.TOI_ERR_ARG
    plan.close()
    p0 = plan_for(w)                             # max_windows = 0
    gpu_image(p0, d, out=False)
    with pytest.raises(toi.ToiError):
        p0.localise(win, s.detach())
    p0.close()
    # a window off the image: zero loss there and TOI_ERR_RANGE
    plan = plan_for(w, max_windows=8)
    gpu_image(plan, d, out=False)
    bad = windows.copy()
    bad[1] = (w.image_size - 8, 0)
    loss = torch.empty(len(bad), dtype=torch.float64, device="cuda")
    plan.localise(torch.from_numpy(bad.astype(np.int32)).cuda(), torch.from_numpy(src).cuda(),
                  loss=loss)
    assert plan.sync_status() == toi.TOI_ERR_RANGE
    lc = loss.cpu().numpy()
    assert lc[1] == 0.0 and lc[0] == pytest.approx(direct["loss"][0], rel=1e-6)
    plan.close()


def test_meerkat_windows_from_tlisi():
    """2016 x 4096 x 4 MeerKAT-shaped snapshots, 2048^2: 64 windows seeded
    from a tLISI matrix; window 0's model, loss and source gradient against
    the oracle (which evaluates that window exactly)."""
    wk = synth.meerkat_workload(n_snap=8)
    snaps = [synth.make_snapshot(wk, s) for s in range(3)]
    plan = toi.Plan(wk.image_size, wk.cell_arcsec, wk.n_bl, wk.n_chan, wk.n_pol, max_windows=64)
    nt = wk.image_size // 32
    row = torch.empty(nt, nt, device="cuda")
    for sn in snaps:
        d = to_dev(sn)
        plan.grid(d["uvw"], d["freq"], d["vis"], flag=d["flag"])
        plan.image(0, None)
        valid = plan.tlisi_update(None, row)
    assert valid
    win, src = plan.localise_seed(row, 64)
    n = 64
    model = torch.empty(n, WIN, WIN, device="cuda")
    loss = torch.empty(n, dtype=torch.float64, device="cuda")
    gsrc = torch.empty(n, 3, dtype=torch.float64, device="cuda")
    # move the starting sources off their pixels so the gradients are not ~0
    src[:, 0] += 0.3 * wk.cell_arcsec * O.ARCSEC
    plan.localise(win, src, model=model, loss=loss, grad_src=gsrc)
    assert plan.sync_status() == toi.TOI_OK
    win_np, src_np = win.cpu().numpy(), src.cpu().numpy()
    plan.close()
    assert len({tuple(x) for x in win_np}) == n
    h = to_np(snaps[-1])
    ref = O.localise(h["uvw"], h["freq"], h["vis"], h["flag"], None, wk.image_size,
                     wk.cell_arcsec, win_np[:1], src_np[:1], WIN)
    em = rel_err(model[0].cpu().numpy(), ref["model"][0])
    el = abs(loss[0].item() - ref["loss"][0]) / ref["loss"][0]
    eg = np.abs(gsrc[0].cpu().numpy() - ref["grad_src"][0]) / np.abs(ref["grad_src"][0])
    print(f"MeerKAT window 0: model {em:.2e} loss {el:.2e} grad_src {eg}")
    assert em < 1e-5 and el < 1e-4 and eg.max() < 1e-4


def test_more_windows_than_one_group():
    """70 windows (two window groups of the facet passes), two pols, no
    weights: losses and source gradients of every window against the
    oracle."""
    w = _workload(n_ant=10, n_chan=40, N=256, n_pol=2, flag_frac=0.05)
    sn = synth.make_snapshot(w, 4)
    h = to_np(sn)
    rng = np.random.default_rng(11)
    windows = rng.integers(0, w.image_size - WIN + 1, size=(70, 2))
    offs = [(float(a), float(b), float(S)) for a, b, S in
            zip(rng.uniform(-3, 3, 70), rng.uniform(-3, 3, 70), rng.uniform(0.5, 2.0, 70))]
    src = _sources(h, w, windows, offs)
    plan = plan_for(w, max_windows=80)
    d = to_dev(sn)
    gpu_image(plan, d, out=False)
    got = _run(plan, windows, src, weight_like=torch.empty(w.n_bl, w.n_chan, w.n_pol,
                                                           device="cuda"))
    plan.close()
    ref = O.localise(h["uvw"], h["freq"], h["vis"], h["flag"], None, w.image_size,
                     w.cell_arcsec, windows, src, WIN)
    el = np.abs(got["loss"] - ref["loss"]).max() / np.abs(ref["loss"]).max()
    eg = np.abs(got["grad_src"] - ref["grad_src"]) / np.abs(ref["grad_src"]).max(axis=0)
    ew = rel_err(got["grad_weight"], ref["grad_weight"])
    print(f"70 windows: loss {el:.2e} grad_src {eg.max():.2e} grad_weight {ew:.2e}")
    assert el < 1e-4 and eg.max() < 1e-4 and ew < 1e-4
