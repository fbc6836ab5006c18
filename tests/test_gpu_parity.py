"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.  Tolerances: float quantities to a max relative
error of 1e-5 of the image peak (FP32 path vs FP64 oracle); S1 geometry to
1e-9; candidate thresholds, scores and boxes bit for bit."""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

import paper_2512_06254_gb300 as toi  # noqa: E402
from paper_2512_06254_gb300 import synth  # noqa: E402
from oracle import toi_oracle as O  # noqa: E402
from gpu_helpers import gpu_image, plan_for, rel_err, to_dev, to_np  # noqa: E402

IMG_TOL = 1e-5


@pytest.fixture(scope="module")
def tiny():
    w = synth.tiny_workload()
    snaps = [synth.make_snapshot(w, s) for s in range(w.n_snap)]
    ref = []
    for sn in snaps:
        s = to_np(sn)
        ref.append(O.image_snapshot(s["uvw"], s["freq"], s["vis"], s["flag"], s["weight"],
                                    w.image_size, w.cell_arcsec, keep_grid=True))
    return w, snaps, ref


def _check_geometry(info, r):
    V = info[:9].reshape(3, 3)
    assert np.abs(V - r["V"]).max() < 1e-9
    assert info[9] == pytest.approx(r["omega"], rel=1e-12)
    assert info[10] == pytest.approx(r["xi"], rel=1e-9, abs=1e-12)
    assert info[11] == pytest.approx(r["eta"], rel=1e-9, abs=1e-12)
    assert info[12] == pytest.approx(r["sumw"], rel=1e-12)
    assert int(info[13]) == r["n_vis"]


def test_tiny_all_stages(tiny):
    """S1..S6 on all 8 tiny snapshots: geometry, half-plane grid, tilted and
    final images."""
    w, snaps, ref = tiny
    plan = plan_for(w)
    for sn, r in zip(snaps, ref):
        d = to_dev(sn)
        plan.grid(d["uvw"], d["freq"], d["vis"], flag=d["flag"])
        H = plan.buffer(toi.BUF_GRID).cpu().numpy()     # before toi_image consumes it
        Href = 2.0 * O.hermitian_half(r["grid"])[:-1]
        assert rel_err(H, Href) < IMG_TOL
        out = gpu_image(plan, d)
        assert out["status"] == toi.TOI_OK
        _check_geometry(out["info"], r)
        assert np.abs(plan.buffer(toi.BUF_GRID).cpu().numpy()).max() == 0.0   # consumed
        tilted = plan.buffer(toi.BUF_TILTED).cpu().numpy()
        assert rel_err(tilted, r["tilted"]) < IMG_TOL
        assert rel_err(out["image"], r["image"]) < IMG_TOL
    plan.close()


def test_tiny_tilted_matches_exact_dft(tiny):
    """The GPU tilted image equals the exact I_D^(2) of Section 3.2 within the
    ES kernel error plus FP32 rounding."""
    w, snaps, ref = tiny
    plan = plan_for(w)
    gpu_image(plan, to_dev(snaps[0]))
    tilted = plan.buffer(toi.BUF_TILTED).cpu().numpy()
    r = ref[0]
    d = O.dirty_image_dft(r["r"][:, 0], r["r"][:, 1], r["c"], w.image_size, w.cell_arcsec,
                          r["omega"], r["sumw"])
    assert rel_err(tilted, d) < IMG_TOL
    plan.close()


def test_tlisi_stream_fused_and_external(tiny):
    """tLISI over the tiny stream: (a) external images (the oracle's float32
    images) through tlisi_update equal the oracle's tLISI on the same images;
    (b) the fused toi_image -> tlisi_update path tracks the oracle pipeline."""
    w, snaps, ref = tiny
    T = 16
    plan = plan_for(w, tlisi_tile=T)
    nt = w.image_size // T
    out = torch.empty(nt, nt, dtype=torch.float32, device="cuda")
    imgs32 = [r["image"].astype(np.float32) for r in ref]
    for i, im in enumerate(imgs32):
        valid = plan.tlisi_update(torch.from_numpy(im).cuda(), out)
        assert valid == (i >= 2)
        if valid:
            exp = O.tlisi(imgs32[i - 2], imgs32[i - 1], im, T)
            assert np.abs(out.cpu().numpy() - exp).max() < 2e-6
    plan.tlisi_reset()
    for i, sn in enumerate(snaps):
        gpu_image(plan, to_dev(sn), out=False)
        valid = plan.tlisi_update(None, out)
        assert valid == (i >= 2)
        if valid:
            exp = O.tlisi(ref[i - 2]["image"], ref[i - 1]["image"], ref[i]["image"], T)
            assert np.abs(out.cpu().numpy() - exp).max() < 1e-4
    plan.close()


def _cand_case(cube, T, mode):
    thr_o = O.candidates(cube, T, mode)
    scores = torch.empty(cube.shape[1], cube.shape[2], dtype=torch.float64, device="cuda")
    thr, boxes, n = toi.tlisi_candidates(torch.from_numpy(cube).cuda(), T, mode, max_boxes=4096,
                                         scores=scores)
    assert np.array_equal(scores.cpu().numpy(), thr_o["scores"]), "scores differ in some bit"
    assert thr == thr_o["threshold"]
    assert n == len(thr_o["boxes"])
    assert boxes == thr_o["boxes"]


@pytest.mark.parametrize("S", [1, 2, 3, 4, 37, 40, 118])
@pytest.mark.parametrize("mode", [toi.TOI_CAND_PERIODIC, toi.TOI_CAND_NONPERIODIC])
def test_candidates_bit_exact(S, mode):
    """S8 on the same cube: thresholds, scores and boxes identical in every
    bit.  Odd S, and even S with S/2 odd (frequencies paired, S/2 alone) or
    S/2 even (S/4 alone as well)."""
    rng = np.random.default_rng(S * 10 + mode)
    cube = (1.0 - np.abs(rng.normal(scale=0.03, size=(S, 16, 16)))).astype(np.float32)
    if S >= 37:
        on = (np.arange(S) % 12) < 6
        cube[on, 3, 4] -= 0.4
        cube[on, 4, 5] -= 0.35
        cube[S // 3:S // 3 + 5, 12, 1] -= 0.5
    _cand_case(cube, 32, mode)


def test_candidates_bit_exact_meerkat_tile_grid():
    """64 x 64 tiles (2048 px, T = 32) and 118 slices, planted pulsar."""
    rng = np.random.default_rng(77)
    S = 118
    cube = (1.0 - np.abs(rng.normal(scale=0.02, size=(S, 64, 64)))).astype(np.float32)
    on = (np.arange(S) % 40) < 20
    cube[on, 30, 41] -= 0.2
    _cand_case(cube, 32, toi.TOI_CAND_PERIODIC)
    _cand_case(cube, 32, toi.TOI_CAND_NONPERIODIC)


def _small_workload(n_ant, n_chan, N, n_pol, flag_frac=0.0, cell=2.0, **kw):
    w = synth.tiny_workload()
    from dataclasses import replace
    return replace(w, n_ant=n_ant, n_chan=n_chan, image_size=N, n_pol=n_pol,
                   flag_frac=flag_frac, cell_arcsec=cell, **kw)


@pytest.mark.parametrize("n_ant,n_chan,N,n_pol,weights", [
    (2, 1, 64, 1, False),       # one baseline, one channel, smallest image
    (5, 37, 64, 2, True),       # ragged channel chunk, two pols, weights
    (11, 70, 256, 4, True),     # ragged everything, 4 pols, flags below
    (16, 200, 512, 4, False),
])
def test_ragged_and_edge_shapes(n_ant, n_chan, N, n_pol, weights):
    w = _small_workload(n_ant, n_chan, N, n_pol, flag_frac=0.2 if n_chan == 70 else 0.0,
                        cell=2.0 * 128 / N)
    sn = synth.make_snapshot(w, 1, with_weights=weights)
    s = to_np(sn)
    r = O.image_snapshot(s["uvw"], s["freq"], s["vis"], s["flag"], s["weight"], N,
                         w.cell_arcsec, keep_grid=True)
    plan = plan_for(w)
    out = gpu_image(plan, to_dev(sn))
    assert out["status"] == toi.TOI_OK
    _check_geometry(out["info"], r)
    assert rel_err(plan.buffer(toi.BUF_TILTED).cpu().numpy(), r["tilted"]) < IMG_TOL
    assert rel_err(out["image"], r["image"]) < IMG_TOL
    plan.close()


def test_flag_bytes_any_nonzero_value():
    """Section 3.5 flags a sample by any nonzero flag byte.  The plane fit's
    unit-weight path (4 pols, no weights, channels a multiple of 4) counts
    flagged hands four channels at a time with a per-byte nonzero test; the
    flag bytes here take the values 0x80, 0xff, 0x7f, 0x02 and 0x01 in every
    combination of the two parallel hands and of the cross hands (which must
    not count), so each bit of that test is exercised."""
    w = _small_workload(12, 64, 256, 4, cell=1.0)
    sn = synth.make_snapshot(w, 2)
    rng = np.random.default_rng(7)
    f = sn["flag"].numpy()
    vals = np.array([0x80, 0xFF, 0x7F, 0x02, 0x01], dtype=np.uint8)
    pick = rng.random(f.shape) < 0.3
    f[:] = np.where(pick, vals[rng.integers(0, len(vals), f.shape)], 0)
    # a block of channels with both hands flagged (deselected) and one with
    # only the cross hands flagged (still selected)
    f[3, 8:16, 0] = 0x80
    f[3, 8:16, 3] = 0x01
    f[4, 20:28, 1:3] = 0xFF
    f[4, 20:28, 0] = 0
    f[4, 20:28, 3] = 0
    s = to_np(sn)
    r = O.image_snapshot(s["uvw"], s["freq"], s["vis"], s["flag"], None, w.image_size,
                         w.cell_arcsec)
    plan = plan_for(w)
    out = gpu_image(plan, to_dev(sn))
    assert out["status"] == toi.TOI_OK
    _check_geometry(out["info"], r)
    assert rel_err(out["image"], r["image"]) < IMG_TOL
    plan.close()


def test_all_flagged_reports_empty():
    w = _small_workload(6, 16, 64, 4)
    sn = synth.make_snapshot(w, 0)
    sn["flag"][:] = 1
    plan = plan_for(w)
    out = gpu_image(plan, to_dev(sn))
    assert out["status"] == toi.TOI_ERR_EMPTY
    assert np.all(out["image"] == 0)
    # the plan stays usable
    sn2 = synth.make_snapshot(w, 0)
    assert gpu_image(plan, to_dev(sn2))["status"] == toi.TOI_OK
    plan.close()


def test_cell_too_large_reports_range():
    w = _small_workload(16, 32, 64, 1, cell=60.0)
    sn = synth.make_snapshot(w, 0)
    plan = plan_for(w)
    out = gpu_image(plan, to_dev(sn))
    assert out["status"] == toi.TOI_ERR_RANGE
    plan.close()


def test_argument_errors_on_host():
    w = _small_workload(4, 8, 64, 1)
    sn = to_dev(synth.make_snapshot(w, 0))
    plan = plan_for(w)
    with pytest.raises(toi.ToiError) as e:
        plan.grid(sn["uvw"], sn["freq"], sn["vis"], n_bl=w.n_bl + 1)
    assert e.value.status == toi.TOI_ERR_ARG
    with pytest.raises(toi.ToiError):
        plan.image(slot=0)          # nothing gridded yet
    plan.grid(sn["uvw"], sn["freq"], sn["vis"])
    plan.image(slot=0)
    with pytest.raises(toi.ToiError):
        plan.image(slot=0)          # the grid was consumed
    with pytest.raises(toi.ToiError):
        plan.grid(sn["uvw"], sn["freq"], sn["vis"], slot=3)
    plan.close()


# ------------------------------------------------------ full MeerKAT shape --

@pytest.fixture(scope="module")
def meerkat_snap():
    w = synth.meerkat_workload()
    return w, synth.make_snapshot(w, 5)


def test_meerkat_geometry_and_sampled_pixels(meerkat_snap):
    """2016 baselines x 4096 channels x 4 pols, 2048^2 image: the plane fit
    matches the oracle and 48 sampled tilted-image pixels match the exact
    dirty image of Section 3.2 evaluated by brute force."""
    w, sn = meerkat_snap
    s = to_np(sn)
    p = O.prepare(s["uvw"], s["freq"], s["vis"], s["flag"], None)
    plan = plan_for(w)
    out = gpu_image(plan, to_dev(sn))
    assert out["status"] == toi.TOI_OK
    _check_geometry(out["info"], p)
    tilted = plan.buffer(toi.BUF_TILTED).cpu().numpy()
    N = w.image_size
    rng = np.random.default_rng(3)
    pk = np.unravel_index(np.argmax(np.abs(tilted)), tilted.shape)
    pix = [(int(a), int(b)) for a, b in rng.integers(0, N, size=(46, 2))] + [pk, (N // 2, N // 2)]
    beta = w.cell_arcsec * O.ARCSEC
    vals, exact = [], []
    for (j2, j1) in pix:
        t1 = -beta * (j1 - N // 2)
        t2 = beta * (j2 - N // 2)
        ph = 2 * np.pi * (p["r"][:, 0] * t1 + p["r"][:, 1] * t2)
        exact.append((p["c"] * np.exp(1j * ph)).sum().real / (p["omega"] * p["sumw"]))
        vals.append(tilted[j2, j1])
    peak = np.abs(tilted).max()
    assert np.abs(np.array(vals) - np.array(exact)).max() < IMG_TOL * peak
    plan.close()


@pytest.mark.slow
def test_meerkat_full_image_vs_oracle(meerkat_snap):
    """Whole 2048^2 final image of one MeerKAT-shaped snapshot vs the oracle."""
    w, sn = meerkat_snap
    s = to_np(sn)
    r = O.image_snapshot(s["uvw"], s["freq"], s["vis"], s["flag"], None, w.image_size,
                         w.cell_arcsec)
    plan = plan_for(w)
    out = gpu_image(plan, to_dev(sn))
    assert rel_err(plan.buffer(toi.BUF_TILTED).cpu().numpy(), r["tilted"]) < IMG_TOL
    assert rel_err(out["image"], r["image"]) < IMG_TOL
    plan.close()
