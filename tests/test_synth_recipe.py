"""The seeded inputs follow the stated recipe of the paper's workloads (the
stand-ins for its Measurement Sets): array size and extent, band, polarisation
structure, flag fraction, the transient and pulsar schedules, Earth-rotation
geometry and determinism.  CPU only; reduced channel counts where the
property does not depend on them."""
import math
from dataclasses import replace

import numpy as np
import torch

from paper_2512_06254_gb300 import synth


def _enu_dist(enu):
    d = enu[:, None, :2] - enu[None, :, :2]
    return torch.sqrt((d * d).sum(-1))


def test_meerkat_array():
    """64 antennas (2016 baselines): 48 in a 1 km core, arms out to 4 km, so
    the longest baseline is close to (and not over) 8 km."""
    w = synth.meerkat_workload()
    enu = synth.array_layout(w)
    assert enu.shape == (64, 3) and w.n_bl == 2016
    r = torch.sqrt(enu[:, 0] ** 2 + enu[:, 1] ** 2)
    assert int((r <= 1000.0).sum()) >= 48
    assert float(r.max()) <= 4000.0 + 1e-6
    longest = float(_enu_dist(enu).max())
    assert 6000.0 < longest <= 8000.0


def test_meerkat_band_and_layouts():
    w = synth.meerkat_workload()
    f = synth.frequencies(w)
    assert f.shape == (4096,) and f[0] == 856e6
    step = (1712e6 - 856e6) / 4096
    assert torch.allclose(f[1:] - f[:-1], torch.full((4095,), step, dtype=torch.float64))
    sn = synth.make_snapshot(replace(w, n_chan=64), 0, with_weights=True)
    assert sn["uvw"].shape == (2016, 3) and sn["uvw"].dtype == torch.float64
    assert sn["vis"].shape == (2016, 64, 4) and sn["vis"].dtype == torch.complex64
    assert sn["flag"].shape == (2016, 64, 4) and sn["flag"].dtype == torch.uint8
    assert sn["weight"].shape == (2016, 64, 4) and float(sn["weight"].min()) > 0.0


def test_linear_feeds_and_flag_fraction():
    """XX = YY = I and XY = YX = 0 without noise; 5% i.i.d. flags."""
    w = replace(synth.meerkat_workload(n_chan=64), noise_sigma=0.0)
    v = synth.make_snapshot(w, 3)["vis"]
    assert torch.equal(v[:, :, 0], v[:, :, 3]) and float(v[:, :, 0].abs().max()) > 0.0
    assert float(v[:, :, 1].abs().max()) == 0.0 and float(v[:, :, 2].abs().max()) == 0.0
    flag = synth.make_snapshot(synth.meerkat_workload(n_chan=64), 3)["flag"]
    frac = float(flag.double().mean())
    sigma = math.sqrt(0.05 * 0.95 / flag.numel())
    assert abs(frac - 0.05) < 6 * sigma


def test_pulsar_and_transient_schedules():
    """The MeerKAT pulsar is on for 20 of every 40 snapshots; the tiny
    stream's transient is on in snapshots 3-5 only."""
    w = synth.meerkat_workload(n_chan=8)
    pulsar = [s for s in w.sources if s.kind == "periodic"]
    assert len(pulsar) == 1 and pulsar[0].flux == 1.0
    only = replace(w, sources=tuple(pulsar), noise_sigma=0.0, flag_frac=0.0)
    for s, on in ((0, True), (19, True), (20, False), (39, False), (40, True)):
        peak = float(synth.make_snapshot(only, s)["vis"].abs().max())
        assert (peak > 0.5) == on, s
    t = synth.tiny_workload()
    assert t.n_bl == 120 and t.n_chan == 64 and t.n_pol == 1 and t.image_size == 128
    tr = [s for s in t.sources if s.kind == "window"]
    assert len(tr) == 1
    assert [tr[0].flux_at(s, t.n_snap) > 0 for s in range(t.n_snap)] == \
        [False, False, False, True, True, True, False, False]


def test_earth_rotation_preserves_baseline_lengths():
    """UVW of a snapshot is the baseline rotated toward the source at that
    hour angle: its length equals the antenna separation, and it changes
    between snapshots 8 s apart."""
    w = synth.meerkat_workload(n_chan=4)
    enu = synth.array_layout(w)
    i, j = torch.triu_indices(64, 64, 1)
    length = torch.linalg.norm(enu[j] - enu[i], dim=1)
    u0 = synth.make_snapshot(w, 0)["uvw"]
    u9 = synth.make_snapshot(w, 9)["uvw"]
    for u in (u0, u9):
        assert torch.allclose(torch.linalg.norm(u, dim=1), length, rtol=1e-12, atol=0)
    assert float((u9 - u0).abs().max()) > 1.0


def test_seeded_and_reproducible():
    w = synth.meerkat_workload(n_chan=16)
    a = synth.make_snapshot(w, 5)
    b = synth.make_snapshot(w, 5)
    c = synth.make_snapshot(w, 6)
    for k in ("uvw", "freq", "vis", "flag"):
        assert torch.equal(a[k], b[k]), k
    assert not torch.equal(a["vis"], c["vis"]) and not torch.equal(a["flag"], c["flag"])
    # the noise is complex Gaussian with the stated sigma per part
    quiet = replace(w, sources=())
    n = torch.view_as_real(synth.make_snapshot(quiet, 2)["vis"]).double()
    assert abs(float(n.std()) - 0.1) < 0.002 and abs(float(n.mean())) < 0.002
    assert np.isfinite(n.numpy()).all()
