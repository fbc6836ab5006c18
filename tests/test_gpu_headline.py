"""The batched engine at the configuration the throughput figure is measured
on, against the FP64 oracle: MeerKAT-shaped snapshots (2016 baselines, up
to 4096 channels x 4 pols), 2048^2 images of 2 arcsec (G = 4096), a plan
with batch_max = 32 and the default lane runs (256 channels at 4096).

* One batch of six distinct snapshots: four full-band, one 2048-channel and
  one 1024-channel sub-band (30 % and 50 % flags), one with weights.  Every
  final image matches the oracle's to 1e-5 of its peak (the FP32 image
  tolerance of Section 3.2's I_D^(2) imaging), and each tLISI row (from the
  third image on) matches the oracle's tLISI of the oracle images to 1e-4.
* The same batch with the lane run forced to 16 and to 512 channels, the two
  ends of the window-slide code, against the same oracle images.
* tLISI at full size over snapshots {0, 1, 2}, {40, 41, 42} (the 40-snapshot
  pulsar on throughout) and {19, 20, 21} (it switches off), Section 2's
  three-image statistic.

The oracle images come from a spawn pool over the host cores (about 12 s of
one core per full-band snapshot)."""
from dataclasses import replace

import numpy as np
import pytest
import torch

import paper_2512_06254_gb300 as toi
from oracle import toi_oracle as O
from paper_2512_06254_gb300 import synth

from gpu_helpers import rel_err
from oracle_pool import Job, oracle_images

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

IMG_TOL = 1e-5
TLISI_TOL = 1e-4
T = 32


def _subband(base, nc, off, flag_frac):
    """A contiguous sub-band of base's channel grid (as synth.uneven_stream)."""
    step = (base.f_hi_hz - base.f_lo_hz) / base.n_chan
    f_lo = base.f_lo_hz + off * step
    return replace(base, n_chan=nc, f_lo_hz=f_lo, f_hi_hz=f_lo + nc * step,
                   flag_frac=flag_frac, name=f"{base.name}-sub-{nc}ch")


def _batch_spec():
    base = synth.meerkat_workload()
    return [
        (base, 40, False),
        (base, 41, False),
        (base, 42, False),
        (_subband(base, 2048, 1024, 0.3), 43, False),
        (_subband(base, 1024, 3072, 0.5), 44, False),
        (base, 45, True),
    ]


@pytest.fixture(scope="module")
def headline():
    spec = _batch_spec()
    early = [(spec[0][0], s, False) for s in (0, 1, 2, 19, 20, 21)]
    jobs = [Job(w, s, with_weights=wt) for (w, s, wt) in spec + early]
    ref = [r["image"] for r in oracle_images(jobs)]
    return spec, ref[:len(spec)], ref[len(spec):]


def _dev_snaps(spec):
    out = []
    for w, s, wt in spec:
        sn = synth.make_snapshot(w, s, with_weights=wt)
        d = {k: (v.cuda() if v is not None else None) for k, v in sn.items()}
        d["image"] = torch.empty(w.image_size, w.image_size, dtype=torch.float32, device="cuda")
        out.append(d)
    return out


def _plan(**kw):
    base = synth.meerkat_workload()
    return toi.Plan(base.image_size, base.cell_arcsec, base.n_bl, base.n_chan, base.n_pol,
                    tlisi_tile=T, batch_max=32, **kw)


def _run_batch(plan, ds):
    nt = plan.N // T
    rows = torch.full((len(ds), nt, nt), -1.0, device="cuda")
    fv = plan.batch(ds, rows)
    assert plan.sync_status() == toi.TOI_OK, plan.last_error()
    return fv, [d["image"].cpu().numpy() for d in ds], rows.cpu().numpy()


def test_default_lane_runs_at_meerkat_shape():
    plan = _plan()
    assert plan.lane_run(4096) == (256, 4)
    assert plan.lane_run(2048) == (128, 4)
    assert plan.lane_run(1024) == (64, 4)
    plan.close()


def test_headline_batch_matches_oracle(headline):
    spec, ref, _ = headline
    ds = _dev_snaps(spec)
    plan = _plan()
    fv, imgs, rows = _run_batch(plan, ds)
    assert fv == 2
    for i, im in enumerate(imgs):
        e = rel_err(im, ref[i])
        print(f"entry {i} ({spec[i][0].n_chan} ch): image rel err {e:.2e}")
        assert e < IMG_TOL, i
    assert np.all(rows[:2] == -1.0)
    for i in range(2, len(ds)):
        exp = O.tlisi(ref[i - 2], ref[i - 1], ref[i], T)
        d = float(np.abs(rows[i] - exp).max())
        print(f"tLISI row {i}: max abs err {d:.2e}")
        assert d < TLISI_TOL, i
    plan.close()


@pytest.mark.parametrize("run", [16, 512])
def test_headline_batch_forced_runs(headline, run):
    spec, ref, _ = headline
    ds = _dev_snaps(spec)
    plan = _plan(grid_run=run)
    assert plan.lane_run(4096)[0] == run
    _, imgs, _ = _run_batch(plan, ds)
    for i, im in enumerate(imgs):
        assert rel_err(im, ref[i]) < IMG_TOL, (run, i)
    plan.close()


def test_tlisi_full_size_pulsar_off_and_on(headline):
    """tLISI of snapshots {0,1,2} and {40,41,42} (the pulsar, on while
    s mod 40 < 20, is on in all three) and {19,20,21} (on, off, off) at 4096
    channels and 2048^2, each as its own three-image stream through the
    batched engine."""
    spec, ref, early = headline
    base = spec[0][0]
    cases = [((0, 1, 2), early[:3]), ((40, 41, 42), ref[:3]), ((19, 20, 21), early[3:])]
    for snaps, imgs_o in cases:
        ds = _dev_snaps([(base, s, False) for s in snaps])
        plan = _plan()
        fv, imgs, rows = _run_batch(plan, ds)
        assert fv == 2
        for im, ro in zip(imgs, imgs_o):
            assert rel_err(im, ro) < IMG_TOL
        exp = O.tlisi(imgs_o[0], imgs_o[1], imgs_o[2], T)
        d = float(np.abs(rows[2] - exp).max())
        print(f"snapshots {snaps}: tLISI max abs err {d:.2e}, min tLISI {exp.min():.4f}")
        assert d < TLISI_TOL
        plan.close()
