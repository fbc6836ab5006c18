"""Periodic candidate search end to end on an 82-snapshot MeerKAT-array
stream (Sections 2 and 6.2): the 64-antenna array (2016 baselines) with 32
channels over 856-1712 MHz, 2048^2 images of 2 arcsec, so 64 x 64 tLISI tiles
of 32 px, with the power-law steady sources and the 1 Jy pulsar of period 40
(on for 20), imaged by the batched engine in batches of 16.

As in the short end-to-end test: the GPU's S8 on the GPU cube is bit-identical
to the oracle's S8 on that cube, and the candidate tiles and boxes of the GPU
pipeline equal those of the FP64 oracle pipeline, with the smallest distance
of an oracle z-score from its threshold larger than the largest z-score
difference between the pipelines.  The 82 oracle images come from a spawn
pool over the host cores."""
import numpy as np
import pytest
import torch

import paper_2512_06254_gb300 as toi
from oracle import toi_oracle as O
from paper_2512_06254_gb300 import synth

from oracle_pool import Job, oracle_images

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

T = 32
S = 82
B = 16


def stream():
    return synth.meerkat_workload(n_snap=S, n_chan=32)


def oracle_cube(w):
    imgs = [r["image"] for r in oracle_images([Job(w, s) for s in range(S)])]
    return np.stack([O.tlisi(imgs[i - 2], imgs[i - 1], imgs[i], T) for i in range(2, S)])


@pytest.fixture(scope="module")
def cubes():
    w = stream()
    cube_o = oracle_cube(w)
    nt = w.image_size // T
    plan = toi.Plan(w.image_size, w.cell_arcsec, w.n_bl, w.n_chan, w.n_pol, tlisi_tile=T,
                    batch_max=B)
    cube_g = torch.full((S, nt, nt), -1.0, dtype=torch.float32, device="cuda")
    for lo in range(0, S, B):
        hi = min(S, lo + B)
        snaps = [{k: (v.cuda() if v is not None else None)
                  for k, v in synth.make_snapshot(w, s).items()} for s in range(lo, hi)]
        plan.batch(snaps, cube_g[lo:hi])
        assert plan.sync_status() == toi.TOI_OK, plan.last_error()
    torch.cuda.synchronize()
    plan.close()
    # row t of the batch output holds the tLISI of image t (t >= 2)
    return cube_o, cube_g[2:].contiguous()


@pytest.mark.parametrize("mode,k", [(toi.TOI_CAND_PERIODIC, 5.0),
                                    (toi.TOI_CAND_NONPERIODIC, 4.0)])
def test_long_stream_candidates(cubes, mode, k):
    cube_o, cube_g = cubes
    nt = cube_o.shape[1]
    assert float(np.abs(cube_g.cpu().numpy() - cube_o).max()) < 1e-4
    scores_g = torch.empty(nt, nt, dtype=torch.float64, device="cuda")
    thr_g, boxes_g, n_g = toi.tlisi_candidates(cube_g, T, mode, max_boxes=4096, scores=scores_g)
    ref_on_g = O.candidates(cube_g.cpu().numpy(), T, mode)
    sg = scores_g.cpu().numpy()
    assert np.array_equal(sg, ref_on_g["scores"]) and thr_g == ref_on_g["threshold"]
    assert n_g == len(ref_on_g["boxes"]) and boxes_g == ref_on_g["boxes"]
    ref = O.candidates(cube_o, T, mode)
    z_o = (ref["scores"] - ref["mean"]) / ref["std"]
    z_g = (sg - ref_on_g["mean"]) / ref_on_g["std"]
    dz = float(np.abs(z_g - z_o).max())
    gap = np.abs(z_o - k)
    worst = tuple(int(a) for a in np.unravel_index(np.argmin(gap), gap.shape))
    print(f"mode {mode}: {int(ref['mask'].sum())} candidate tiles, {len(ref['boxes'])} boxes, "
          f"max |dz| {dz:.2e}, min |z - {k:g}| {gap.min():.3f} at tile {worst}")
    assert ref["mask"].any(), "the pulsar must be found"
    assert gap.min() > dz, f"tile {worst} is within max |dz| = {dz:.2e} of the threshold"
    assert np.array_equal(sg > thr_g, ref["mask"])
    assert boxes_g == ref["boxes"]
