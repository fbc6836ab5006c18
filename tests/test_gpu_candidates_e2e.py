"""End-to-end candidates: the GPU pipeline (S1-S7 in FP32 through the C ABI,
then S8 on its own tLISI cube) against the oracle pipeline (S1-S7 in FP64,
then S8), on a seeded stream with a transient window and a pulsar.

FP32 images cannot match FP64 images bit for bit, so two things are checked.
First, the GPU's S8 on the GPU cube is bit-identical to the oracle's S8 on
that same cube: scores, threshold and boxes.  Second, the candidate tile sets
of the two pipelines are equal.  Each mode also reports the largest z-score
difference between the pipelines, max |dz|, and the smallest distance of an
oracle z-score from its threshold, min |z - k|.  The test requires the margin
to exceed max |dz|, so that equal sets are not luck; a failure names the tile
that sits closest to the threshold.  The detection rules are those of
Sections 2, 6.2 and 6.3."""
from dataclasses import replace

import numpy as np
import pytest
import torch

import paper_2512_06254_gb300 as toi
from oracle import toi_oracle as O
from paper_2512_06254_gb300 import synth

from gpu_helpers import gpu_image, plan_for, to_dev, to_np

pytestmark = pytest.mark.gpu

T = 16


def _stream():
    """The MeerKAT array with 16 channels, 256^2 pixels of 2 arcsec and 26
    snapshots: the steady power-law sources, a 0.3 Jy transient on in
    snapshots 9-12 and a 0.3 Jy pulsar with period 8 (on for 4)."""
    base = synth.meerkat_workload(n_snap=26, n_chan=16, image_size=256)
    steady = [s for s in base.sources if s.kind == "steady"]
    l1, m1 = synth.random_position(base.fov_rad, base.seed_sky + 300)
    l2, m2 = synth.random_position(base.fov_rad, base.seed_sky + 301)
    src = steady + [synth.Source(l1, m1, 0.3, kind="window", on_from=9, on_to=13),
                    synth.Source(l2, m2, 0.3, kind="periodic", period=8, duty=4)]
    return replace(base, sources=tuple(src))


def _z(scores, mean, std):
    return (np.asarray(scores, np.float64) - mean) / std


@pytest.fixture(scope="module")
def cubes():
    w = _stream()
    snaps = [synth.make_snapshot(w, s) for s in range(w.n_snap)]
    imgs = []
    for sn in snaps:
        h = to_np(sn)
        imgs.append(O.image_snapshot(h["uvw"], h["freq"], h["vis"], h["flag"], h["weight"],
                                     w.image_size, w.cell_arcsec)["image"])
    cube_o = np.stack([O.tlisi(imgs[i - 2], imgs[i - 1], imgs[i], T)
                       for i in range(2, len(imgs))])
    plan = plan_for(w, tlisi_tile=T)
    nt = w.image_size // T
    cube_g = torch.empty(w.n_snap - 2, nt, nt, dtype=torch.float32, device="cuda")
    row = torch.empty(nt, nt, dtype=torch.float32, device="cuda")
    for i, sn in enumerate(snaps):
        assert gpu_image(plan, to_dev(sn), out=False)["status"] == toi.TOI_OK
        if plan.tlisi_update(None, row):
            cube_g[i - 2].copy_(row)
    torch.cuda.synchronize()
    plan.close()
    return cube_o, cube_g


@pytest.mark.parametrize("mode,k", [(toi.TOI_CAND_PERIODIC, 5.0),
                                    (toi.TOI_CAND_NONPERIODIC, 4.0)])
def test_candidates_end_to_end(cubes, mode, k):
    cube_o, cube_g = cubes
    nt = cube_o.shape[1]
    # (i) the GPU's S8 on the GPU cube, bit for bit against the oracle's S8
    scores_g = torch.empty(nt, nt, dtype=torch.float64, device="cuda")
    thr_g, boxes_g, n_g = toi.tlisi_candidates(cube_g, T, mode, max_boxes=1024, scores=scores_g)
    ref_on_g = O.candidates(cube_g.cpu().numpy(), T, mode)
    sg = scores_g.cpu().numpy()
    assert np.array_equal(sg, ref_on_g["scores"]) and thr_g == ref_on_g["threshold"]
    assert n_g == len(ref_on_g["boxes"]) and boxes_g == ref_on_g["boxes"]
    # (ii) the two pipelines: equal candidate sets, with a margin above |dz|
    ref = O.candidates(cube_o, T, mode)
    z_o = _z(ref["scores"], ref["mean"], ref["std"])
    z_g = _z(sg, ref_on_g["mean"], ref_on_g["std"])
    dz = float(np.abs(z_g - z_o).max())
    gap = np.abs(z_o - k)
    worst = tuple(int(a) for a in np.unravel_index(np.argmin(gap), gap.shape))
    print(f"mode {mode}: {int(ref['mask'].sum())} candidate tiles, max |dz| {dz:.2e}, "
          f"min |z - {k:g}| {gap.min():.3f} at tile {worst}")
    assert ref["mask"].any(), "the stream must give candidates"
    assert gap.min() > dz, f"tile {worst} is within max |dz| = {dz:.2e} of the threshold"
    assert np.array_equal(sg > thr_g, ref["mask"]), \
        f"candidate tiles differ: {np.argwhere((sg > thr_g) != ref['mask']).tolist()}"
    assert boxes_g == ref["boxes"]
