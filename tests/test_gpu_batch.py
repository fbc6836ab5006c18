"""Batched uneven snapshots (toi_batch_*, toi_autotune) through the C ABI
against the FP64 oracle on the same seeded inputs: per-snapshot channel
counts (contiguous sub-bands), flag fractions 0-60 %, weights, batches
smaller than batch_max, the image stream and tLISI continuing across
batches, a CUDA graph captured once and replayed for later batches, and the
autotuner leaving the stream untouched."""
from dataclasses import replace

import numpy as np
import pytest
import torch

import paper_2512_06254_gb300 as toi
from oracle import toi_oracle as O
from paper_2512_06254_gb300 import synth

from gpu_helpers import rel_err, to_np

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5
T_TILE = 16


def _stream(n_snap, N=128, seed=5):
    base = replace(synth.tiny_workload(), n_ant=14, n_chan=96, n_pol=4, image_size=N,
                   n_snap=n_snap)
    ws = synth.uneven_stream(base, n_snap, seed=seed, channel_choices=(24, 48, 96),
                             flag_max=0.6, image_sizes=(N,))
    snaps = []
    for s, w in enumerate(ws):
        sn = synth.make_snapshot(w, s, with_weights=(s % 3 == 1))
        snaps.append((w, sn))
    return base, snaps


def _oracle_images(snaps):
    out = []
    for w, sn in snaps:
        h = to_np(sn)
        out.append(O.image_snapshot(h["uvw"], h["freq"], h["vis"], h["flag"], h["weight"],
                                    w.image_size, w.cell_arcsec)["image"])
    return out


def _dev_snap(sn, N):
    d = {k: (v.cuda() if v is not None else None) for k, v in sn.items()}
    d["image"] = torch.empty(N, N, dtype=torch.float32, device="cuda")
    return d


def _plan(base, B, **kw):
    return toi.Plan(base.image_size, base.cell_arcsec, base.n_bl, base.n_chan, base.n_pol,
                    tlisi_tile=T_TILE, batch_max=B, **kw)


def _check_stream(imgs, tl, first_valids, batches, ref):
    """Images equal the oracle's; tLISI rows equal the oracle's tLISI on the
    oracle images for every three-image window."""
    for i, im in enumerate(imgs):
        assert rel_err(im, ref[i]) < IMG_TOL, i
    t = 0
    for (lo, hi), fv, rows in zip(batches, first_valids, tl):
        assert fv == max(0, min(2 - lo, hi - lo))
        for j in range(fv, hi - lo):
            s = lo + j
            exp = O.tlisi(ref[s - 2], ref[s - 1], ref[s], T_TILE)
            assert np.abs(rows[j] - exp).max() < 1e-4, s
        t += hi - lo


def test_uneven_batches_match_oracle():
    base, snaps = _stream(11)
    ref = _oracle_images(snaps)
    N = base.image_size
    nt = N // T_TILE
    B = 4
    plan = _plan(base, B)
    batches = [(0, 4), (4, 7), (7, 11)]            # 4, 3 (< batch_max), 4
    imgs, tl, fvs = [], [], []
    for lo, hi in batches:
        ds = [_dev_snap(sn, N) for _, sn in snaps[lo:hi]]
        rows = torch.full((hi - lo, nt, nt), -1.0, device="cuda")
        fvs.append(plan.batch(ds, rows))
        assert plan.sync_status() == toi.TOI_OK
        imgs += [d["image"].cpu().numpy() for d in ds]
        tl.append(rows.cpu().numpy())
    _check_stream(imgs, tl, fvs, batches, ref)
    # rows without a window are left untouched
    assert np.all(tl[0][:2] == -1.0)
    plan.close()


def test_batch_equals_single_path():
    """Images to 1e-6 (the two gridders sum in different orders); tLISI to
    5e-5: it is made from differences of consecutive images, about a tenth
    of their peak, so the images' float32 rounding weighs ~10x more there."""
    base, snaps = _stream(6, seed=9)
    N = base.image_size
    nt = N // T_TILE
    single = _plan(base, 0)
    out_single, tl_single = [], []
    row = torch.empty(nt, nt, device="cuda")
    for w, sn in snaps:
        d = _dev_snap(sn, N)
        single.grid(d["uvw"], d["freq"], d["vis"], flag=d["flag"], weight=d["weight"])
        single.image(0, d["image"])
        v = single.tlisi_update(None, row)
        out_single.append(d["image"].cpu().numpy())
        tl_single.append(row.cpu().numpy() if v else None)
    single.close()
    plan = _plan(base, 6)
    ds = [_dev_snap(sn, N) for _, sn in snaps]
    rows = torch.empty(6, nt, nt, device="cuda")
    assert plan.batch(ds, rows) == 2
    for i, d in enumerate(ds):
        a = d["image"].cpu().numpy()
        assert rel_err(a, out_single[i]) < 1e-6
        if tl_single[i] is not None:
            assert np.abs(rows[i].cpu().numpy() - tl_single[i]).max() < 5e-5
    plan.close()


def test_graph_captured_once_replays_later_batches():
    base, snaps = _stream(10, seed=13)
    ref = _oracle_images(snaps)
    N = base.image_size
    nt = N // T_TILE
    B = 4
    stream = torch.cuda.Stream()
    plan = _plan(base, B, stream=stream)
    batches = [(0, 4), (4, 8), (8, 10)]
    imgs, tl, fvs = [], [], []
    graph = None
    for lo, hi in batches:
        ds = [_dev_snap(sn, N) for _, sn in snaps[lo:hi]]
        rows = torch.full((hi - lo, nt, nt), -1.0, device="cuda")
        torch.cuda.synchronize()
        fvs.append(plan.batch_prepare(ds, rows))
        if graph is None:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                plan.batch_run()
        with torch.cuda.stream(stream):
            graph.replay()
        stream.synchronize()
        assert plan.sync_status() == toi.TOI_OK
        imgs += [d["image"].cpu().numpy() for d in ds]
        tl.append(rows.cpu().numpy())
    _check_stream(imgs, tl, fvs, batches, ref)
    plan.close()


def test_autotune_keeps_the_stream():
    base, snaps = _stream(7, seed=17)
    ref = _oracle_images(snaps)
    N = base.image_size
    nt = N // T_TILE
    plan = _plan(base, 4)
    ds0 = [_dev_snap(sn, N) for _, sn in snaps[:3]]
    rows0 = torch.empty(3, nt, nt, device="cuda")
    plan.batch(ds0, rows0)
    runs, us = plan.autotune([_dev_snap(sn, N) for _, sn in snaps[3:7]])
    assert runs and all(r in (16, 32, 64, 128, 256) for r in runs.values())
    assert all(v > 0 for v in us.values())
    ds1 = [_dev_snap(sn, N) for _, sn in snaps[3:7]]
    rows1 = torch.empty(4, nt, nt, device="cuda")
    assert plan.batch(ds1, rows1) == 0
    assert plan.sync_status() == toi.TOI_OK
    imgs = [d["image"].cpu().numpy() for d in ds0 + ds1]
    _check_stream(imgs, [rows0.cpu().numpy(), rows1.cpu().numpy()], [2, 0],
                  [(0, 3), (3, 7)], ref)
    plan.close()


def test_batch_argument_errors():
    base, snaps = _stream(3, seed=21)
    N = base.image_size
    ds = [_dev_snap(sn, N) for _, sn in snaps]
    p0 = _plan(base, 0)
    with pytest.raises(toi.ToiError) as e:
        p0.batch(ds[:1])
    assert e.value.status == toi.TOI_ERR_ARG
    p0.close()
    p = _plan(base, 2)
    with pytest.raises(toi.ToiError) as e:
        p.batch(ds)                                  # 3 > batch_max
    assert e.value.status == toi.TOI_ERR_ARG
    with pytest.raises(toi.ToiError) as e:
        p.batch_run()                                # nothing prepared
    assert e.value.status == toi.TOI_ERR_ARG
    bad = dict(ds[0])
    bad["freq"] = torch.linspace(1.0e9, 1.1e9, base.n_chan + 1, dtype=torch.float64,
                                 device="cuda")          # more channels than max_channels
    with pytest.raises(toi.ToiError) as e:
        p.batch([ds[1], bad])
    assert e.value.status == toi.TOI_ERR_ARG and "snapshot 1" in str(e.value)
    p.close()
