"""The native streaming runtime (toi_stream_*: one CUDA stream per pipeline
stage, depth-3 grid ring, depth-5 image ring, host tLISI row ring) against
the FP64 oracle on the same seeded host snapshots (uneven channel counts,
flags and weights), and its host-side protocols (row ring, input buffers)."""
from dataclasses import replace

import numpy as np
import pytest
import torch

import paper_2512_06254_gb300 as toi
from oracle import toi_oracle as O
from paper_2512_06254_gb300 import synth

from gpu_helpers import to_np

pytestmark = pytest.mark.gpu

T_TILE = 16


def _stream(n_snap, N=128, seed=7):
    base = replace(synth.tiny_workload(), n_ant=14, n_chan=96, n_pol=4, image_size=N,
                   n_snap=n_snap)
    ws = synth.uneven_stream(base, n_snap, seed=seed, channel_choices=(24, 48, 96),
                             flag_max=0.6, image_sizes=(N,))
    return base, [(w, synth.make_snapshot(w, s, with_weights=(s % 3 == 1)))
                  for s, w in enumerate(ws)]


def _pinned(sn):
    return {k: (v.pin_memory() if v is not None else None) for k, v in sn.items()}


def _plan(base):
    return toi.Plan(base.image_size, base.cell_arcsec, base.n_bl, base.n_chan, base.n_pol,
                    tlisi_tile=T_TILE, grid_slots=3)


def test_stream_rows_match_oracle():
    base, snaps = _stream(11)
    ref = []
    for w, sn in snaps:
        h = to_np(sn)
        ref.append(O.image_snapshot(h["uvw"], h["freq"], h["vis"], h["flag"], h["weight"],
                                    w.image_size, w.cell_arcsec)["image"])
    plan = _plan(base)
    st = toi.Stream(plan, host_depth=4, n_copy=3, with_weights=True)
    rows = {}
    for _, sn in snaps:
        st.push(_pinned(sn))
        while (r := st.pop(wait=False)) is not None:
            rows[r[0]] = r[1].numpy().copy()
    while (r := st.pop(wait=True)) is not None:
        rows[r[0]] = r[1].numpy().copy()
    assert st.input_free(len(snaps) - 1, wait=True)
    st.close()
    plan.close()
    assert sorted(rows) == list(range(len(snaps) - 2))
    for r, row in rows.items():
        exp = O.tlisi(ref[r], ref[r + 1], ref[r + 2], T_TILE)
        assert np.abs(row - exp).max() < 1e-4, r


def test_stream_equals_single_path():
    base, snaps = _stream(6, seed=19)
    nt = base.image_size // T_TILE
    plan = _plan(base)
    single = []
    row = torch.empty(nt, nt, device="cuda")
    for _, sn in snaps:
        d = {k: (v.cuda() if v is not None else None) for k, v in sn.items()}
        plan.grid(d["uvw"], d["freq"], d["vis"], flag=d["flag"], weight=d["weight"])
        plan.image(0, None)
        if plan.tlisi_update(None, row):
            single.append(row.cpu().numpy().copy())
    st = toi.Stream(plan, host_depth=8, n_copy=2, with_weights=True)
    for _, sn in snaps:
        st.push(_pinned(sn))
    got = []
    while (r := st.pop(wait=True)) is not None:
        got.append(r[1].numpy().copy())
    st.close()
    plan.close()
    assert len(got) == len(single) == len(snaps) - 2
    for a, b in zip(got, single):
        assert np.abs(a - b).max() < 5e-5


def test_stream_host_ring_and_arguments():
    base, snaps = _stream(6, seed=23)
    plan = _plan(base)
    st = toi.Stream(plan, host_depth=2, n_copy=1, with_weights=True)
    for _, sn in snaps[:4]:
        st.push(_pinned(sn))                   # rows 0 and 1 fill the host ring
    with pytest.raises(toi.ToiError) as e:
        st.push(_pinned(snaps[4][1]))          # would overwrite row 0, not popped
    assert e.value.status == toi.TOI_ERR_ARG and "pop" in str(e.value)
    r0 = st.pop(wait=True)
    assert r0[0] == 0
    st.push(_pinned(snaps[4][1]))
    with pytest.raises(ValueError):
        st.push({k: (v.cuda() if v is not None else None) for k, v in snaps[5][1].items()})
    st.close()
    plan.close()
    p1 = toi.Plan(base.image_size, base.cell_arcsec, base.n_bl, base.n_chan, base.n_pol)
    with pytest.raises(toi.ToiError) as e:
        toi.Stream(p1)                         # grid_slots = 1
    assert e.value.status == toi.TOI_ERR_ARG
    p1.close()


def _decoded(q, scale):
    """What the kernels read: scale_c x half, as complex128."""
    f = q.to(torch.float64) * scale.to(torch.float64)[None, :, None, None]
    return torch.view_as_complex(f.contiguous()).numpy()


def test_stream_fp16_visibilities():
    """Float16 visibilities with per-channel scales through the stream equal
    the oracle's images of the decoded values (tLISI rows to 1e-4)."""
    base, snaps = _stream(6, seed=29)
    plan = toi.Plan(base.image_size, base.cell_arcsec, base.n_bl, base.n_chan, base.n_pol,
                    tlisi_tile=T_TILE, grid_slots=3, vis_dtype=toi.TOI_VIS_C16_CHANSCALE)
    st = toi.Stream(plan, host_depth=8, n_copy=2, with_weights=True)
    ref = []
    for w, sn in snaps:
        q, scale = synth.to_fp16_channel_scaled(sn["vis"])
        st.push(_pinned(dict(sn, vis=q, chan_scale=scale)))
        h = to_np(sn)
        ref.append(O.image_snapshot(h["uvw"], h["freq"], _decoded(q, scale), h["flag"],
                                    h["weight"], w.image_size, w.cell_arcsec)["image"])
    rows = []
    while (r := st.pop(wait=True)) is not None:
        rows.append(r[1].numpy().copy())
    st.close()
    plan.close()
    assert len(rows) == len(snaps) - 2
    for r, row in enumerate(rows):
        exp = O.tlisi(ref[r], ref[r + 1], ref[r + 2], T_TILE)
        assert np.abs(row - exp).max() < 1e-4, r
