"""Host-side extent checks of the binding.  The C calls take bare addresses,
so a tensor smaller than the layout include/toi.h documents is refused with
TOI_ERR_ARG before any launch (a kernel would otherwise read or write past
its end).  Counts the library itself rejects (above the plan's maxima) are
left to its own checks.  Runs on the CPU: every check comes before the
library is called, on a Plan whose extents are set without a device."""
import pytest
import torch

import paper_2512_06254_gb300 as toi
from paper_2512_06254_gb300.binding import Plan, ToiError

N, T, NBL, NCH, NPOL = 64, 16, 10, 8, 4


def _plan(half=False, batch_max=4):
    p = object.__new__(Plan)
    p.N, p.T, p._torch, p.handle = N, T, torch, None
    p._generation = [0]
    p._set_extents(NBL, NCH, NPOL, toi.TOI_VIS_C16_CHANSCALE if half else toi.TOI_VIS_C64,
                   batch_max)
    return p


def _inputs(nbl=NBL, nch=NCH):
    return dict(uvw=torch.zeros(nbl, 3, dtype=torch.float64),
                freq=torch.zeros(nch, dtype=torch.float64),
                vis=torch.zeros(nbl, nch, NPOL, dtype=torch.complex64),
                flag=torch.zeros(nbl, nch, NPOL, dtype=torch.uint8),
                weight=torch.zeros(nbl, nch, NPOL, dtype=torch.float32))


def _refused(fn, name):
    with pytest.raises(ToiError) as e:
        fn()
    assert e.value.status == toi.TOI_ERR_ARG and name in str(e.value)


def _passes_extent_checks(fn):
    """The call gets past the extent checks: what stops it on the CPU is the
    device check or the missing device, never a TOI_ERR_ARG from the binding."""
    with pytest.raises(Exception) as e:
        fn()
    assert not isinstance(e.value, ToiError), e.value


def test_grid_inputs_must_cover_their_layouts():
    p = _plan()
    d = _inputs()
    _passes_extent_checks(lambda: p.grid(**d))
    for key, short in (("uvw", torch.zeros(NBL, dtype=torch.float64)),
                       ("vis", torch.zeros(NBL, NCH, 2, dtype=torch.complex64)),
                       ("flag", torch.zeros(NBL * NCH * NPOL - 1, dtype=torch.uint8)),
                       ("weight", torch.zeros(NBL, NCH, dtype=torch.float32))):
        bad = dict(d, **{key: short})
        _refused(lambda: p.grid(**bad), key)
    # n_bl and n_ch given explicitly set the extents too (otherwise they are
    # the lengths of uvw and freq)
    _refused(lambda: p.grid(**dict(_inputs(nbl=4), n_bl=5)), "uvw")
    _refused(lambda: p.grid(**dict(d, freq=torch.zeros(NCH - 1, dtype=torch.float64), n_ch=NCH)),
             "freq")
    # counts above the plan's maxima go to the library's own check
    _passes_extent_checks(lambda: p.grid(**dict(d, n_bl=NBL + 1)))


def test_fp16_visibilities_take_four_bytes_a_record():
    p = _plan(half=True)
    d = _inputs()
    d["vis"] = torch.zeros(NBL, NCH, NPOL, 2, dtype=torch.float16)
    d["chan_scale"] = torch.ones(NCH, dtype=torch.float32)
    _passes_extent_checks(lambda: p.grid(**d))
    _refused(lambda: p.grid(**dict(d, vis=torch.zeros(NBL, NCH, NPOL, dtype=torch.float16))), "vis")
    _refused(lambda: p.grid(**dict(d, chan_scale=torch.ones(NCH - 2))), "chan_scale")


def test_image_and_tlisi_outputs():
    p = _plan()
    _refused(lambda: p.image(0, torch.zeros(N, N - 1)), "image")
    _refused(lambda: p.image(0, None, torch.zeros(15, dtype=torch.float64)), "snap_info")
    _refused(lambda: p.tlisi_update(None, torch.zeros(N // T, N // T - 1)), "tlisi")
    _refused(lambda: p.tlisi_update(torch.zeros(N - 1, N), None), "image")
    _passes_extent_checks(lambda: p.image(0, torch.zeros(N, N), torch.zeros(16, dtype=torch.float64)))


def test_reverse_mode_outputs_follow_the_slots_last_grid():
    p = _plan()
    g = torch.zeros(N, N)
    # nothing gridded through this object yet: only the image extents are known
    _passes_extent_checks(lambda: p.degrid_backward(g, grad_sample=torch.zeros(1, dtype=torch.complex64)))
    p._slot_dims[0] = (NBL, NCH)
    _refused(lambda: p.degrid_backward(g, grad_sample=torch.zeros(NBL, NCH - 1, dtype=torch.complex64)),
             "grad_sample")
    _refused(lambda: p.degrid_backward(g, grad_vis=torch.zeros(NBL, NCH, 1, dtype=torch.complex64)),
             "grad_vis")
    _refused(lambda: p.degrid_backward(g, image=g, grad_weight=torch.zeros(NBL, NCH, NPOL - 1)),
             "grad_weight")
    _refused(lambda: p.degrid_backward(torch.zeros(N, 2)), "grad_image")
    _passes_extent_checks(lambda: p.degrid_backward(
        g, image=g, grad_sample=torch.zeros(NBL, NCH, dtype=torch.complex64),
        grad_vis=torch.zeros(NBL, NCH, NPOL, dtype=torch.complex64),
        grad_weight=torch.zeros(NBL, NCH, NPOL)))


def test_localisation_arguments():
    p = _plan()
    p._slot_dims[0] = (NBL, NCH)
    row = torch.zeros(N // T, N // T)
    win = torch.zeros(3, 2, dtype=torch.int32)
    src = torch.zeros(3, 3, dtype=torch.float64)
    _refused(lambda: p.localise_seed(row, 4, win=win, src=torch.zeros(4, 3, dtype=torch.float64)),
             "win")
    _refused(lambda: p.localise_seed(row[:1], 3, win=win, src=src), "tlisi")
    _refused(lambda: p.localise(win, src[:2]), "src")
    _refused(lambda: p.localise(win, src, model=torch.zeros(3, 32, 31)), "model")
    _refused(lambda: p.localise(win, src, loss=torch.zeros(2, dtype=torch.float64)), "loss")
    _refused(lambda: p.localise(win, src, grad_weight=torch.zeros(NBL, NCH)), "grad_weight")
    _passes_extent_checks(lambda: p.localise(win, src, model=torch.zeros(3, 32, 32),
                                             loss=torch.zeros(3, dtype=torch.float64),
                                             grad_src=torch.zeros(3, 3, dtype=torch.float64)))


def test_batch_snapshots_and_rows():
    p = _plan(batch_max=4)
    snaps = [dict(_inputs(), image=torch.zeros(N, N)) for _ in range(3)]
    rows = torch.zeros(3, N // T, N // T)
    _passes_extent_checks(lambda: p.batch(snaps, rows))
    _refused(lambda: p.batch(snaps, rows[:2]), "tlisi")
    short = [snaps[0], dict(snaps[1], image=torch.zeros(N, 8)), snaps[2]]
    _refused(lambda: p.batch(short, rows), "snapshot 1: image")
    short = [snaps[0], snaps[1], dict(snaps[2], flag=torch.zeros(NBL, NCH, dtype=torch.uint8))]
    _refused(lambda: p.batch_prepare(short, rows), "snapshot 2: flag")
    # more snapshots than batch_max, or raw row addresses: the library decides
    _passes_extent_checks(lambda: p.batch(snaps * 2, rows))
    _passes_extent_checks(lambda: p.batch(snaps, 12345))
