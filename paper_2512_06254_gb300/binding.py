"""ctypes binding of libtoi (include/toi.h), argument marshalling only.

Every function keeps the C name and forwards device pointers (torch CUDA
tensors or raw integers) and the current CUDA stream; all computation
happens in the library's kernels.  The binding refuses to run without the
compiled library: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "lib", "libtoi.so")

TOI_OK = 0
TOI_ERR_ARG = 1
TOI_ERR_CUDA = 2
TOI_ERR_OOM = 3
TOI_ERR_EMPTY = 4
TOI_ERR_TIMEOUT = 5
TOI_ERR_UNSUPPORTED = 6
TOI_ERR_RANGE = 7
TOI_VIS_C64 = 0
TOI_VIS_C16_CHANSCALE = 1
TOI_CAND_PERIODIC = 0
TOI_CAND_NONPERIODIC = 1
BUF_GRID, BUF_TILTED, BUF_SNAP, BUF_RING = 0, 1, 2, 3

EXPORTS = ("toi_config_default", "toi_plan", "toi_plan_destroy", "toi_set_stream", "toi_grid",
           "toi_image", "tlisi_update", "tlisi_reset", "tlisi_candidates",
           "tlisi_candidates_noalloc",
           "toi_degrid_backward", "toi_batch_prepare", "toi_batch_run", "toi_batch",
           "toi_autotune", "toi_grid_lane_run", "toi_mode3_info", "toi_localise_seed",
           "toi_localise",
           "toi_stream_open", "toi_stream_push", "toi_stream_input_free", "toi_stream_pop",
           "toi_stream_close",
           "toi_plan_buffer", "toi_profile_enable", "toi_profile_read",
           "toi_sync_status", "toi_last_error", "toi_status_string")
PROF_STAGES = ("prep", "bin", "grid", "fft_rows", "fft_cols", "reproject", "tlisi", "backward",
               "localise")
LOC_WINDOW = 32


class ToiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libtoi status {status}: {msg}")
        self.status = status


class toi_config(C.Structure):
    _fields_ = [("image_size", C.c_int32), ("cell_arcsec", C.c_double),
                ("max_baselines", C.c_int32), ("max_channels", C.c_int32),
                ("n_pol", C.c_int32), ("vis_dtype", C.c_int32), ("kernel_support", C.c_int32),
                ("oversample", C.c_int32), ("tlisi_tile", C.c_int32), ("grid_slots", C.c_int32),
                ("grid_run", C.c_int32), ("batch_max", C.c_int32), ("mode", C.c_int32),
                ("max_moments", C.c_int32), ("grid_rows", C.c_int32), ("max_windows", C.c_int32),
                ("reserved", C.c_int32 * 1)]


class toi_snapshot(C.Structure):
    _fields_ = [("uvw", C.c_void_p), ("freq", C.c_void_p), ("vis", C.c_void_p),
                ("chan_scale", C.c_void_p), ("weight", C.c_void_p), ("flag", C.c_void_p),
                ("image", C.c_void_p), ("n_bl", C.c_int32), ("n_ch", C.c_int32)]


_lib = None


def lib():
    """Load libtoi.so (built in-tree by paper_2512_06254_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2512_06254_gb300.build`")
    L = C.CDLL(LIB_PATH)
    P, I, D = C.c_void_p, C.c_int32, C.c_double
    sig = {
        "toi_config_default": [C.POINTER(toi_config), I, D, I, I, I],
        "toi_plan": [C.POINTER(toi_config), P, C.POINTER(C.c_void_p)],
        "toi_plan_destroy": [P],
        "toi_set_stream": [P, P],
        "toi_grid": [P, P, P, P, P, P, P, I, I, I],
        "toi_image": [P, I, P, P],
        "tlisi_update": [P, P, P, C.POINTER(I)],
        "tlisi_reset": [P],
        "tlisi_candidates": [P, I, I, I, I, I, P, C.POINTER(D), P, C.POINTER(I), I, P],
        "tlisi_candidates_noalloc": [P, I, I, I, I, I, P, C.POINTER(D), P, C.POINTER(I), I, P],
        "toi_degrid_backward": [P, I, P, P, P, P, P],
        "toi_batch_prepare": [P, P, I, P, C.POINTER(I)],
        "toi_batch_run": [P],
        "toi_batch": [P, P, I, P, C.POINTER(I)],
        "toi_autotune": [P, P, I, P, P],
        "toi_mode3_info": [P, I, P],
        "toi_grid_lane_run": [P, I, I, C.POINTER(I), C.POINTER(I)],
        "toi_localise_seed": [P, I, P, I, P, P],
        "toi_localise": [P, I, I, P, P, P, P, P, P],
        "toi_stream_open": [P, I, I, I, C.POINTER(C.c_void_p)],
        "toi_stream_push": [P, P, C.POINTER(C.c_int64)],
        "toi_stream_input_free": [P, C.c_int64, I, C.POINTER(I)],
        "toi_stream_pop": [P, P, C.POINTER(C.c_int64), I, C.POINTER(I)],
        "toi_stream_close": [P],
        "toi_plan_buffer": [P, I, I, P, C.c_int64, C.POINTER(C.c_int64)],
        "toi_profile_enable": [P, I],
        "toi_profile_read": [P, P, P, I],
        "toi_sync_status": [P],
        "toi_last_error": [P],
        "toi_status_string": [I],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_char_p if name in ("toi_last_error", "toi_status_string") else C.c_int
    _lib = L
    return L


def _ptr(x) -> Optional[int]:
    """Device/host address of a torch tensor, an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors passed to libtoi must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)}")


def _dev(x, dtype=None, name="tensor"):
    if x is None:
        return None
    if hasattr(x, "is_cuda"):
        if not x.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if dtype is not None and x.dtype != dtype:
            raise TypeError(f"{name} must have dtype {dtype}, got {x.dtype}")
    return _ptr(x)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(status: int, plan=None):
    if status != TOI_OK:
        raise ToiError(status, lib().toi_last_error(plan).decode())


def _need(x, nbytes: int, name: str):
    """The C calls receive bare addresses and cannot see the extent behind
    them, so a tensor smaller than what a call reads or writes (the layouts
    of toi.h) is refused here with TOI_ERR_ARG, before any launch.  Raw
    integer addresses are the caller's responsibility."""
    if x is None or isinstance(x, int):
        return
    have = x.numel() * x.element_size()
    if have < nbytes:
        raise ToiError(TOI_ERR_ARG, f"{name} holds {have} bytes; the call needs {nbytes}")


def config_default(image_size, cell_arcsec, max_baselines, max_channels, n_pol) -> toi_config:
    cfg = toi_config()
    _check(lib().toi_config_default(C.byref(cfg), image_size, cell_arcsec, max_baselines,
                                    max_channels, n_pol))
    return cfg


class Plan:
    """Owner of a toi_plan_t; methods map one-to-one onto the C entry points."""

    def __init__(self, image_size: int, cell_arcsec: float, max_baselines: int,
                 max_channels: int, n_pol: int, *, vis_dtype: int = TOI_VIS_C64,
                 tlisi_tile: int = 32, grid_slots: int = 1, grid_run: int = 0, batch_max: int = 0,
                 mode: int = 2, max_moments: int = 0, grid_rows: int = 0, max_windows: int = 0,
                 stream=None):
        import torch
        self.cfg = config_default(image_size, cell_arcsec, max_baselines, max_channels, n_pol)
        self.cfg.vis_dtype = vis_dtype
        self.cfg.tlisi_tile = tlisi_tile
        self.cfg.grid_slots = grid_slots
        self.cfg.grid_run = grid_run
        self.cfg.batch_max = batch_max
        self.cfg.mode = mode
        self.cfg.max_moments = max_moments
        self.cfg.grid_rows = grid_rows
        self.cfg.max_windows = max_windows
        self.N = image_size
        self.T = tlisi_tile
        h = C.c_void_p()
        _check(lib().toi_plan(C.byref(self.cfg), _stream(stream), C.byref(h)))
        self.handle = h.value
        self._torch = torch
        self._generation = [0] * grid_slots
        self._set_extents(max_baselines, max_channels, n_pol, vis_dtype, batch_max)

    # ------------------------------------------------- extent checks (host)
    def _set_extents(self, max_bl, max_ch, n_pol, vis_dtype, batch_max):
        self.max_bl, self.max_ch, self.npol = max_bl, max_ch, n_pol
        self.half = vis_dtype == TOI_VIS_C16_CHANSCALE
        self.batch_max = batch_max
        self.nt = self.N // self.T
        self._slot_dims = {}          # slot -> (n_bl, n_ch) of its last grid call

    def _in_limits(self, nbl, nch) -> bool:
        """Counts the library accepts; others are refused by its own checks
        before it touches any buffer."""
        return 0 < nbl <= self.max_bl and 0 < nch <= self.max_ch

    def _need_inputs(self, nbl, nch, uvw, freq, vis, chan_scale, weight, flag, who=""):
        rec = nbl * nch * self.npol
        _need(uvw, 24 * nbl, who + "uvw")
        _need(freq, 8 * nch, who + "freq")
        _need(vis, rec * (4 if self.half else 8), who + "vis")
        _need(chan_scale, 4 * nch, who + "chan_scale")
        _need(weight, 4 * rec, who + "weight")
        _need(flag, rec, who + "flag")

    def _need_per_record(self, slot, grad_sample=None, grad_vis=None, grad_weight=None):
        dims = self._slot_dims.get(slot)
        if dims is None:              # gridded elsewhere (batch): nothing known here
            return
        nbl, nch = dims
        rec = nbl * nch * self.npol
        _need(grad_sample, 8 * nbl * nch, "grad_sample")
        _need(grad_vis, 8 * rec, "grad_vis")
        _need(grad_weight, 4 * rec, "grad_weight")

    # ---------------------------------------------------------------- calls
    def set_stream(self, stream):
        _check(lib().toi_set_stream(self.handle, _stream(stream)), self.handle)

    def grid(self, uvw, freq, vis, flag=None, weight=None, chan_scale=None, slot: int = 0,
             n_bl: Optional[int] = None, n_ch: Optional[int] = None):
        t = self._torch
        nbl = n_bl if n_bl is not None else uvw.shape[0]
        nch = n_ch if n_ch is not None else freq.shape[0]
        if self._in_limits(nbl, nch):
            self._need_inputs(nbl, nch, uvw, freq, vis, chan_scale, weight, flag)
        _check(lib().toi_grid(self.handle, _dev(uvw, t.float64, "uvw"), _dev(freq, t.float64, "freq"),
                              _dev(vis, None, "vis"), _dev(chan_scale, t.float32, "chan_scale"),
                              _dev(weight, t.float32, "weight"), _dev(flag, t.uint8, "flag"),
                              nbl, nch, slot), self.handle)
        self._generation[slot] += 1
        self._slot_dims[slot] = (nbl, nch)

    def slot_generation(self, slot: int = 0) -> int:
        """Number of toi_grid calls made on `slot` through this object."""
        return self._generation[slot]

    def image(self, slot: int = 0, out=None, snap_info=None):
        t = self._torch
        _need(out, 4 * self.N * self.N, "image")
        _need(snap_info, 8 * 16, "snap_info")
        _check(lib().toi_image(self.handle, slot, _dev(out, t.float32, "image"),
                               _dev(snap_info, t.float64, "snap_info")), self.handle)
        return out

    def tlisi_update(self, image=None, out=None) -> bool:
        _need(image, 4 * self.N * self.N, "image")
        _need(out, 4 * self.nt * self.nt, "tlisi")
        valid = C.c_int32(0)
        _check(lib().tlisi_update(self.handle, _dev(image, None, "image"), _dev(out, None, "tlisi"),
                                  C.byref(valid)), self.handle)
        return bool(valid.value)

    def tlisi_reset(self):
        _check(lib().tlisi_reset(self.handle), self.handle)

    def degrid_backward(self, grad_image, image=None, grad_sample=None, grad_vis=None,
                        grad_weight=None, slot: int = 0):
        """toi_degrid_backward: fills the given output tensors (complex64
        grad_sample [n_bl, n_ch], complex64 grad_vis [n_bl, n_ch, n_pol],
        float32 grad_weight [n_bl, n_ch, n_pol]; image is toi_image's float32
        output, needed for grad_weight)."""
        t = self._torch
        _need(grad_image, 4 * self.N * self.N, "grad_image")
        _need(image, 4 * self.N * self.N, "image")
        self._need_per_record(slot, grad_sample, grad_vis, grad_weight)
        _check(lib().toi_degrid_backward(
            self.handle, slot, _dev(grad_image, t.float32, "grad_image"),
            _dev(image, t.float32, "image"), _dev(grad_sample, t.complex64, "grad_sample"),
            _dev(grad_vis, t.complex64, "grad_vis"), _dev(grad_weight, t.float32, "grad_weight")),
            self.handle)

    # --------------------------------------------------------- localisation
    def localise_seed(self, tlisi, n_win: int, win=None, src=None, slot: int = 0):
        """toi_localise_seed: (win int32 [n_win, 2], src float64 [n_win, 3])
        from a tLISI matrix of this slot's snapshot."""
        t = self._torch
        win = t.empty(n_win, 2, dtype=t.int32, device="cuda") if win is None else win
        src = t.empty(n_win, 3, dtype=t.float64, device="cuda") if src is None else src
        _need(tlisi, 4 * self.nt * self.nt, "tlisi")
        if n_win > 0:
            _need(win, 8 * n_win, "win")
            _need(src, 24 * n_win, "src")
        _check(lib().toi_localise_seed(self.handle, slot, _dev(tlisi, t.float32, "tlisi"), n_win,
                                       _dev(win, t.int32, "win"), _dev(src, t.float64, "src")),
               self.handle)
        return win, src

    def localise(self, win, src, model=None, loss=None, grad_src=None, grad_weight=None,
                 slot: int = 0):
        """toi_localise: fills the given outputs (float32 model [n_win, 32, 32],
        float64 loss [n_win], float64 grad_src [n_win, 3], float32
        grad_weight [n_bl, n_ch, n_pol])."""
        t = self._torch
        n = win.shape[0]
        _need(src, 24 * n, "src")
        _need(model, 4 * n * LOC_WINDOW * LOC_WINDOW, "model")
        _need(loss, 8 * n, "loss")
        _need(grad_src, 24 * n, "grad_src")
        self._need_per_record(slot, grad_weight=grad_weight)
        _check(lib().toi_localise(
            self.handle, slot, win.shape[0], _dev(win, t.int32, "win"), _dev(src, t.float64, "src"),
            _dev(model, t.float32, "model"), _dev(loss, t.float64, "loss"),
            _dev(grad_src, t.float64, "grad_src"), _dev(grad_weight, t.float32, "grad_weight")),
            self.handle)

    # ---------------------------------------------------------------- batch
    def _snapshots(self, snaps):
        """toi_snapshot array for a list of dicts (uvw, freq, vis, flag,
        weight, chan_scale, image); the tensors are kept referenced."""
        t = self._torch
        for i, d in enumerate(snaps):           # every snapshot checked before any is marshalled
            nbl, nch = d["uvw"].shape[0], d["freq"].shape[0]
            if self._in_limits(nbl, nch):
                self._need_inputs(nbl, nch, d["uvw"], d["freq"], d["vis"], d.get("chan_scale"),
                                  d.get("weight"), d.get("flag"), f"snapshot {i}: ")
            _need(d.get("image"), 4 * self.N * self.N, f"snapshot {i}: image")
        arr = (toi_snapshot * len(snaps))()
        for i, d in enumerate(snaps):
            arr[i].uvw = _dev(d["uvw"], t.float64, "uvw")
            arr[i].freq = _dev(d["freq"], t.float64, "freq")
            arr[i].vis = _dev(d["vis"], None, "vis")
            arr[i].chan_scale = _dev(d.get("chan_scale"), t.float32, "chan_scale")
            arr[i].weight = _dev(d.get("weight"), t.float32, "weight")
            arr[i].flag = _dev(d.get("flag"), t.uint8, "flag")
            arr[i].image = _dev(d.get("image"), t.float32, "image")
            arr[i].n_bl = d["uvw"].shape[0]
            arr[i].n_ch = d["freq"].shape[0]
        self._batch_refs = list(snaps)
        return arr

    def _need_rows(self, snaps, tlisi):
        if 0 < len(snaps) <= self.batch_max:
            _need(tlisi, 4 * len(snaps) * self.nt * self.nt, "tlisi")

    def batch_prepare(self, snaps, tlisi=None) -> int:
        """toi_batch_prepare; returns first_valid."""
        self._need_rows(snaps, tlisi)
        arr = self._snapshots(snaps)
        fv = C.c_int32(0)
        _check(lib().toi_batch_prepare(self.handle, C.cast(arr, C.c_void_p), len(snaps),
                                       _dev(tlisi, self._torch.float32, "tlisi"), C.byref(fv)),
               self.handle)
        return fv.value

    def batch_run(self):
        _check(lib().toi_batch_run(self.handle), self.handle)

    def batch(self, snaps, tlisi=None) -> int:
        """toi_batch (prepare + run); returns first_valid."""
        self._need_rows(snaps, tlisi)
        arr = self._snapshots(snaps)
        fv = C.c_int32(0)
        _check(lib().toi_batch(self.handle, C.cast(arr, C.c_void_p), len(snaps),
                               _dev(tlisi, self._torch.float32, "tlisi"), C.byref(fv)), self.handle)
        return fv.value

    def autotune(self, snaps):
        """toi_autotune: ({bucket: run}, {bucket: microseconds per snapshot})."""
        arr = self._snapshots(snaps)
        runs = (C.c_int32 * 4)()
        us = (C.c_double * 4)()
        _check(lib().toi_autotune(self.handle, C.cast(arr, C.c_void_p), len(snaps),
                                  C.cast(runs, C.c_void_p), C.cast(us, C.c_void_p)), self.handle)
        return ({b: runs[b] for b in range(4) if runs[b]}, {b: us[b] for b in range(4) if runs[b]})

    def lane_run(self, n_ch: int, batched: bool = True):
        """toi_grid_lane_run: (channels per lane, window rows per lane)."""
        run, rows = C.c_int32(0), C.c_int32(0)
        _check(lib().toi_grid_lane_run(self.handle, n_ch, 1 if batched else 0, C.byref(run),
                                       C.byref(rows)), self.handle)
        return run.value, rows.value

    def mode3_info(self, slot: int = 0):
        """toi_mode3_info as a dict."""
        out = (C.c_double * 8)()
        _check(lib().toi_mode3_info(self.handle, slot, C.cast(out, C.c_void_p)), self.handle)
        keys = ("n_slab", "K", "phi_max", "alpha_slab", "dr3", "r3min", "r3max", "t3max")
        return {k: (int(out[i]) if i < 2 else out[i]) for i, k in enumerate(keys)}

    def buffer(self, which: int, slot: int = 0):
        """Copy of a plan-owned buffer as a new CUDA tensor (see toi_plan_buffer)."""
        t = self._torch
        n = C.c_int64()
        _check(lib().toi_plan_buffer(self.handle, which, slot, None, 0, C.byref(n)), self.handle)
        G = 2 * self.N
        if which == BUF_GRID:
            out = t.empty(G // 2, G, dtype=t.complex64, device="cuda")
        elif which == BUF_SNAP:
            out = t.empty(16, dtype=t.float64, device="cuda")
        else:
            out = t.empty(self.N, self.N, dtype=t.float32, device="cuda")
        _check(lib().toi_plan_buffer(self.handle, which, slot, out.data_ptr(),
                                     out.numel() * out.element_size(), C.byref(n)), self.handle)
        return out

    def profile_enable(self, on: bool = True):
        _check(lib().toi_profile_enable(self.handle, 1 if on else 0), self.handle)

    def profile_read(self):
        """{stage: (milliseconds, launches)} accumulated since the last read."""
        n = len(PROF_STAGES)
        ms = (C.c_double * n)()
        la = (C.c_int64 * n)()
        _check(lib().toi_profile_read(self.handle, C.cast(ms, C.c_void_p), C.cast(la, C.c_void_p), n),
               self.handle)
        return {k: (ms[i], la[i]) for i, k in enumerate(PROF_STAGES)}

    def sync_status(self) -> int:
        return lib().toi_sync_status(self.handle)

    def last_error(self) -> str:
        return lib().toi_last_error(self.handle).decode()

    def close(self):
        if getattr(self, "handle", None):
            lib().toi_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tlisi_candidates(cube, tile: int, mode: int, max_boxes: int = 256, scores=None,
                     stream=None):
    """Candidate search on a device tLISI cube [S, nty, ntx] (float32).
    Returns (threshold, boxes [n, 4] list, n_found)."""
    import torch
    if cube.dtype != torch.float32 or not cube.is_cuda or cube.dim() != 3:
        raise ValueError("cube must be a 3-D float32 CUDA tensor")
    S, nty, ntx = cube.shape
    _need(scores, 8 * nty * ntx, "scores")
    thr = C.c_double()
    nb = C.c_int32()
    boxes = (C.c_int32 * (4 * max(1, max_boxes)))()
    _check(lib().tlisi_candidates(_ptr(cube), S, nty, ntx, tile, mode, _stream(stream),
                                  C.byref(thr), C.cast(boxes, C.c_void_p), C.byref(nb), max_boxes,
                                  _dev(scores, torch.float64, "scores")))
    n = min(nb.value, max_boxes)
    out = [[boxes[4 * i + j] for j in range(4)] for i in range(n)]
    return thr.value, out, nb.value


def tlisi_candidates_noalloc(cube, tile: int, mode: int, max_boxes: int = 256, scores=None,
                             stream=None):
    """tlisi_candidates using the library's fixed device scratch (no
    allocation; see toi.h for the size limit and sharing rules)."""
    import torch
    if cube.dtype != torch.float32 or not cube.is_cuda or cube.dim() != 3:
        raise ValueError("cube must be a 3-D float32 CUDA tensor")
    S, nty, ntx = cube.shape
    _need(scores, 8 * nty * ntx, "scores")
    thr = C.c_double()
    nb = C.c_int32()
    boxes = (C.c_int32 * (4 * max(1, max_boxes)))()
    _check(lib().tlisi_candidates_noalloc(_ptr(cube), S, nty, ntx, tile, mode, _stream(stream),
                                          C.byref(thr), C.cast(boxes, C.c_void_p), C.byref(nb),
                                          max_boxes, _dev(scores, torch.float64, "scores")))
    n = min(nb.value, max_boxes)
    out = [[boxes[4 * i + j] for j in range(4)] for i in range(n)]
    return thr.value, out, nb.value


class Stream:
    """toi_stream_*: the native multi-stream snapshot pipeline of a plan
    (grid_slots >= 3).  push() takes a dict of PINNED host tensors (uvw,
    freq, vis, flag, weight, chan_scale); pop() returns (row index, float32
    tensor [N/T, N/T]) of the oldest finished tLISI row, or None."""

    def __init__(self, plan: Plan, host_depth: int = 8, n_copy: int = 4, with_weights: bool = False):
        import torch
        self._torch = torch
        self.plan = plan
        self.nt = plan.N // plan.T
        h = C.c_void_p()
        _check(lib().toi_stream_open(plan.handle, host_depth, n_copy, 1 if with_weights else 0,
                                     C.byref(h)), plan.handle)
        self.handle = h.value
        self.host_depth = host_depth
        self._inputs = {}
        self.pushed = 0
        self.popped = 0

    @property
    def pending_rows(self) -> int:
        """tLISI rows produced (or in flight) and not yet popped."""
        return max(0, self.pushed - 2) - self.popped

    def push(self, snap) -> int:
        s = toi_snapshot()
        for k in ("uvw", "freq", "vis", "flag", "weight", "chan_scale"):
            x = snap.get(k)
            if x is not None and (x.is_cuda or not x.is_pinned()):
                raise ValueError(f"{k} must be a pinned host tensor")
        s.uvw = _ptr(snap["uvw"])
        s.freq = _ptr(snap["freq"])
        s.vis = _ptr(snap["vis"])
        s.flag = _ptr(snap.get("flag"))
        s.weight = _ptr(snap.get("weight"))
        s.chan_scale = _ptr(snap.get("chan_scale"))
        s.n_bl = snap["uvw"].shape[0]
        s.n_ch = snap["freq"].shape[0]
        if self.plan._in_limits(s.n_bl, s.n_ch):
            self.plan._need_inputs(s.n_bl, s.n_ch, snap["uvw"], snap["freq"], snap["vis"],
                                   snap.get("chan_scale"), snap.get("weight"), snap.get("flag"))
        idx = C.c_int64(0)
        _check(lib().toi_stream_push(self.handle, C.byref(s), C.byref(idx)), self.plan.handle)
        self.pushed = idx.value + 1
        # the host tensors stay referenced until their copies are done
        self._inputs[idx.value] = snap
        for k in [k for k in self._inputs if k < idx.value]:
            if self.input_free(k):
                del self._inputs[k]
        return idx.value

    def input_free(self, index: int, wait: bool = False) -> bool:
        f = C.c_int32(0)
        _check(lib().toi_stream_input_free(self.handle, index, 1 if wait else 0, C.byref(f)),
               self.plan.handle)
        return bool(f.value)

    def pop(self, wait: bool = True, out=None):
        t = self._torch
        if out is not None and out.is_cuda:
            raise ValueError("out must be a host tensor")
        row = t.empty(self.nt, self.nt, dtype=t.float32) if out is None else out
        _need(row, 4 * self.nt * self.nt, "out")
        r = C.c_int64(0)
        got = C.c_int32(0)
        _check(lib().toi_stream_pop(self.handle, row.data_ptr(), C.byref(r), 1 if wait else 0,
                                    C.byref(got)), self.plan.handle)
        if got.value:
            self.popped = r.value + 1
            return r.value, row
        return None

    def close(self):
        if self.handle:
            _check(lib().toi_stream_close(self.handle), self.plan.handle)
            self.handle = None
            self._inputs.clear()
