"""The allocation-free candidate search (tlisi_candidates_noalloc) gives the
same threshold, scores and boxes, bit for bit, as tlisi_candidates, on two
calls in a row through the C ABI; oversized cubes are refused on the host.

It serves callers that cannot allocate device memory during the search (a
real-time pipeline that must not stall on cudaMalloc, or an application whose
allocator owns all device memory).  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

import paper_2512_06254_gb300 as toi  # noqa: E402
from paper_2512_06254_gb300 import binding as B  # noqa: E402


def _abi_call(fn, cube, T, mode, max_boxes, scores):
    S, nty, ntx = cube.shape
    thr = C.c_double()
    nb = C.c_int32()
    boxes = (C.c_int32 * (4 * max_boxes))()
    st = fn(cube.data_ptr(), S, nty, ntx, T, mode, torch.cuda.current_stream().cuda_stream,
            C.byref(thr), C.cast(boxes, C.c_void_p), C.byref(nb), max_boxes,
            None if scores is None else scores.data_ptr())
    return st, thr.value, nb.value, [list(boxes[4 * i:4 * i + 4]) for i in range(min(nb.value, max_boxes))]


def _cube(seed, S, n):
    rng = np.random.default_rng(seed)
    cube = (1.0 - np.abs(rng.normal(scale=0.02, size=(S, n, n)))).astype(np.float32)
    on = (np.arange(S) % 40) < 20
    cube[on, n // 3, n // 2] -= 0.25
    cube[S // 2:S // 2 + 6, 2, n - 3] -= 0.4
    return torch.from_numpy(cube).cuda()


@pytest.mark.parametrize("mode", [toi.TOI_CAND_PERIODIC, toi.TOI_CAND_NONPERIODIC])
def test_noalloc_matches_allocating_search_twice(mode):
    # start from an idle device: no earlier test's work may still be running
    # on another stream when this test's tensors are allocated
    torch.cuda.synchronize()
    L = B.lib()
    for call, (seed, S, n) in enumerate([(101, 118, 64), (202, 300, 32)]):
        cube = _cube(seed + mode, S, n)
        s_ref = torch.empty(n, n, dtype=torch.float64, device="cuda")
        s_new = torch.empty(n, n, dtype=torch.float64, device="cuda")
        st_ref, thr_ref, nb_ref, boxes_ref = _abi_call(L.tlisi_candidates, cube, 32, mode, 64, s_ref)
        st_new, thr_new, nb_new, boxes_new = _abi_call(L.tlisi_candidates_noalloc, cube, 32, mode, 64,
                                                       s_new)
        assert st_ref == toi.TOI_OK and st_new == toi.TOI_OK, f"call {call}"
        assert thr_new == thr_ref
        assert nb_new == nb_ref and boxes_new == boxes_ref
        assert torch.equal(s_new, s_ref)


def test_noalloc_without_scores_buffer():
    """scores NULL: the scores stay in the fixed array; threshold and boxes
    still equal the allocating search's, on two calls in a row."""
    L = B.lib()
    for seed in (303, 404):
        cube = _cube(seed, 118, 64)
        s_ref = torch.empty(64, 64, dtype=torch.float64, device="cuda")
        st_ref, thr_ref, nb_ref, boxes_ref = _abi_call(L.tlisi_candidates, cube, 32,
                                                       toi.TOI_CAND_PERIODIC, 64, s_ref)
        st_new, thr_new, nb_new, boxes_new = _abi_call(L.tlisi_candidates_noalloc, cube, 32,
                                                       toi.TOI_CAND_PERIODIC, 64, None)
        assert st_ref == toi.TOI_OK and st_new == toi.TOI_OK
        assert thr_new == thr_ref and nb_new == nb_ref and boxes_new == boxes_ref
        assert nb_ref >= 1


def test_noalloc_refuses_cube_beyond_its_scratch():
    L = B.lib()
    cube = torch.full((2000, 64, 64), 0.9, dtype=torch.float32, device="cuda")
    scores = torch.empty(64, 64, dtype=torch.float64, device="cuda")
    st, _, _, _ = _abi_call(L.tlisi_candidates_noalloc, cube, 32, toi.TOI_CAND_PERIODIC, 16, scores)
    assert st == toi.TOI_ERR_ARG
    assert b"16777216" in L.toi_last_error(None)
