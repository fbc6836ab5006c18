"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
function include/toi.h declares, and rejects bad arguments on the host
before touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libtoi():
    from paper_2512_06254_gb300 import build
    if not build.up_to_date():
        build.build()
    import paper_2512_06254_gb300 as toi
    return toi


def declared_functions():
    src = open(os.path.join(ROOT, "include", "toi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(libtoi):
    names = declared_functions()
    assert len(names) >= 14
    L = C.CDLL(libtoi.binding.LIB_PATH)
    for n in names:
        assert hasattr(L, n), f"{n} declared in toi.h but not exported"
    assert set(names) == set(libtoi.binding.EXPORTS)


def test_host_validation_without_gpu(libtoi):
    from paper_2512_06254_gb300 import binding as b
    L = libtoi.lib()
    h = C.c_void_p()
    cases = [((100, 2.0, 10, 10, 4), libtoi.TOI_ERR_UNSUPPORTED),
             ((112, 2.0, 10, 10, 4), libtoi.TOI_ERR_UNSUPPORTED),     # 7 x 16
             ((16384, 1.0, 10, 10, 4), libtoi.TOI_ERR_UNSUPPORTED),   # above 8192
             ((12288, 1.0, 10, 10, 4), libtoi.TOI_ERR_UNSUPPORTED),   # 3 x 2^12 > 6144
             ((20480, 1.0, 10, 10, 4), libtoi.TOI_ERR_UNSUPPORTED),   # above 10240
             ((48, 2.0, 10, 10, 4), libtoi.TOI_ERR_ARG),              # below 64
             ((32, 2.0, 10, 10, 4), libtoi.TOI_ERR_ARG),
             ((128, -1.0, 10, 10, 4), libtoi.TOI_ERR_ARG),
             ((128, 2.0, 0, 10, 4), libtoi.TOI_ERR_ARG),
             ((128, 2.0, 10, 10, 3), libtoi.TOI_ERR_ARG)]
    for args, want in cases:
        cfg = b.config_default(*args)
        assert L.toi_plan(C.byref(cfg), None, C.byref(h)) == want
        assert L.toi_last_error(None)
    cfg = b.config_default(128, 2.0, 10, 10, 4)
    cfg.tlisi_tile = 48
    assert L.toi_plan(C.byref(cfg), None, C.byref(h)) == libtoi.TOI_ERR_ARG
    cfg = b.config_default(128, 2.0, 10, 10, 4)
    cfg.reserved[0] = 1
    assert L.toi_plan(C.byref(cfg), None, C.byref(h)) == libtoi.TOI_ERR_ARG
    cfg = b.config_default(128, 2.0, 10, 10, 4)
    cfg.max_windows = 257                                  # above 256
    assert L.toi_plan(C.byref(cfg), None, C.byref(h)) == libtoi.TOI_ERR_ARG
    assert L.toi_grid(None, None, None, None, None, None, None, 1, 1, 0) == libtoi.TOI_ERR_ARG
    assert L.toi_localise(None, 0, 1, None, None, None, None, None, None) == libtoi.TOI_ERR_ARG
    assert L.toi_localise_seed(None, 0, None, 1, None, None) == libtoi.TOI_ERR_ARG
    out = C.c_void_p()
    assert L.toi_stream_open(None, 2, 1, 0, C.byref(out)) == libtoi.TOI_ERR_ARG
    assert L.toi_stream_push(None, None, None) == libtoi.TOI_ERR_ARG
    got = C.c_int32(0)
    assert L.toi_stream_pop(None, None, None, 0, C.byref(got)) == libtoi.TOI_ERR_ARG
    assert L.toi_stream_input_free(None, 0, 0, C.byref(got)) == libtoi.TOI_ERR_ARG
    assert L.toi_stream_close(None) == libtoi.TOI_ERR_ARG
    assert L.tlisi_candidates(None, 1, 1, 1, 1, 0, None, None, None, None, 0, None) == libtoi.TOI_ERR_ARG
    # the candidate search's single-block labelling takes at most 2^17 tiles; refused on the
    # host (the cube address is never touched)
    thr, nb = C.c_double(), C.c_int32()
    for fn in (L.tlisi_candidates, L.tlisi_candidates_noalloc):
        assert fn(C.c_void_p(256), 10, 363, 362, 32, 0, None, C.byref(thr), None, C.byref(nb), 0,
                  None) == libtoi.TOI_ERR_ARG
        assert b"131072" in L.toi_last_error(None)
    assert L.toi_status_string(libtoi.TOI_ERR_RANGE)


def test_config_fields_validated_on_the_host(libtoi):
    """Every toi_config field outside its documented range is refused by
    toi_plan before any CUDA call (so this runs without a GPU)."""
    from paper_2512_06254_gb300 import binding as b
    L = libtoi.lib()
    h = C.c_void_p()
    ARG, UNS = libtoi.TOI_ERR_ARG, libtoi.TOI_ERR_UNSUPPORTED
    cases = [("vis_dtype", 2, ARG), ("kernel_support", 6, UNS), ("oversample", 3, UNS),
             ("grid_slots", 0, ARG), ("grid_slots", 17, ARG), ("grid_run", 7, ARG),
             ("grid_run", 1025, ARG), ("batch_max", -1, ARG), ("batch_max", 65, ARG),
             ("mode", 1, ARG), ("mode", 4, ARG), ("max_moments", -1, ARG),
             ("max_moments", 1025, ARG), ("grid_rows", 5, ARG), ("max_windows", -1, ARG),
             ("cell_arcsec", float("inf"), ARG), ("cell_arcsec", float("nan"), ARG),
             ("max_channels", 0, ARG)]
    for field, value, want in cases:
        cfg = b.config_default(128, 2.0, 10, 10, 4)
        setattr(cfg, field, value)
        assert L.toi_plan(C.byref(cfg), None, C.byref(h)) == want, (field, value)
        assert h.value is None
    cfg = b.config_default(128, 2.0, 10, 10, 4)
    cfg.mode, cfg.batch_max = 3, 4                       # the batch is 2-D only
    assert L.toi_plan(C.byref(cfg), None, C.byref(h)) == UNS
    cfg = b.config_default(128, 2.0, 1 << 20, 1 << 20, 4)   # 2^42 records
    assert L.toi_plan(C.byref(cfg), None, C.byref(h)) == ARG
    assert L.toi_plan(None, None, C.byref(h)) == ARG
