"""Boundary tests that need no GPU: the library builds, loads, exports every
symbol include/perfmodel.h declares, its struct layouts match the binding,
and bad arguments are rejected with the documented status before anything
is launched."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pm():
    from paper_2605_04178_gb300 import build as B
    B.build()
    import paper_2605_04178_gb300 as pm
    return pm


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "perfmodel.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pm_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("pm_probe_run", "pm_gemm_run", "pm_model_predict", "pm_model_grad", "pm_autotune_pick",
              "pm_grouped_gemm_run", "pm_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol(pm):
    lib = ctypes.CDLL(pm.LIB_PATH)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    assert set(declared_symbols()) == set(pm.EXPORTS)


def test_struct_layouts(pm):
    assert ctypes.sizeof(pm.pm_cfg) == 24 == pm.CFG_DTYPE.itemsize
    assert ctypes.sizeof(pm.pm_params) == 4 * pm.N_PARAMS == 72
    assert pm.SEGMENT_DTYPE.itemsize == 64 and ctypes.sizeof(pm.pm_segment_params) == 8 * pm.N_PSI == 136
    assert pm.pm_version() == 10000
    assert pm._lib.pm_shutdown() == pm.PM_OK                 # nothing created yet: nothing to release
    # reading switch: default measured, round trip, bad value refused
    assert pm.pm_model_reading() == pm.PM_READING_MEASURED
    pm.pm_model_set_reading(pm.PM_READING_LITERAL)
    assert pm.pm_model_reading() == pm.PM_READING_LITERAL
    pm.pm_model_set_reading(pm.PM_READING_MEASURED)
    assert pm._lib.pm_model_set_reading(2) == pm.PM_EINVAL and pm.pm_model_reading() == pm.PM_READING_MEASURED


def test_invalid_tile_rejected_before_launch(pm):
    bad = [pm.cfg(512, 512, 512, BM=96), pm.cfg(512, 512, 512, BK=48), pm.cfg(512, 512, 512, stages=7),
           pm.cfg(512, 512, 512, BM=256, BN=256, BK=128, stages=2), pm.cfg(512, 512, 512, cta_group=3),
           pm.cfg(512, 512, 512, dtype=5)]
    for c in bad:
        st = pm._lib.pm_gemm_run(ctypes.byref(c), None, None, None, None, None)
        assert st == pm.PM_EUNSUPPORTED, (c.BM, c.BK, c.stages, st)
        assert "valid space" in pm.pm_last_error()
    # TMEM strategy B: one-SM tiles of whole 128-row blocks with room for the A ring
    for c in (pm.cfg(512, 512, 512, BM=128, BN=128, cta_group=2, tmem_a=1), pm.cfg(512, 512, 512, BM=64, tmem_a=1),
              pm.cfg(512, 512, 512, BM=256, BN=256, BK=64, stages=2, dtype=2, tmem_a=1),
              pm.cfg(512, 512, 512, tmem_a=2)):
        st = pm._lib.pm_gemm_run(ctypes.byref(c), None, None, None, None, None)
        assert st == pm.PM_EUNSUPPORTED, (c.BM, c.BN, c.cta_group, c.tmem_a, st)
    c = pm.cfg(512, 512, 512, kind=pm.PM_KIND_COPY)
    assert pm._lib.pm_gemm_run(ctypes.byref(c), None, None, None, None, None) == pm.PM_EINVAL
    c = pm.cfg(0, 512, 512)
    assert pm._lib.pm_gemm_run(ctypes.byref(c), None, None, None, None, None) == pm.PM_EINVAL
    assert pm._lib.pm_gemm_run(None, None, None, None, None, None) == pm.PM_EINVAL


def test_bad_arguments_rejected(pm):
    L = pm._lib
    a = pm.probe_args(pm.PM_PROBE_COPY, n=1024)
    res = pm.pm_probe_result()
    assert L.pm_probe_run(ctypes.byref(a), None, None, None, 1, 0, None, ctypes.byref(res)) == pm.PM_EINVAL
    assert L.pm_probe_run(None, None, None, None, 1, 1, None, ctypes.byref(res)) == pm.PM_EINVAL
    assert L.pm_probe_launch(ctypes.byref(a), None, None, None, None) == pm.PM_EINVAL
    a = pm.probe_args(99, n=16)
    assert L.pm_probe_launch(ctypes.byref(a), ctypes.c_void_p(16), ctypes.c_void_p(32), None, None) == pm.PM_EINVAL
    a = pm.probe_args(pm.PM_PROBE_TMA2D, rows=64, cols=64, tile_r=4, tile_c=64)
    assert L.pm_probe_launch(ctypes.byref(a), ctypes.c_void_p(16), ctypes.c_void_p(32), None, None) == pm.PM_EINVAL
    th = pm.params(np.ones(pm.N_PARAMS))
    assert L.pm_model_predict(None, 10, ctypes.byref(th), 152, None, None) == pm.PM_EINVAL
    assert L.pm_model_predict(ctypes.c_void_p(8), 10, ctypes.byref(th), 0, ctypes.c_void_p(8), None) == pm.PM_EINVAL
    assert L.pm_model_predict(None, 0, ctypes.byref(th), 152, None, None) == pm.PM_OK   # empty batch: nothing to do
    assert L.pm_model_grad(None, 0, ctypes.byref(th), 152, None, None, 0, None, None) == pm.PM_EINVAL
    th64 = (ctypes.c_double * 16)(*([1.0] * 16))
    assert L.pm_model_grad_f64(None, 10, ctypes.cast(th64, ctypes.c_void_p), 152, None, None, 0, None,
                               None) == pm.PM_EINVAL
    assert L.pm_model_grad_f64(ctypes.c_void_p(8), 1000, ctypes.cast(th64, ctypes.c_void_p), 152, ctypes.c_void_p(8),
                               ctypes.c_void_p(8), 8, ctypes.c_void_p(8), None) == pm.PM_ENOMEM
    sz = ctypes.c_size_t()
    assert L.pm_model_grad_workspace(1000, ctypes.byref(sz)) == pm.PM_OK and sz.value >= 17 * 8
    assert L.pm_model_grad(ctypes.c_void_p(8), 1000, ctypes.byref(th), 152, ctypes.c_void_p(8), ctypes.c_void_p(8),
                           8, ctypes.c_void_p(8), None) in (pm.PM_ENOMEM, pm.PM_ECUDA)
    assert L.pm_autotune_pick(ctypes.c_void_p(8), 4, 7, ctypes.byref(th), 152, ctypes.c_void_p(8),
                              ctypes.c_void_p(8), None) == pm.PM_EINVAL
    a_b, b_b = ctypes.c_size_t(), ctypes.c_size_t()
    assert L.pm_gemm_operand_bytes(0, 512, 256, 128, ctypes.byref(a_b), ctypes.byref(b_b)) == pm.PM_OK
    assert a_b.value == 2 * 4 * 512 * 128 and b_b.value == 2 * 4 * 256 * 128
    assert L.pm_gemm_operand_bytes(3, 512, 256, 128, ctypes.byref(a_b), ctypes.byref(b_b)) == pm.PM_EINVAL
    assert L.pm_gemm_prepare(1, None, None, 16, 16, 16, None, None, None, None) == pm.PM_EINVAL
    Mh = (ctypes.c_int32 * 2)(16, 0)
    o16 = (ctypes.c_int16 * 2)()
    launch = (ctypes.c_int32 * 3)()
    t = ctypes.c_float()
    assert L.pm_grouped_autotune(2, Mh, 64, 64, 1, ctypes.byref(th), 152, o16, o16, launch, ctypes.byref(t),
                                 None) == pm.PM_EINVAL
    assert L.pm_watchdog_selftest(0, None) == pm.PM_EINVAL
    Mg = (ctypes.c_int32 * 2)(16, 32)
    bad16 = (ctypes.c_int16 * 2)(96, 96)
    tf = ctypes.c_float()
    assert L.pm_grouped_predict(2, Mg, 64, 64, bad16, bad16, 64, 4, 1, 1, ctypes.byref(th), 152, ctypes.byref(tf),
                                None) == pm.PM_EUNSUPPORTED
    assert L.pm_grouped_predict(0, Mg, 64, 64, bad16, bad16, 64, 4, 1, 1, ctypes.byref(th), 152, ctypes.byref(tf),
                                None) == pm.PM_EINVAL
    assert L.pm_grouped_gemm_autotune(2, Mg, 64, 64, ctypes.byref(th), 152, 0, ctypes.c_void_p(16),
                                      ctypes.c_void_p(16), ctypes.c_void_p(16), 1, 1, None, o16, o16, launch,
                                      None, None) == pm.PM_EINVAL
    assert L.pm_grouped_gemm_autotune(2, Mg, 64, 64, ctypes.byref(th), 152, 4, None, None, None, 1, 1, None,
                                      o16, o16, launch, None, None) == pm.PM_EINVAL
    ps = pm.pm_segment_params()
    assert L.pm_segment_predict(None, 4, ctypes.byref(th), ctypes.byref(ps), 152, None, None) == pm.PM_EINVAL
    assert L.pm_segment_predict(None, 0, ctypes.byref(th), ctypes.byref(ps), 152, None, None) == pm.PM_OK
    assert L.pm_segment_predict(ctypes.c_void_p(12), 4, ctypes.byref(th), ctypes.byref(ps), 152, ctypes.c_void_p(16),
                                None) == pm.PM_EINVAL                    # misaligned records
    # concurrent-stream probe: argument checks come before any CUDA call
    bufs = (ctypes.c_void_p * 8)(*([16] * 8))
    vp = ctypes.cast(bufs, ctypes.c_void_p)
    copy = pm.probe_args(pm.PM_PROBE_COPY, n=1024)
    assert L.pm_streams_run(ctypes.byref(copy), 0, vp, vp, None, 1, 1, None, ctypes.byref(res)) == pm.PM_EINVAL
    assert L.pm_streams_run(ctypes.byref(copy), 9, vp, vp, None, 1, 1, None, ctypes.byref(res)) == pm.PM_EINVAL
    assert L.pm_streams_run(ctypes.byref(copy), 2, vp, None, None, 1, 1, None, ctypes.byref(res)) == pm.PM_EINVAL
    triad = pm.probe_args(pm.PM_PROBE_TRIAD, n=1024)
    assert L.pm_streams_run(ctypes.byref(triad), 2, vp, vp, None, 1, 1, None, ctypes.byref(res)) == pm.PM_EINVAL
    chase = pm.probe_args(pm.PM_PROBE_PCHASE, n=1024, hops=10)
    assert L.pm_streams_run(ctypes.byref(chase), 2, vp, vp, None, 1, 1, None, ctypes.byref(res)) == pm.PM_EINVAL
    assert L.pm_streams_run(ctypes.byref(copy), 2, vp, vp, None, 1, 0, None, ctypes.byref(res)) == pm.PM_EINVAL
    assert L.pm_streams_run(None, 2, vp, vp, None, 1, 1, None, ctypes.byref(res)) == pm.PM_EINVAL


def test_tile_space_matches_oracle_rule(pm):
    # the library's validity rule (reached through pm_gemm_run's early check)
    # and the oracle's independent implementation agree on all 540 points of
    # each TMEM strategy
    import oracle as O
    import synthetic as S
    for ta in (0, 1):
        for dt in (0, 1, 2):
            for (bm, bn, bk, s, g) in S.tile_space(dt):
                c = pm.cfg(256, 256, 256, bm, bn, bk, s, g, dt, tmem_a=ta)
                st = pm._lib.pm_gemm_run(ctypes.byref(c), None, None, None, None, None)
                lib_valid = st != pm.PM_EUNSUPPORTED
                assert lib_valid == O.cfg_valid(bm, bn, bk, s, g, dt, ta), (ta, dt, bm, bn, bk, s, g, st)
