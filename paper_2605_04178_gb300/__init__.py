"""Python binding of libperfmodel.so (include/perfmodel.h), the GB300 hot path of
the stage-centric GPU performance model of arxiv 2605.04178.

Argument marshalling only: every step runs in the CUDA library.  The
functions carry the C names (pm_probe_run, pm_gemm_prepare, pm_gemm_run,
pm_grouped_gemm_run, pm_model_predict, pm_model_grad, pm_autotune_pick,
pm_grouped_autotune, ...); device buffers are torch CUDA tensors, streams
default to torch's current stream.  If the compiled library is missing the
import fails: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libperfmodel.so")

PM_OK, PM_EINVAL, PM_EUNSUPPORTED, PM_ECUDA, PM_ETIMEOUT, PM_ENOMEM = 0, -1, -2, -3, -4, -5
PM_FP32, PM_BF16, PM_FP8E4M3 = 0, 1, 2
PM_KIND_GEMM, PM_KIND_COPY, PM_KIND_TRIAD, PM_KIND_TMA2D = 0, 1, 2, 3
PM_READING_LITERAL, PM_READING_MEASURED = 0, 1
N_PARAMS = 18                     # PM_NPARAMS: entries of theta (pm_params)
N_GRAD_OUT = N_PARAMS + 1         # pm_model_grad output: loss, then the gradient
N_PSI = 17                        # PM_NPSI: entries of the segment parameters (pm_segment_params)
PM_PROBE_COPY, PM_PROBE_TRIAD, PM_PROBE_TMA2D, PM_PROBE_PCHASE = 1, 2, 3, 4
PM_PROBE_H2D, PM_PROBE_D2H, PM_PROBE_MMA, PM_PROBE_MBAR, PM_PROBE_TMEM_LD, PM_PROBE_TMEM_ST = 5, 6, 7, 8, 9, 10
PM_PROBE_HOST_READ, PM_PROBE_HOST_WRITE, PM_PROBE_STENCIL = 11, 12, 13

# numpy view of pm_cfg (24 bytes)
CFG_DTYPE = np.dtype([("M", "<i4"), ("N", "<i4"), ("K", "<i4"), ("BM", "<i2"), ("BN", "<i2"), ("BK", "<i2"),
                      ("stages", "i1"), ("cta_group", "i1"), ("dtype", "i1"), ("kind", "i1"),
                      ("tmem_a", "<i2")], align=True)
assert CFG_DTYPE.itemsize == 24


class pm_cfg(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("N", ctypes.c_int32), ("K", ctypes.c_int32), ("BM", ctypes.c_int16),
                ("BN", ctypes.c_int16), ("BK", ctypes.c_int16), ("stages", ctypes.c_int8),
                ("cta_group", ctypes.c_int8), ("dtype", ctypes.c_int8), ("kind", ctypes.c_int8),
                ("tmem_a", ctypes.c_int16)]


class pm_params(ctypes.Structure):
    _fields_ = [("v", ctypes.c_float * N_PARAMS)]


# numpy view of pm_segment (64 bytes)
SEGMENT_DTYPE = np.dtype([("flops", "<f8"), ("bytes", "<f8"), ("working_set", "<f8"), ("h2d_bytes", "<f8"),
                          ("d2h_bytes", "<f8"), ("cls", "<i4"), ("precision", "<i4"), ("kernels", "<i4"),
                          ("syncs", "<i4"), ("execs", "<i4"), ("streams", "<i4")], align=True)
assert SEGMENT_DTYPE.itemsize == 64
PM_SEG_MEMORY, PM_SEG_COMPUTE, PM_SEG_BALANCED, PM_SEG_STENCIL = 0, 1, 2, 3


class pm_segment_params(ctypes.Structure):
    _fields_ = [("v", ctypes.c_double * N_PSI)]


class pm_probe_args(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("tile_r", ctypes.c_int32), ("tile_c", ctypes.c_int32),
                ("start", ctypes.c_uint32), ("n", ctypes.c_int64), ("rows", ctypes.c_int64),
                ("cols", ctypes.c_int64), ("hops", ctypes.c_int64), ("scalar", ctypes.c_float),
                ("reserved", ctypes.c_int32)]


class pm_probe_result(ctypes.Structure):
    _fields_ = [("median_s", ctypes.c_double), ("p25_s", ctypes.c_double), ("p75_s", ctypes.c_double),
                ("min_s", ctypes.c_double), ("bytes", ctypes.c_double), ("final_index", ctypes.c_uint32),
                ("sm_mhz_begin", ctypes.c_uint32), ("sm_mhz_end", ctypes.c_uint32), ("sm_max_mhz", ctypes.c_uint32),
                ("clock_reasons", ctypes.c_uint64)]


class pm_clock(ctypes.Structure):
    _fields_ = [("sm_mhz", ctypes.c_uint32), ("sm_max_mhz", ctypes.c_uint32), ("mem_mhz", ctypes.c_uint32),
                ("power_mw", ctypes.c_uint32), ("reasons", ctypes.c_uint64), ("host_time_s", ctypes.c_double)]


assert ctypes.sizeof(pm_cfg) == 24 and ctypes.sizeof(pm_probe_args) == 56 and ctypes.sizeof(pm_probe_result) == 64
assert ctypes.sizeof(pm_clock) == 32

# NVML clock event reasons (bitmask of pm_clock.reasons / pm_probe_result.clock_reasons)
CLOCK_REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
                 0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
                 0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}


def clock_reason_names(mask: int) -> list:
    return [name for bit, name in sorted(CLOCK_REASONS.items()) if mask & bit]


def _timing(res) -> dict:
    """A harness result as a dict: device times, bytes, and the clock record of the timed region."""
    return dict(median_s=res.median_s, p25_s=res.p25_s, p75_s=res.p75_s, min_s=res.min_s, bytes=res.bytes,
                final_index=res.final_index, sm_mhz_begin=res.sm_mhz_begin, sm_mhz_end=res.sm_mhz_end,
                sm_max_mhz=res.sm_max_mhz, clock_reasons=clock_reason_names(res.clock_reasons))

# Every exported symbol of include/perfmodel.h
EXPORTS = ("pm_probe_launch", "pm_probe_run", "pm_streams_run", "pm_gemm_operand_bytes", "pm_gemm_prepare", "pm_gemm_run",
           "pm_gemm_bench", "pm_gemm_host_workspace", "pm_gemm_host",
           "pm_grouped_gemm_run", "pm_model_predict", "pm_model_set_reading", "pm_model_reading", "pm_model_grad_workspace", "pm_model_grad", "pm_model_grad_f64", "pm_model_grad_noalloc",
           "pm_autotune_pick", "pm_autotune_topk", "pm_gemm_autotune", "pm_grouped_predict", "pm_grouped_grad", "pm_grouped_candidates", "pm_grouped_autotune", "pm_grouped_gemm_autotune", "pm_segment_predict", "pm_last_error", "pm_device_status", "pm_shutdown",
           "pm_watchdog_selftest", "pm_version", "pm_clock_sample")


class PMError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__("%s -> status %d: %s" % (where, status, msg))
        self.status = status


def _load():
    # Compile on first import (nvcc, sm_103a) when the library is missing or
    # older than its sources; a failed build raises: there is no fallback.
    from . import build as _build
    try:
        _build.build()
    except Exception as e:  # noqa: BLE001
        raise ImportError("libperfmodel.so could not be built: %s" % e) from e
    if not os.path.exists(LIB_PATH):
        raise ImportError("libperfmodel.so is missing (%s)" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    sig = {
        "pm_probe_launch": [ctypes.POINTER(pm_probe_args), P, P, P, P],
        "pm_probe_run": [ctypes.POINTER(pm_probe_args), P, P, P, ctypes.c_int, ctypes.c_int, P,
                         ctypes.POINTER(pm_probe_result)],
        "pm_streams_run": [ctypes.POINTER(pm_probe_args), i32, P, P, P, ctypes.c_int, ctypes.c_int, P,
                           ctypes.POINTER(pm_probe_result)],
        "pm_gemm_operand_bytes": [i32, i32, i32, i32, ctypes.POINTER(sz), ctypes.POINTER(sz)],
        "pm_gemm_prepare": [i32, P, P, i32, i32, i32, P, P, P, P],
        "pm_gemm_run": [ctypes.POINTER(pm_cfg), P, P, P, P, P],
        "pm_gemm_host_workspace": [ctypes.POINTER(pm_cfg), i32, ctypes.POINTER(sz)],
        "pm_gemm_host": [ctypes.POINTER(pm_cfg), P, P, P, P, sz, i32, P],
        "pm_gemm_bench": [ctypes.POINTER(pm_cfg), P, P, P, P, ctypes.c_int, ctypes.c_int, P,
                          ctypes.POINTER(pm_probe_result)],
        "pm_grouped_gemm_run": [i32, P, i32, i32, P, P, i32, i32, i32, P, P, P, P],
        "pm_model_predict": [P, i64, ctypes.POINTER(pm_params), i32, P, P],
        "pm_model_grad_workspace": [i64, ctypes.POINTER(sz)],
        "pm_model_grad": [P, i64, ctypes.POINTER(pm_params), i32, P, P, sz, P, P],
        "pm_model_grad_noalloc": [P, i64, ctypes.POINTER(pm_params), i32, P, P, P],
        "pm_model_grad_f64": [P, i64, P, i32, P, P, sz, P, P],
        "pm_autotune_pick": [P, i64, i32, ctypes.POINTER(pm_params), i32, P, P, P],
        "pm_autotune_topk": [P, i64, i32, ctypes.POINTER(pm_params), i32, i32, P, P, P],
        "pm_gemm_autotune": [ctypes.POINTER(pm_cfg), i32, ctypes.POINTER(pm_params), i32, P, P, P, P, ctypes.c_int,
                             ctypes.c_int, P, ctypes.POINTER(pm_cfg), ctypes.POINTER(pm_probe_result)],
        "pm_grouped_autotune": [i32, P, i32, i32, i32, ctypes.POINTER(pm_params), i32, P, P, P, P, P],
        "pm_grouped_predict": [i32, P, i32, i32, P, P, i32, i32, i32, i32, ctypes.POINTER(pm_params), i32, P, P],
        "pm_grouped_grad": [i32, P, i32, i32, P, P, i32, i32, i32, i32, P, i32, P, P],
        "pm_grouped_candidates": [i32, P, i32, i32, i32, ctypes.POINTER(pm_params), i32, P, P, P, P, P],
        "pm_segment_predict": [P, i64, ctypes.POINTER(pm_params), ctypes.POINTER(pm_segment_params), i32, P, P],
        "pm_grouped_gemm_autotune": [i32, P, i32, i32, ctypes.POINTER(pm_params), i32, i32, P, P, P, ctypes.c_int,
                                     ctypes.c_int, P, P, P, P, P, ctypes.POINTER(pm_probe_result)],
        "pm_device_status": [ctypes.c_int],
        "pm_clock_sample": [ctypes.POINTER(pm_clock)],
        "pm_shutdown": [],
        "pm_model_set_reading": [i32],
        "pm_model_reading": [],
        "pm_watchdog_selftest": [i32, P],
        "pm_version": [],
        "pm_last_error": [],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int32
    lib.pm_last_error.restype = ctypes.c_char_p
    return lib


_lib = _load()


def _check(status: int, where: str) -> int:
    if status != PM_OK:
        raise PMError(status, where, _lib.pm_last_error().decode(errors="replace"))
    return status


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def params(theta) -> pm_params:
    p = pm_params()
    th = np.asarray(theta, dtype=np.float32)
    assert th.size == N_PARAMS, "theta has %d entries, not %d" % (th.size, N_PARAMS)
    for j in range(N_PARAMS):
        p.v[j] = float(th[j])
    return p


def cfg(M, N, K, BM=128, BN=128, BK=64, stages=4, cta_group=1, dtype=PM_BF16, kind=PM_KIND_GEMM,
        tmem_a=0) -> pm_cfg:
    """One pm_cfg; tmem_a = 1 selects TMEM strategy B (A operand copied into tensor memory)."""
    return pm_cfg(int(M), int(N), int(K), int(BM), int(BN), int(BK), int(stages), int(cta_group), int(dtype),
                  int(kind), int(tmem_a))


def cfg_array(fields: dict) -> np.ndarray:
    """Structured pm_cfg array from a dict of equal-length columns (missing columns are 0)."""
    n = len(fields["M"])
    a = np.zeros(n, dtype=CFG_DTYPE)
    for k, v in fields.items():
        a[k] = v
    return a


def cfg_tensor(fields: dict, device="cuda"):
    """pm_cfg records on the device as a uint8 tensor (24 bytes per configuration)."""
    import torch
    a = cfg_array(fields)
    return torch.from_numpy(a.view(np.uint8).copy()).to(device)


# --------------------------------------------------------------------- probes
def probe_args(kind, n=0, rows=0, cols=0, tile_r=0, tile_c=0, hops=0, start=0, scalar=3.0) -> pm_probe_args:
    return pm_probe_args(int(kind), int(tile_r), int(tile_c), int(start), int(n), int(rows), int(cols), int(hops),
                         float(scalar), 0)


def pm_probe_launch(args: pm_probe_args, buf0, buf1=None, buf2=None, stream=None):
    _check(_lib.pm_probe_launch(ctypes.byref(args), _ptr(buf0), _ptr(buf1), _ptr(buf2), _stream(stream)),
           "pm_probe_launch")


def pm_probe_run(args: pm_probe_args, buf0, buf1=None, buf2=None, warmup=10, reps=100, stream=None) -> dict:
    res = pm_probe_result()
    _check(_lib.pm_probe_run(ctypes.byref(args), _ptr(buf0), _ptr(buf1), _ptr(buf2), int(warmup), int(reps),
                             _stream(stream), ctypes.byref(res)), "pm_probe_run")
    return _timing(res)


def pm_streams_run(args: pm_probe_args, bufs0, bufs1=None, bufs2=None, warmup=10, reps=100, stream=None) -> dict:
    """The probe `args` on len(bufs0) concurrent streams (stream i on bufs0[i], bufs1[i], bufs2[i]);
    median/quartiles of the makespan."""
    n = len(bufs0)

    def arr(bufs):
        if bufs is None:
            return None
        assert len(bufs) == n
        a = (ctypes.c_void_p * n)(*[_ptr(b) for b in bufs])
        return ctypes.cast(a, ctypes.c_void_p), a

    a0, a1, a2 = arr(bufs0), arr(bufs1), arr(bufs2)
    res = pm_probe_result()
    _check(_lib.pm_streams_run(ctypes.byref(args), int(n), a0[0], a1[0] if a1 else None, a2[0] if a2 else None,
                               int(warmup), int(reps), _stream(stream), ctypes.byref(res)), "pm_streams_run")
    return _timing(res)


# ----------------------------------------------------------------------- GEMM
def pm_gemm_operand_bytes(dtype, M, N, K):
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    _check(_lib.pm_gemm_operand_bytes(int(dtype), int(M), int(N), int(K), ctypes.byref(a), ctypes.byref(b)),
           "pm_gemm_operand_bytes")
    return a.value, b.value


def pm_gemm_prepare(dtype, A, B, M, N, K, A_op, B_op, scales=None, stream=None):
    _check(_lib.pm_gemm_prepare(int(dtype), _ptr(A), _ptr(B), int(M), int(N), int(K), _ptr(A_op), _ptr(B_op),
                                _ptr(scales), _stream(stream)), "pm_gemm_prepare")


def pm_gemm_run(c: pm_cfg, A_op, B_op, C, scales=None, stream=None):
    _check(_lib.pm_gemm_run(ctypes.byref(c), _ptr(A_op), _ptr(B_op), _ptr(C), _ptr(scales), _stream(stream)),
           "pm_gemm_run")


def pm_gemm_bench(c: pm_cfg, A_op, B_op, C, scales=None, warmup=10, reps=100, stream=None) -> dict:
    res = pm_probe_result()
    _check(_lib.pm_gemm_bench(ctypes.byref(c), _ptr(A_op), _ptr(B_op), _ptr(C), _ptr(scales), int(warmup), int(reps),
                              _stream(stream), ctypes.byref(res)), "pm_gemm_bench")
    return _timing(res)


def pm_gemm_host_workspace(c: pm_cfg, chunks) -> int:
    b = ctypes.c_size_t()
    _check(_lib.pm_gemm_host_workspace(ctypes.byref(c), int(chunks), ctypes.byref(b)), "pm_gemm_host_workspace")
    return b.value


def pm_gemm_host(c: pm_cfg, A_host, B_host, C_host, workspace, chunks=4, stream=None):
    """C_host = A_host @ B_host from (pinned) host FP32 tensors, copies overlapped with compute."""
    _check(_lib.pm_gemm_host(ctypes.byref(c), _ptr(A_host), _ptr(B_host), _ptr(C_host), _ptr(workspace),
                             int(workspace.numel() * workspace.element_size()), int(chunks), _stream(stream)),
           "pm_gemm_host")


def pm_grouped_gemm_run(M_list, N, K, BM_list, BN_list, BK, stages, cta_group, A_op, B_op, C, stream=None):
    G = len(M_list)
    Mh = (ctypes.c_int32 * G)(*[int(m) for m in M_list])
    BMh = (ctypes.c_int16 * G)(*[int(m) for m in BM_list])
    BNh = (ctypes.c_int16 * G)(*[int(m) for m in BN_list])
    _check(_lib.pm_grouped_gemm_run(G, Mh, int(N), int(K), BMh, BNh, int(BK), int(stages), int(cta_group),
                                    _ptr(A_op), _ptr(B_op), _ptr(C), _stream(stream)), "pm_grouped_gemm_run")


class GemmOperands:
    """Device operand buffers for one (dtype, M, N, K), allocated with torch."""

    def __init__(self, dtype, M, N, K, device="cuda"):
        import torch
        a, b = pm_gemm_operand_bytes(dtype, M, N, K)
        self.dtype, self.M, self.N, self.K = dtype, M, N, K
        self.A_op = torch.empty(a, dtype=torch.uint8, device=device)
        self.B_op = torch.empty(b, dtype=torch.uint8, device=device)
        self.scales = torch.zeros(4, dtype=torch.float32, device=device)

    def prepare(self, A, B, stream=None):
        pm_gemm_prepare(self.dtype, A, B, self.M, self.N, self.K, self.A_op, self.B_op, self.scales, stream)

    def run(self, c: pm_cfg, C, stream=None):
        pm_gemm_run(c, self.A_op, self.B_op, C, self.scales, stream)

    def bench(self, c: pm_cfg, C, warmup=10, reps=100, stream=None) -> dict:
        return pm_gemm_bench(c, self.A_op, self.B_op, C, self.scales, warmup, reps, stream)


# ---------------------------------------------------------------------- model
def pm_model_predict(cfgs_dev, n, theta, n_sm, t_out, stream=None):
    _check(_lib.pm_model_predict(_ptr(cfgs_dev), int(n), ctypes.byref(params(theta)), int(n_sm), _ptr(t_out),
                                 _stream(stream)), "pm_model_predict")


def pm_model_grad_workspace(n) -> int:
    b = ctypes.c_size_t()
    _check(_lib.pm_model_grad_workspace(int(n), ctypes.byref(b)), "pm_model_grad_workspace")
    return b.value


def pm_model_grad(cfgs_dev, n, theta, n_sm, t_meas, workspace, out, stream=None):
    _check(_lib.pm_model_grad(_ptr(cfgs_dev), int(n), ctypes.byref(params(theta)), int(n_sm), _ptr(t_meas),
                              _ptr(workspace), int(workspace.numel() * workspace.element_size()), _ptr(out),
                              _stream(stream)), "pm_model_grad")


def pm_model_grad_f64(cfgs_dev, n, theta, n_sm, t_meas, workspace, out, stream=None):
    """pm_model_grad in FP64 throughout: theta as N_PARAMS doubles, t_meas a float64 device tensor."""
    assert len(theta) == N_PARAMS
    th = (ctypes.c_double * N_PARAMS)(*[float(v) for v in theta])
    _check(_lib.pm_model_grad_f64(_ptr(cfgs_dev), int(n), ctypes.cast(th, ctypes.c_void_p), int(n_sm), _ptr(t_meas),
                                  _ptr(workspace), int(workspace.numel() * workspace.element_size()), _ptr(out),
                                  _stream(stream)), "pm_model_grad_f64")


def pm_model_grad_noalloc(cfgs_dev, n, theta, n_sm, t_meas, out, stream=None):
    """pm_model_grad with the library's built-in scratch array instead of a
    caller workspace (for callers that cannot allocate device memory)."""
    _check(_lib.pm_model_grad_noalloc(_ptr(cfgs_dev), int(n), ctypes.byref(params(theta)), int(n_sm), _ptr(t_meas),
                                      _ptr(out), _stream(stream)), "pm_model_grad_noalloc")


def pm_autotune_pick(MNK_dev, n, dtype, theta, n_sm, picks_dev, t_pred_dev, stream=None):
    _check(_lib.pm_autotune_pick(_ptr(MNK_dev), int(n), int(dtype), ctypes.byref(params(theta)), int(n_sm),
                                 _ptr(picks_dev), _ptr(t_pred_dev), _stream(stream)), "pm_autotune_pick")


def pm_autotune_topk(MNK_dev, n, dtype, theta, n_sm, k, picks_dev, t_pred_dev, stream=None):
    _check(_lib.pm_autotune_topk(_ptr(MNK_dev), int(n), int(dtype), ctypes.byref(params(theta)), int(n_sm), int(k),
                                 _ptr(picks_dev), _ptr(t_pred_dev), _stream(stream)), "pm_autotune_topk")


def pm_gemm_autotune(shape: pm_cfg, k, theta, n_sm, A_op, B_op, C, scales=None, warmup=3, reps=15, stream=None):
    """(picked pm_cfg, timing dict) of the model-pruned measured search."""
    pick = pm_cfg()
    res = pm_probe_result()
    _check(_lib.pm_gemm_autotune(ctypes.byref(shape), int(k), ctypes.byref(params(theta)), int(n_sm), _ptr(A_op),
                                 _ptr(B_op), _ptr(C), _ptr(scales), int(warmup), int(reps), _stream(stream),
                                 ctypes.byref(pick), ctypes.byref(res)), "pm_gemm_autotune")
    return pick, _timing(res)


def pm_grouped_predict(M_list, N, K, BM_list, BN_list, BK, stages, cta_group, dtype, theta, n_sm, stream=None):
    """Stage-model makespan (s) of one grouped launch with the given per-group tiles."""
    G = len(M_list)
    Mh = (ctypes.c_int32 * G)(*[int(m) for m in M_list])
    bm = (ctypes.c_int16 * G)(*[int(v) for v in BM_list])
    bn = (ctypes.c_int16 * G)(*[int(v) for v in BN_list])
    t = ctypes.c_float()
    _check(_lib.pm_grouped_predict(G, Mh, int(N), int(K), bm, bn, int(BK), int(stages), int(cta_group), int(dtype),
                                   ctypes.byref(params(theta)), int(n_sm), ctypes.byref(t), _stream(stream)),
           "pm_grouped_predict")
    return float(t.value)


def pm_grouped_grad(M_list, N, K, BM_list, BN_list, BK, stages, cta_group, dtype, theta, n_sm, stream=None):
    """(T_hat, dT_hat/dtheta) of one grouped launch, FP64 on the GPU."""
    G = len(M_list)
    Mh = (ctypes.c_int32 * G)(*[int(m) for m in M_list])
    bm = (ctypes.c_int16 * G)(*[int(v) for v in BM_list])
    bn = (ctypes.c_int16 * G)(*[int(v) for v in BN_list])
    assert len(theta) == N_PARAMS
    th = (ctypes.c_double * N_PARAMS)(*[float(v) for v in theta])
    out = (ctypes.c_double * N_GRAD_OUT)()
    _check(_lib.pm_grouped_grad(G, Mh, int(N), int(K), bm, bn, int(BK), int(stages), int(cta_group), int(dtype),
                                ctypes.cast(th, ctypes.c_void_p), int(n_sm), ctypes.cast(out, ctypes.c_void_p),
                                _stream(stream)), "pm_grouped_grad")
    return float(out[0]), np.array(out[1:], dtype=np.float64)


def pm_grouped_candidates(M_list, N, K, dtype, theta, n_sm, stream=None):
    """The grouped autotuner's 20 launch-level candidates: list of
    (t_pred, BM list, BN list, (BK, stages, cta_group))."""
    G = len(M_list)
    Mh = (ctypes.c_int32 * G)(*[int(m) for m in M_list])
    t = (ctypes.c_float * 20)()
    bm = (ctypes.c_int16 * (20 * G))()
    bn = (ctypes.c_int16 * (20 * G))()
    launch = (ctypes.c_int32 * 60)()
    _check(_lib.pm_grouped_candidates(G, Mh, int(N), int(K), int(dtype), ctypes.byref(params(theta)), int(n_sm),
                                      t, bm, bn, launch, _stream(stream)), "pm_grouped_candidates")
    return [(float(t[i]), list(bm[i * G:(i + 1) * G]), list(bn[i * G:(i + 1) * G]), tuple(launch[3 * i:3 * i + 3]))
            for i in range(20)]


def pm_grouped_autotune(M_list, N, K, dtype, theta, n_sm, stream=None):
    G = len(M_list)
    Mh = (ctypes.c_int32 * G)(*[int(m) for m in M_list])
    bm = (ctypes.c_int16 * G)()
    bn = (ctypes.c_int16 * G)()
    launch = (ctypes.c_int32 * 3)()
    t = ctypes.c_float()
    _check(_lib.pm_grouped_autotune(G, Mh, int(N), int(K), int(dtype), ctypes.byref(params(theta)), int(n_sm), bm,
                                    bn, launch, ctypes.byref(t), _stream(stream)), "pm_grouped_autotune")
    return float(t.value), list(bm), list(bn), tuple(launch)


def pm_grouped_gemm_autotune(M_list, N, K, theta, n_sm, k, A_op, B_op, C, warmup=2, reps=5, stream=None):
    """The grouped autotuner's k best launches timed on these operands; returns
    (t_pred, BM list, BN list, (BK, stages, cta_group), timing dict)."""
    G = len(M_list)
    Mh = (ctypes.c_int32 * G)(*[int(m) for m in M_list])
    bm = (ctypes.c_int16 * G)()
    bn = (ctypes.c_int16 * G)()
    launch = (ctypes.c_int32 * 3)()
    t = ctypes.c_float()
    res = pm_probe_result()
    _check(_lib.pm_grouped_gemm_autotune(G, Mh, int(N), int(K), ctypes.byref(params(theta)), int(n_sm), int(k),
                                         _ptr(A_op), _ptr(B_op), _ptr(C), int(warmup), int(reps), _stream(stream),
                                         bm, bn, launch, ctypes.byref(t), ctypes.byref(res)),
           "pm_grouped_gemm_autotune")
    return float(t.value), list(bm), list(bn), tuple(launch), _timing(res)


# ------------------------------------------------------- generic segment model
def segment_array(fields: dict) -> np.ndarray:
    """Structured pm_segment array from a dict of equal-length columns (missing columns are 0; execs 1)."""
    n = len(next(iter(fields.values())))
    a = np.zeros(n, dtype=SEGMENT_DTYPE)
    a["execs"] = 1
    for k, v in fields.items():
        a[k] = v
    return a


def pm_segment_predict(segs: np.ndarray, theta, psi, n_sm, stream=None) -> np.ndarray:
    """Generic-path time (FP64 seconds) of each pm_segment record, evaluated on the GPU."""
    import torch
    n = len(segs)
    dev = torch.from_numpy(np.ascontiguousarray(segs).view(np.uint8).copy()).cuda()
    out = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    assert len(psi) == N_PSI, "psi has %d entries, not %d" % (len(psi), N_PSI)
    ps = pm_segment_params((ctypes.c_double * N_PSI)(*[float(v) for v in psi]))
    _check(_lib.pm_segment_predict(_ptr(dev), int(n), ctypes.byref(params(theta)), ctypes.byref(ps), int(n_sm),
                                   _ptr(out), _stream(stream)), "pm_segment_predict")
    return out[:n].cpu().numpy()


def pm_model_set_reading(reading: int) -> None:
    """Process-wide reading of the stage model's open points (PM_READING_LITERAL / _MEASURED)."""
    _check(_lib.pm_model_set_reading(int(reading)), "pm_model_set_reading")


def pm_model_reading() -> int:
    return int(_lib.pm_model_reading())


# ---------------------------------------------------------------- diagnostics
def pm_last_error() -> str:
    return _lib.pm_last_error().decode(errors="replace")


def pm_shutdown() -> None:
    """Release the library's streams, host pipeline and descriptor caches (re-created on demand)."""
    _check(_lib.pm_shutdown(), "pm_shutdown")


def pm_clock_sample():
    """One read-only NVML sample of the current device as a dict (SM, maximum
    SM and memory clocks in MHz, power in W, clock event reasons, host
    monotonic time in s), or None where NVML cannot be read."""
    c = pm_clock()
    if _lib.pm_clock_sample(ctypes.byref(c)) != PM_OK:
        return None
    return dict(sm_mhz=c.sm_mhz, sm_max_mhz=c.sm_max_mhz, mem_mhz=c.mem_mhz, power_w=c.power_mw / 1e3,
                reasons=clock_reason_names(c.reasons), host_time_s=c.host_time_s)


def pm_device_status(clear=True) -> int:
    return int(_lib.pm_device_status(1 if clear else 0))


def pm_watchdog_selftest(limit_us=200000, stream=None) -> int:
    return int(_lib.pm_watchdog_selftest(int(limit_us), _stream(stream)))


def pm_version() -> int:
    return int(_lib.pm_version())


def sm_count(device=None) -> int:
    import torch
    return torch.cuda.get_device_properties(device or torch.cuda.current_device()).multi_processor_count
