"""CPU FP64 oracle of the GB300 performance-model hot path (arxiv 2605.04178).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the bench's
CPU-baseline arm import this module; the product library never does, and it
imports nothing from the product package.  The arithmetic lives in
oracle.cpp (FP64, plain loops, one function per passage of the paper); this
file compiles it with g++ and wraps it for numpy arrays.

Parity status of each part (pins are in tests/test_oracle_*.py):
  gemm_f64            pinned: numpy FP64 matmul, integer matrices, identity/permutation
  to_bf16/tf32/e4m3   pinned: exhaustive/structural checks against the format definitions
  triad_f32           pinned: exact rational arithmetic (fractions) on random cases
  stencil5_f32        pinned: exact rational arithmetic of each rounding step on random grids
  pchase              pinned: single-cycle walk returns to its start after n hops
  model_batch         pinned: hand-evaluated rows, closed forms, homogeneity, monotonicity
  model gradient      pinned: central differences and Euler's homogeneity identity
  autotune            pinned: brute force in plain Python on small spaces
  grouped model       pinned: reduces to the single-GEMM stage time for one group; brute-force
                      worker loop of the launch's schedule; central differences and Euler's
                      identity for its gradient
  segment_predict     pinned: closed forms of each term (Eq. 16 off, pure transfers, extra launches,
                      executions, concurrent streams), hand-evaluated rows, homogeneity
  mma/tmem probe sums closed forms (exact integer arithmetic)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

KIND_GEMM, KIND_COPY, KIND_TRIAD, KIND_TMA2D = 0, 1, 2, 3
DT_FP32, DT_BF16, DT_FP8 = 0, 1, 2
N_PARAMS = 18

PARAM_NAMES = ("T_launch", "B_sus", "B_peak", "w0", "L_TMA", "B_TMA", "R_tf32", "R_bf16", "R_fp8",
               "L_mma", "BW_tmem_rd", "BW_tmem_wr", "L_mbar", "L_tmem_mgmt", "S_2SM", "c_alpha", "rho_L2",
               "B_drain")
# Time-like parameters (seconds) and rate-like parameters (bytes or FLOP per
# second); the rest (w0, S_2SM, c_alpha, rho_L2) are dimensionless or sizes.
LATENCY_IDX = (0, 4, 9, 12, 13)
RATE_IDX = (1, 2, 5, 6, 7, 8, 10, 11, 17)


def build(force: bool = False) -> str:
    """Compile oracle.cpp into oracle/_build/liboracle.so (g++, OpenMP, FP64)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
               _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            lib.orc_gemm_f64.argtypes = [P, P, i64, i64, i64, P]
            lib.orc_gemm_f64_f64.argtypes = [P, P, i64, i64, i64, P]
            lib.orc_to_bf16.argtypes = [P, i64, P]
            lib.orc_tf32_split.argtypes = [P, i64, P, P]
            lib.orc_to_e4m3.argtypes = [P, i64, P]
            lib.orc_from_e4m3.argtypes = [P, i64, P]
            lib.orc_triad_f32.argtypes = [P, P, ctypes.c_float, i64, P]
            lib.orc_pchase.argtypes = [P, i64, ctypes.c_uint32, i64]
            lib.orc_pchase.restype = ctypes.c_uint32
            lib.orc_cfg_valid.argtypes = [ctypes.c_int] * 7
            lib.orc_cfg_valid.restype = ctypes.c_int
            lib.orc_model_batch.argtypes = [i64] + [P] * 11 + [P, ctypes.c_int, P, P]
            lib.orc_model_loss_grad.argtypes = [i64] + [P] * 11 + [P, ctypes.c_int, P, P, P]
            lib.orc_autotune.argtypes = [i64, P, ctypes.c_int, P, ctypes.c_int, P, P]
            lib.orc_grouped_predict.argtypes = [ctypes.c_int, P, ctypes.c_int32, ctypes.c_int32, P, P,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                P, ctypes.c_int]
            lib.orc_grouped_predict.restype = ctypes.c_double
            lib.orc_grouped_predict_grad.argtypes = lib.orc_grouped_predict.argtypes + [P]
            lib.orc_grouped_predict_grad.restype = ctypes.c_double
            lib.orc_grouped_autotune.argtypes = [ctypes.c_int, P, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.c_int, P, ctypes.c_int, P, P, P]
            lib.orc_grouped_autotune.restype = ctypes.c_double
            lib.orc_set_reading.argtypes = [ctypes.c_int]
            lib.orc_reading.restype = ctypes.c_int
            lib.orc_segment_predict.argtypes = [i64] + [P] * 11 + [P, P, ctypes.c_int, P]
            lib.orc_stencil5_f32.argtypes = [P, i64, i64, P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ----------------------------------------------------------------------------- GEMM
def gemm_f64(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """FP64 C = A.B of FP32 row-major A [M, K], B [K, N] (the definition, k ascending)."""
    A = _c(A, np.float32)
    B = _c(B, np.float32)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    C = np.empty((M, N), dtype=np.float64)
    _load().orc_gemm_f64(_ptr(A), _ptr(B), M, N, K, _ptr(C))
    return C


def gemm_f64_f64(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    A = _c(A, np.float64)
    B = _c(B, np.float64)
    M, K = A.shape
    _, N = B.shape
    C = np.empty((M, N), dtype=np.float64)
    _load().orc_gemm_f64_f64(_ptr(A), _ptr(B), M, N, K, _ptr(C))
    return C


# ----------------------------------------------------------------------------- formats
def to_bf16(x: np.ndarray) -> np.ndarray:
    """FP32 values rounded to bf16 (RNE), returned as FP32."""
    x = _c(x, np.float32)
    y = np.empty_like(x)
    _load().orc_to_bf16(_ptr(x), x.size, _ptr(y))
    return y


def tf32_split(x: np.ndarray):
    """(hi, lo) with hi = tf32_rn(x), lo = tf32_rn(x - hi), both FP32 with 13 zero low bits."""
    x = _c(x, np.float32)
    hi = np.empty_like(x)
    lo = np.empty_like(x)
    _load().orc_tf32_split(_ptr(x), x.size, _ptr(hi), _ptr(lo))
    return hi, lo


def to_e4m3(x: np.ndarray) -> np.ndarray:
    """FP8 e4m3 codes (uint8) of FP32 values, RNE with saturation to +-448."""
    x = _c(x, np.float32)
    y = np.empty(x.shape, dtype=np.uint8)
    _load().orc_to_e4m3(_ptr(x), x.size, _ptr(y))
    return y


def from_e4m3(code: np.ndarray) -> np.ndarray:
    code = _c(code, np.uint8)
    y = np.empty(code.shape, dtype=np.float32)
    _load().orc_from_e4m3(_ptr(code), code.size, _ptr(y))
    return y


def fp8_scale(x: np.ndarray) -> np.float32:
    """Per-tensor scale 448 / max|x| in FP32 (one IEEE division)."""
    amax = np.float32(np.max(np.abs(x)))
    return np.float32(np.float32(448.0) / amax)


# ----------------------------------------------------------------------------- probes
def triad_f32(b: np.ndarray, c: np.ndarray, s: float) -> np.ndarray:
    b = _c(b, np.float32)
    c = _c(c, np.float32)
    a = np.empty_like(b)
    _load().orc_triad_f32(_ptr(b), _ptr(c), ctypes.c_float(s), b.size, _ptr(a))
    return a


def pchase(buf: np.ndarray, stride_words: int, start: int, hops: int) -> int:
    buf = _c(buf, np.uint32)
    return int(_load().orc_pchase(_ptr(buf), stride_words, start, hops))


# ----------------------------------------------------------------------------- model
def cfg_valid(BM, BN, BK, s, g, dtype, tmem_a=0) -> bool:
    """Tile-space validity; tmem_a = 1 asks for TMEM strategy B (Sec. III-A.1)."""
    return bool(_load().orc_cfg_valid(int(BM), int(BN), int(BK), int(s), int(g), int(dtype), int(tmem_a)))


_FIELDS = ("M", "N", "K", "BM", "BN", "BK", "stages", "cta_group", "dtype", "kind", "tmem_a")


def _soa(cfgs: dict):
    n = len(cfgs["M"])
    cols = []
    for f in _FIELDS:
        v = cfgs.get(f)
        if v is None:
            v = np.zeros(n, dtype=np.int32)
        cols.append(_c(v, np.int32))
    return n, cols


def model_batch(cfgs: dict, theta, n_sm: int, grad: bool = False):
    """Stage-model prediction (FP64) per configuration; with grad, also dT/dtheta [n, N_PARAMS]."""
    n, cols = _soa(cfgs)
    th = _c(theta, np.float64)
    assert th.size == N_PARAMS
    t = np.empty(n, dtype=np.float64)
    g = np.empty((n, N_PARAMS), dtype=np.float64) if grad else None
    _load().orc_model_batch(n, *[_ptr(c) for c in cols], _ptr(th), int(n_sm), _ptr(t),
                            _ptr(g) if grad else None)
    return (t, g) if grad else t


def model_loss_grad(cfgs: dict, theta, n_sm: int, t_meas):
    """Mean squared log error and its gradient in theta (FP64)."""
    n, cols = _soa(cfgs)
    th = _c(theta, np.float64)
    tm = _c(t_meas, np.float64)
    loss = np.zeros(1, dtype=np.float64)
    grad = np.zeros(N_PARAMS, dtype=np.float64)
    _load().orc_model_loss_grad(n, *[_ptr(c) for c in cols], _ptr(th), int(n_sm), _ptr(tm),
                                _ptr(loss), _ptr(grad))
    return float(loss[0]), grad


def autotune(MNK: np.ndarray, dtype: int, theta, n_sm: int):
    """Model-optimal (BM, BN, BK, stages, cta_group) per shape, first minimum in lexicographic order."""
    MNK = _c(MNK, np.int32).reshape(-1, 3)
    n = MNK.shape[0]
    th = _c(theta, np.float64)
    pick = np.zeros((n, 5), dtype=np.int32)
    t = np.zeros(n, dtype=np.float64)
    _load().orc_autotune(n, _ptr(MNK), int(dtype), _ptr(th), int(n_sm), _ptr(pick), _ptr(t))
    return pick, t


def grouped_predict(Mg, N, K, BMg, BNg, BK, s, g, dtype, theta, n_sm) -> float:
    Mg = _c(Mg, np.int32)
    BMg = _c(BMg, np.int32)
    BNg = _c(BNg, np.int32)
    th = _c(theta, np.float64)
    return float(_load().orc_grouped_predict(len(Mg), _ptr(Mg), int(N), int(K), _ptr(BMg), _ptr(BNg),
                                             int(BK), int(s), int(g), int(dtype), _ptr(th), int(n_sm)))


def grouped_predict_grad(Mg, N, K, BMg, BNg, BK, s, g, dtype, theta, n_sm):
    """(T_hat, dT_hat/dtheta [N_PARAMS]) of one grouped launch (dual numbers)."""
    Mg = _c(Mg, np.int32)
    BMg = _c(BMg, np.int32)
    BNg = _c(BNg, np.int32)
    th = _c(theta, np.float64)
    grad = np.zeros(N_PARAMS, dtype=np.float64)
    t = _load().orc_grouped_predict_grad(len(Mg), _ptr(Mg), int(N), int(K), _ptr(BMg), _ptr(BNg), int(BK), int(s),
                                         int(g), int(dtype), _ptr(th), int(n_sm), _ptr(grad))
    return float(t), grad


def grouped_autotune(Mg, N, K, dtype, theta, n_sm):
    """(T_hat, BM per group, BN per group, (BK, stages, cta_group)) of the best grouped launch."""
    Mg = _c(Mg, np.int32)
    G = len(Mg)
    th = _c(theta, np.float64)
    bm = np.zeros(G, dtype=np.int32)
    bn = np.zeros(G, dtype=np.int32)
    launch = np.zeros(3, dtype=np.int32)
    t = _load().orc_grouped_autotune(G, _ptr(Mg), int(N), int(K), int(dtype), _ptr(th), int(n_sm),
                                     _ptr(bm), _ptr(bn), _ptr(launch))
    return float(t), bm, bn, tuple(int(v) for v in launch)


def stencil5_f32(x: np.ndarray) -> np.ndarray:
    """Five-point stencil of a 2-D FP32 grid (interior 0.5 x + 0.125 (vertical + horizontal sums),
    every operation rounded separately; border copied)."""
    x = _c(x, np.float32)
    assert x.ndim == 2
    y = np.empty_like(x)
    _load().orc_stencil5_f32(_ptr(x), x.shape[0], x.shape[1], _ptr(y))
    return y


_SEG_F64 = ("flops", "bytes", "working_set", "h2d_bytes", "d2h_bytes")
_SEG_I32 = ("cls", "precision", "kernels", "syncs", "execs", "streams")
N_PSI = 17


def segment_predict(segs: dict, theta, psi, n_sm: int) -> np.ndarray:
    """Generic-path time (FP64) of each segment; segs holds equal-length columns
    (missing: 0, execs 1)."""
    n = len(next(iter(segs.values())))
    cols = [_c(segs.get(f, np.zeros(n)), np.float64) for f in _SEG_F64]
    cols += [_c(segs.get(f, np.ones(n) if f == "execs" else np.zeros(n)), np.int32) for f in _SEG_I32]
    th = _c(theta, np.float64)
    ps = _c(psi, np.float64)
    assert th.size == N_PARAMS and ps.size == N_PSI
    t = np.empty(n, dtype=np.float64)
    _load().orc_segment_predict(n, *[_ptr(c) for c in cols], _ptr(th), _ptr(ps), int(n_sm), _ptr(t))
    return t


READING_LITERAL, READING_MEASURED = 0, 1


def set_reading(reading: int) -> None:
    """Select the readings of the stage model's open points (process-wide):
    0 the literal equations (L_mma per K-step, alpha = 1 - c/s, T_sync in Eqs. 7 and 8,
    TMEM management amortised per K-step),
    1 the readings measured on the GPU's kernels (L_mma per tensor-pipe instruction,
    alpha = 1 - c/(s-1), T_sync once, the ring bubble (T_tma + T_c + T_sync)/s as a
    lower bound of T_step, B_TMA scaled by the L2-residency factor
    rho(W) = 1 + (rho_L2 - 1) exp(-W/w0) over the launch's working set W, TMEM
    management once per launch, 64-row one-SM tiles at the tensor time of 128 rows, and
    each tile of a launch whose accumulator cannot be double-buffered paying its drain,
    4 BM BN / B_drain, before the next tile starts)."""
    _load().orc_set_reading(int(reading))


def reading() -> int:
    return int(_load().orc_reading())


def prior_theta(n_sm: int, f_hz: float = 1.9e9, reading: int = READING_MEASURED) -> np.ndarray:
    """Prior parameter vector built from the paper's printed values (Table "parameters",
    Sec. II-A sustained figures); cycles are converted with the clock f_hz.  c_alpha puts
    alpha in the printed 0.85-0.95 range under either overlap law."""
    th = np.zeros(N_PARAMS, dtype=np.float64)
    th[0] = 5e-6                      # launch overhead, 5-12 us (Sec. V-B, memory-bound class)
    th[1] = 6.8e12                    # sustained HBM (Sec. II-A)
    th[2] = 8.0e12                    # HBM peak (Table "arch-params")
    th[3] = 64.0 * 2 ** 20            # w0, tunable (Eq. 16)
    th[4] = 420.0 / f_hz              # L_TMA 420 cycles
    th[5] = th[1] / n_sm              # B_TMA per SM (not printed)
    th[7] = 8192.0 * f_hz             # dense BF16 FLOP/cycle/SM
    th[6] = th[7] / 2.0               # TF32 at half the BF16 rate
    th[8] = 2.0 * th[7]               # FP8 at twice the BF16 rate (2,250 vs 4,500 TFLOPS)
    th[9] = 12.0 / f_hz               # tcgen05.mma latency 11-14 cycles
    th[10] = 16e12                    # TMEM read
    th[11] = 8e12                     # TMEM write
    th[12] = 45.0 / f_hz              # L_mbar 40-50 cycles
    th[13] = 100e-9                   # TMEM alloc + dealloc (not printed)
    th[14] = 1.0                      # S_2SM
    # alpha(2) = 0.85, alpha(6) = 0.95 (reading 0); alpha(2) = 0.85, alpha(3) = 0.925 (reading 1)
    th[15] = 0.3 if reading == READING_LITERAL else 0.15
    th[16] = th[2] / th[1]            # rho_L2: an L2-resident launch loads at the HBM peak/sustained ratio
    th[17] = th[1] / n_sm             # B_drain per SM (not printed): the SM's share of sustained HBM, like B_TMA
    return th


# ----------------------------------------------------------------- instruction probes
def mma_probe_value(n: int, dtype: int) -> np.float32:
    """D[0][0] after n MMAs of 1.0 x 1.0 with K = 32 bytes of each operand row
    (8 TF32, 16 BF16, 32 FP8 products per instruction), accumulated exactly."""
    k = {DT_FP32: 8, DT_BF16: 16, DT_FP8: 32}[dtype]
    return np.float32(n * k)


def tmem_probe_sums(iters: int, store: bool) -> np.ndarray:
    """Per-thread sums (mod 2^32) of the TMEM probe for the 256 threads of one
    SM: thread t covers lane 32*(w%4) + t%32 and columns 256*(w/4) .. +255
    (w = t // 32); lanes hold lane*512 + column, loads sum `iters` passes,
    stores leave lane*512 + column + iters - 1."""
    t = np.arange(256, dtype=np.int64)
    w = t // 32
    lane = 32 * (w % 4) + t % 32
    c0 = 256 * (w // 4)
    col_sum = 256 * c0 + 255 * 256 // 2
    if store:
        s = 256 * 512 * lane + col_sum + 256 * (iters - 1)
    else:
        s = iters * (256 * 512 * lane + col_sum)
    return (s % (1 << 32)).astype(np.uint32)
