"""Seeded synthetic inputs shared by the CPU oracle, the tests and the bench.

This module holds no arithmetic of the performance model, of the GEMM or of
the probes: it only draws numbers.  Every generator is counter based, so any
slice of a stream (one row of a matrix, one sampled element) can be drawn on
its own and equals the same slice of the whole stream.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014; the 64-bit finaliser as published by
S. Vigna in splitmix64.c).  Output i (0-based) of the stream with seed s is
mix(s + (i + 1) * 0x9E3779B97F4A7C15).

Recipes (the workloads of the paper's Blackwell validation, Sec. V, re-drawn
synthetically; the paper's own suites are not used):
  * uniform[-1, 1): top 24 bits u of a draw, x = u * 2^-23 - 1 (exact in FP32);
  * normal(0, 1): Box-Muller on two consecutive draws, computed in FP64 and
    rounded once to FP32;
  * cyclic pointer-chase permutation: nodes visited in the order of a random
    permutation (argsort of one draw per node), which is a uniformly random
    single cycle;
  * grouped-GEMM row counts: M_g = round(exp(U[ln 16, ln 4096]));
  * model configuration batches: shapes log-uniform in [16, 16384] rounded to
    a multiple of 16, tile configuration uniform over the enumerated space,
    dtype uniform.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+n-1 of the SplitMix64 stream with this seed (uint64)."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed) + idx * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _splitmix64_chunked(seed: int, n: int, offset: int, fn, out: np.ndarray, chunk: int = 1 << 24):
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        out[s:e] = fn(splitmix64(seed, e - s, offset + s))
    return out


def _u24_to_pm1(z: np.ndarray) -> np.ndarray:
    u = (z >> np.uint64(40)).astype(np.float32)
    return u * np.float32(2.0 ** -23) - np.float32(1.0)


def uniform_pm1(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n FP32 values uniform on [-1, 1) with 2^-23 spacing, stream positions offset..offset+n-1."""
    out = np.empty(n, dtype=np.float32)
    return _splitmix64_chunked(seed, n, offset, _u24_to_pm1, out)


def uniform01_f64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n FP64 values uniform on [0, 1) from the top 53 bits."""
    z = splitmix64(seed, n, offset)
    return (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def normal(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n FP32 normal(0,1) values; value j uses stream draws 2*(offset+j) and 2*(offset+j)+1."""
    out = np.empty(n, dtype=np.float32)
    chunk = 1 << 23
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        z = splitmix64(seed, 2 * (e - s), 2 * (offset + s)).reshape(-1, 2)
        u1 = ((z[:, 0] >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53  # (0, 1]
        u2 = (z[:, 1] >> np.uint64(11)).astype(np.float64) * 2.0 ** -53          # [0, 1)
        out[s:e] = (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)).astype(np.float32)
    return out


def matrix(seed: int, rows: int, cols: int, dist: str = "uniform", offset: int = 0) -> np.ndarray:
    """A rows x cols FP32 row-major matrix; element (i, j) is stream position offset + i*cols + j."""
    n = rows * cols
    if dist == "uniform":
        v = uniform_pm1(seed, n, offset)
    elif dist == "normal":
        v = normal(seed, n, offset)
    else:
        raise ValueError(dist)
    return v.reshape(rows, cols)


def matrix_rows(seed: int, rows: np.ndarray, cols: int, dist: str = "uniform", offset: int = 0) -> np.ndarray:
    """The listed rows of matrix(seed, *, cols, dist, offset), drawn without the rest."""
    out = np.empty((len(rows), cols), dtype=np.float32)
    for r, i in enumerate(rows):
        out[r] = matrix(seed, 1, cols, dist, offset + int(i) * cols)[0]
    return out


def gemm_operands(M: int, N: int, K: int, seed: int, dist: str = "uniform"):
    """Row-major FP32 A [M, K] and B [K, N]: A takes stream positions [0, MK), B [MK, MK+KN)."""
    A = matrix(seed, M, K, dist, 0)
    B = matrix(seed, K, N, dist, M * K)
    return A, B


def integer_matrix(seed: int, rows: int, cols: int, lo: int = -2, hi: int = 2, offset: int = 0) -> np.ndarray:
    """FP32 matrix of integers uniform on [lo, hi] (exact in e4m3, bf16 and tf32)."""
    z = splitmix64(seed, rows * cols, offset)
    span = np.uint64(hi - lo + 1)
    v = (z >> np.uint64(32)) % span
    return (v.astype(np.int64) + lo).astype(np.float32).reshape(rows, cols)


def sampled_rows(seed: int, M: int, count: int) -> np.ndarray:
    """count distinct row indices of [0, M), sorted, chosen by one draw per row."""
    if count >= M:
        return np.arange(M, dtype=np.int64)
    keys = splitmix64(seed ^ 0x5A5A5A5A, M)
    return np.sort(np.argsort(keys, kind="stable")[:count]).astype(np.int64)


def cyclic_permutation(n_nodes: int, seed: int) -> np.ndarray:
    """next[i] (uint32) of one random cycle through all n_nodes nodes."""
    order = np.argsort(splitmix64(seed, n_nodes), kind="stable").astype(np.uint32)
    nxt = np.empty(n_nodes, dtype=np.uint32)
    nxt[order] = np.roll(order, -1)
    return nxt


def pchase_buffer(n_nodes: int, seed: int, stride_bytes: int = 64) -> np.ndarray:
    """Pointer-chase memory image: node i sits at byte offset stride_bytes*i and holds next[i] as uint32."""
    words = stride_bytes // 4
    buf = np.zeros(n_nodes * words, dtype=np.uint32)
    buf[::words] = cyclic_permutation(n_nodes, seed)
    return buf


def grouped_m(G: int = 64, seed: int = 3, lo: int = 16, hi: int = 4096) -> np.ndarray:
    """Row counts of the grouped GEMM: M_g = round(exp(U[ln lo, ln hi])) (int32)."""
    u = uniform01_f64(seed, G)
    m = np.rint(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo))))
    return np.clip(m, lo, hi).astype(np.int32)


# Tile-configuration space of the GEMM sweep: BM, BN in {64,128,256}, two BK
# values per dtype, 2..6 pipeline stages, cta_group 1 or 2 (180 per dtype).
BM_SET = (64, 128, 256)
BN_SET = (64, 128, 256)
BK_SET = {0: (32, 64), 1: (64, 128), 2: (64, 128)}   # dtype 0 = FP32 (3xTF32), 1 = BF16, 2 = FP8 e4m3
STAGE_SET = (2, 3, 4, 5, 6)
CTA_GROUP_SET = (1, 2)


def tile_space(dtype: int):
    """The 180 (BM, BN, BK, stages, cta_group) tuples in lexicographic order."""
    return [(bm, bn, bk, s, g) for bm in BM_SET for bn in BN_SET for bk in BK_SET[dtype]
            for s in STAGE_SET for g in CTA_GROUP_SET]


def model_config_batch(n: int, seed: int = 4):
    """Structured array of n random GEMM configurations (fields of the library's config record)."""
    z = splitmix64(seed, 6 * n).reshape(n, 6)
    u = (z[:, :3] >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    shp = np.exp(np.log(16.0) + u * (np.log(16384.0) - np.log(16.0)))
    shp = np.clip(np.rint(shp / 16.0) * 16.0, 16, 16384).astype(np.int32)
    dtype = ((z[:, 3] >> np.uint64(32)) % np.uint64(3)).astype(np.int8)
    tidx = ((z[:, 4] >> np.uint64(32)) % np.uint64(180)).astype(np.int64)
    spaces = {d: np.array(tile_space(d), dtype=np.int32) for d in (0, 1, 2)}
    tiles = np.empty((n, 5), dtype=np.int32)
    for d in (0, 1, 2):
        m = dtype == d
        tiles[m] = spaces[d][tidx[m]]
    return dict(M=shp[:, 0], N=shp[:, 1], K=shp[:, 2], BM=tiles[:, 0], BN=tiles[:, 1], BK=tiles[:, 2],
                stages=tiles[:, 3], cta_group=tiles[:, 4], dtype=dtype)
