"""Pins of the oracle's GEMM and number-format references (CPU only).

Each check compares the oracle with something other than itself: numpy's
FP64 matmul, exact integer arithmetic, permutation structure, torch's CPU
casts, or bit-level definitions of the formats.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (7, 5, 3), (64, 48, 32), (256, 256, 256), (130, 97, 211)])
def test_gemm_matches_numpy_fp64(M, N, K):
    A, B = S.gemm_operands(M, N, K, seed=0)
    C = O.gemm_f64(A, B)
    ref = A.astype(np.float64) @ B.astype(np.float64)
    # Products of FP32 values are exact in FP64; only the summation order differs.
    assert np.max(np.abs(C - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_gemm_integer_entries_exact():
    # Entries in {-2..2}: every partial sum is an integer below 2^53, so the
    # FP64 result is the exact integer product (compared with int64 matmul).
    A = S.integer_matrix(11, 96, 300)
    B = S.integer_matrix(12, 300, 80)
    C = O.gemm_f64(A, B)
    ref = A.astype(np.int64) @ B.astype(np.int64)
    assert np.array_equal(C, ref.astype(np.float64))


def test_gemm_identity_and_permutation():
    A, _ = S.gemm_operands(33, 1, 40, seed=5)
    I = np.eye(40, dtype=np.float32)
    assert np.array_equal(O.gemm_f64(A, I), A.astype(np.float64))
    perm = np.argsort(S.splitmix64(9, 40))
    P = np.eye(40, dtype=np.float32)[:, perm]        # column permutation
    assert np.array_equal(O.gemm_f64(A, P), A[:, perm].astype(np.float64))


def test_gemm_sampled_rows_equal_full_rows():
    M, N, K = 300, 40, 64
    A, B = S.gemm_operands(M, N, K, seed=2, dist="normal")
    rows = S.sampled_rows(7, M, 17)
    Ar = S.matrix_rows(2, rows, K, "normal", 0)
    assert np.array_equal(Ar, A[rows])
    assert np.array_equal(O.gemm_f64(Ar, B), O.gemm_f64(A, B)[rows])


def _bits(x):
    return np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)


def _special_values():
    rng = S.splitmix64(21, 4096)
    raw = (rng >> np.uint64(32)).astype(np.uint32)
    x = raw.view(np.float32)
    x = x[np.isfinite(x)]
    extra = np.array([0.0, -0.0, 1.0, -1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -11,
                      1.0 + 3 * 2 ** -11, 3.4e38, 1e-40, -1e-45, 1.17549435e-38], dtype=np.float32)
    return np.concatenate([x, extra, S.normal(3, 2048)])


def test_bf16_matches_torch_cast():
    x = _special_values()
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    got = O.to_bf16(x)
    finite = np.isfinite(ref)
    assert np.array_equal(_bits(got[finite]), _bits(ref[finite]))


def test_tf32_split_bit_definition():
    x = _special_values()
    x = x[np.abs(x) < 1e38]
    hi, lo = O.tf32_split(x)
    # Bit definition of round-to-nearest-even to 10 mantissa bits.
    b = _bits(x).astype(np.uint64)
    rnd = (b + np.uint64(0xFFF) + ((b >> np.uint64(13)) & np.uint64(1))) & np.uint64(0xFFFFE000)
    ref_hi = rnd.astype(np.uint32).view(np.float32)
    assert np.array_equal(_bits(hi), _bits(ref_hi))
    assert np.all((_bits(hi) & 0x1FFF) == 0) and np.all((_bits(lo) & 0x1FFF) == 0)
    # hi + lo reproduces x to 2^-22 relative (two 11-bit significands).
    # (normal range only: below 2^-100 the low half becomes subnormal)
    nz = np.abs(x) >= 2.0 ** -100
    rel = np.abs((hi.astype(np.float64)[nz] + lo[nz] - x[nz]) / x[nz])
    assert np.all(rel <= 2.0 ** -21)


def test_e4m3_all_codes_round_trip():
    codes = np.arange(256, dtype=np.uint8)
    vals = O.from_e4m3(codes)
    nan = np.isnan(vals)
    assert nan.sum() == 2                                  # 0x7F and 0xFF
    back = O.to_e4m3(vals[~nan])
    # +0 and -0 keep their sign bits
    assert np.array_equal(back, codes[~nan])
    assert vals[0x7E] == 448.0 and vals[0x08] == 2.0 ** -6 and vals[0x01] == 2.0 ** -9


def test_e4m3_matches_torch_in_range():
    x = np.concatenate([S.normal(5, 4096) * np.float32(100.0), S.uniform_pm1(6, 4096) * np.float32(0.01)])
    x = x[np.abs(x) <= 448.0]
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(O.to_e4m3(x), ref)


def test_e4m3_saturates():
    x = np.array([448.0, 463.99, 464.0, 500.0, 1e6, -1e30, np.inf, -np.inf], dtype=np.float32)
    v = O.from_e4m3(O.to_e4m3(x))
    assert np.array_equal(np.abs(v), np.full(len(x), 448.0, dtype=np.float32))
    assert np.array_equal(np.sign(v), np.sign(x))


def test_fp8_quantised_gemm_error_within_bound():
    # Quantisation of N(0,1) operands with the per-tensor 448/amax scale: the
    # relative Frobenius error of the product stays near 0.04 and below 0.06.
    M = N = K = 128
    A, B = S.gemm_operands(M, N, K, seed=2, dist="normal")
    sa, sb = O.fp8_scale(A), O.fp8_scale(B)
    Aq = O.from_e4m3(O.to_e4m3(A * sa)).astype(np.float64) / sa
    Bq = O.from_e4m3(O.to_e4m3(B * sb)).astype(np.float64) / sb
    C = O.gemm_f64(A, B)
    Cq = O.gemm_f64_f64(Aq, Bq)
    err = np.linalg.norm(Cq - C) / np.linalg.norm(C)
    assert 0.01 < err < 0.06
