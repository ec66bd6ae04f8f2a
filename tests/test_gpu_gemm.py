"""GPU parity of the tcgen05 GEMM family and its operand preparation against
the FP64 CPU oracle.

  * operand preparation: bf16 / tf32 hi-lo / e4m3 codes bit-exact;
  * integer operands in {-2..2}: every tile configuration of every dtype
    gives the exact integer product (bit-exact for BF16 and three-pass TF32;
    FP8 only adds the one rounding of the 1/(s_A s_B) rescale);
  * real-valued operands: FP32 normwise-max error <= 1e-5, BF16 relative
    Frobenius <= 2e-2, FP8 e4m3 <= 6e-2 against C = A.B in FP64.
"""
import functools

import numpy as np
import pytest

import oracle as O
import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT_NAMES = {0: "fp32", 1: "bf16", 2: "fp8"}


def run_gemm(lib, A, B, c, dtype):
    M, K = A.shape
    _, N = B.shape
    ops = lib.GemmOperands(dtype, M, N, K)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    ops.prepare(Ad, Bd)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    ops.run(c, C)
    torch.cuda.synchronize()
    assert lib.pm_device_status(True) == lib.PM_OK
    return C.cpu().numpy(), ops


def valid_space(dt, tmem_a=0):
    return [t for t in S.tile_space(dt) if O.cfg_valid(*t, dt, tmem_a)]


def space_ids(dt, tmem_a=0):
    return ["%s-bm%d-bn%d-bk%d-s%d-g%d" % ((DT_NAMES[dt],) + t) for t in valid_space(dt, tmem_a)]


B_SPACE = [(dt, t) for dt in (0, 1, 2) for t in valid_space(dt, 1)]
B_IDS = ["tmemB-" + i for dt in (0, 1, 2) for i in space_ids(dt, 1)]


# ------------------------------------------------------------------ operand prep
@pytest.mark.parametrize("M,N,K", [(33, 70, 96), (256, 128, 512)])
def test_prepare_bf16_bit_exact(lib, M, N, K):
    A, B = S.gemm_operands(M, N, K, seed=2, dist="normal")
    ops = lib.GemmOperands(1, M, N, K)
    ops.prepare(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    a = ops.A_op.view(torch.int16).cpu().numpy().astype(np.uint16).astype(np.uint32) << 16
    b = ops.B_op.view(torch.int16).cpu().numpy().astype(np.uint16).astype(np.uint32) << 16
    assert np.array_equal(a.view(np.float32).reshape(M, K), O.to_bf16(A))
    assert np.array_equal(b.view(np.float32).reshape(N, K), O.to_bf16(B.T.copy()))


@pytest.mark.parametrize("M,N,K", [(33, 70, 96), (512, 512, 512)])
def test_prepare_tf32_split_bit_exact(lib, M, N, K):
    A, B = S.gemm_operands(M, N, K, seed=0)
    ops = lib.GemmOperands(0, M, N, K)
    ops.prepare(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    a = ops.A_op.view(torch.float32).cpu().numpy().reshape(2, M, K)
    b = ops.B_op.view(torch.float32).cpu().numpy().reshape(2, N, K)
    hi, lo = O.tf32_split(A)
    assert np.array_equal(a[0].view(np.uint32), hi.view(np.uint32)) and np.array_equal(a[1].view(np.uint32), lo.view(np.uint32))
    hi, lo = O.tf32_split(B.T.copy())
    assert np.array_equal(b[0].view(np.uint32), hi.view(np.uint32)) and np.array_equal(b[1].view(np.uint32), lo.view(np.uint32))


@pytest.mark.parametrize("M,N,K", [(33, 70, 96), (1024, 512, 256)])
def test_prepare_fp8_codes_bit_exact(lib, M, N, K):
    A, B = S.gemm_operands(M, N, K, seed=2, dist="normal")
    ops = lib.GemmOperands(2, M, N, K)
    ops.prepare(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    sc = ops.scales.cpu().numpy()
    sa, sb = O.fp8_scale(A), O.fp8_scale(B)
    assert sc[0] == sa and sc[1] == sb
    assert np.array_equal(ops.A_op.cpu().numpy().reshape(M, K), O.to_e4m3(A * sa))
    assert np.array_equal(ops.B_op.cpu().numpy().reshape(N, K), O.to_e4m3(B.T.copy() * sb))


# -------------------------------------------------------- exact integer products
def _int_case(M, N, K):
    A = S.integer_matrix(11, M, K)
    B = S.integer_matrix(12, K, N)
    return A, B, O.gemm_f64(A, B)


@pytest.mark.parametrize("t", valid_space(1), ids=space_ids(1))
def test_exact_integer_bf16(lib, t):
    A, B, ref = _int_case(300, 200, 320)
    C, _ = run_gemm(lib, A, B, lib.cfg(300, 200, 320, *t, dtype=1), 1)
    assert np.array_equal(C.astype(np.float64), ref)


@pytest.mark.parametrize("t", valid_space(0), ids=space_ids(0))
def test_exact_integer_fp32(lib, t):
    A, B, ref = _int_case(300, 200, 320)
    C, _ = run_gemm(lib, A, B, lib.cfg(300, 200, 320, *t, dtype=0), 0)
    assert np.array_equal(C.astype(np.float64), ref)


@pytest.mark.parametrize("t", valid_space(2), ids=space_ids(2))
def test_exact_integer_fp8(lib, t):
    A, B, ref = _int_case(300, 200, 320)
    C, _ = run_gemm(lib, A, B, lib.cfg(300, 200, 320, *t, dtype=2), 2)
    # codes and the FP32 accumulation are exact; the rescale by 1/(s_A s_B)
    # rounds once
    assert np.all(np.abs(C - ref) <= 2.0 ** -23 * np.abs(ref))


@pytest.mark.parametrize("shape", [(1, 1, 16), (17, 33, 64), (129, 260, 4096), (1000, 8, 48), (64, 1024, 1040)])
@pytest.mark.parametrize("t", [(128, 128, 64, 4, 1), (128, 256, 64, 4, 2), (256, 128, 128, 2, 1), (64, 64, 64, 2, 2)])
def test_exact_integer_ragged_shapes(lib, shape, t):
    M, N, K = shape
    A, B, ref = _int_case(M, N, K)
    C, _ = run_gemm(lib, A, B, lib.cfg(M, N, K, *t, dtype=1), 1)
    assert np.array_equal(C.astype(np.float64), ref)


# ------------------------------------------- TMEM strategy B (A operand in TMEM)
@pytest.mark.parametrize("dt,t", B_SPACE, ids=B_IDS)
def test_exact_integer_tmem_strategy_b(lib, dt, t):
    A, B, ref = _int_case(300, 200, 320)
    C, _ = run_gemm(lib, A, B, lib.cfg(300, 200, 320, *t, dtype=dt, tmem_a=1), dt)
    if dt == 2:
        assert np.all(np.abs(C - ref) <= 2.0 ** -23 * np.abs(ref))
    else:
        assert np.array_equal(C.astype(np.float64), ref)


@pytest.mark.parametrize("shape", [(1, 1, 16), (17, 33, 64), (129, 260, 4096), (1000, 8, 48), (300, 1024, 1040)])
@pytest.mark.parametrize("dt,t", [(1, (128, 128, 64, 4, 1)), (1, (256, 128, 64, 4, 1)), (2, (128, 256, 128, 4, 1)),
                                  (0, (128, 128, 32, 3, 1))])
def test_exact_integer_tmem_strategy_b_ragged(lib, shape, dt, t):
    M, N, K = shape
    if (K * (4 if dt == 0 else (2 if dt == 1 else 1))) % 16:
        pytest.skip("K rows must be 16-byte multiples for TMA")
    A, B, ref = _int_case(M, N, K)
    C, _ = run_gemm(lib, A, B, lib.cfg(M, N, K, *t, dtype=dt, tmem_a=1), dt)
    if dt == 2:
        assert np.all(np.abs(C - ref) <= 2.0 ** -23 * np.abs(ref))
    else:
        assert np.array_equal(C.astype(np.float64), ref)


@pytest.mark.parametrize("dt,tol,t", [(1, 2e-2, (128, 256, 64, 4, 1)), (2, 6e-2, (256, 128, 128, 4, 1)),
                                      (0, 1e-5, (128, 128, 32, 2, 1))])
def test_tmem_strategy_b_accuracy(lib, dt, tol, t):
    M = N = K = 1024 if dt else 512
    A, B = S.gemm_operands(M, N, K, seed=2 if dt else 0, dist="normal" if dt else "uniform")
    C, _ = run_gemm(lib, A, B, lib.cfg(M, N, K, *t, dtype=dt, tmem_a=1), dt)
    ref = O.gemm_f64(A, B)
    if dt == 0:
        err = np.max(np.abs(C - ref)) / np.max(np.abs(ref))
    else:
        err = np.linalg.norm(C - ref) / np.linalg.norm(ref)
    assert err <= tol, err


# ---------------------------------------------------------- real-valued accuracy
def test_fp32_512_normwise(lib):
    # 512^3, uniform[-1,1) seed 0, BM=BN=128, BK=32, 2 stages, cta_group 1
    A, B = S.gemm_operands(512, 512, 512, seed=0)
    C, _ = run_gemm(lib, A, B, lib.cfg(512, 512, 512, 128, 128, 32, 2, 1, dtype=0), 0)
    ref = O.gemm_f64(A, B)
    err = np.max(np.abs(C - ref)) / np.max(np.abs(ref))
    assert err <= 1e-5, err


@pytest.mark.parametrize("dt,tol", [(1, 2e-2), (2, 6e-2)])
@pytest.mark.parametrize("t", [(128, 256, 64, 4, 1), (128, 256, 64, 4, 2), (256, 128, 128, 2, 2)])
def test_lowp_frobenius(lib, dt, tol, t):
    M = N = K = 1024
    A, B = S.gemm_operands(M, N, K, seed=2, dist="normal")
    C, _ = run_gemm(lib, A, B, lib.cfg(M, N, K, *t, dtype=dt), dt)
    ref = O.gemm_f64(A, B)
    err = np.linalg.norm(C - ref) / np.linalg.norm(ref)
    assert err <= tol, err


@functools.lru_cache(maxsize=2)
def normal_operands(n):
    # generated once per size (a 16384^3 pair takes about a minute on the host)
    return S.gemm_operands(n, n, n, seed=2, dist="normal")


@pytest.mark.parametrize("dt", [1, 2])
def test_large_sampled_rows(lib, dt):
    # full 8192^3 launch in the configuration the model picks; 128 sampled rows
    M = N = K = 8192
    A, B = normal_operands(M)
    th = O.prior_theta(lib.sm_count())
    pick, _ = O.autotune(np.array([[M, N, K]], np.int32), dt, th, lib.sm_count())
    C, _ = run_gemm(lib, A, B, lib.cfg(M, N, K, *pick[0], dtype=dt), dt)
    rows = S.sampled_rows(9, M, 128)
    ref = O.gemm_f64(A[rows], B)
    err = np.linalg.norm(C[rows] - ref) / np.linalg.norm(ref)
    assert err <= (2e-2 if dt == 1 else 6e-2), err


# The launch configurations the bench and the sweep's exhaustive search time
# at full size (8192^3 and 16384^3), checked on seeded sampled rows.
FULL_SIZE = [(1, 8192, (256, 256, 64, 4, 2)), (2, 8192, (256, 256, 128, 3, 1)),
             (1, 16384, (256, 256, 64, 3, 2)), (2, 16384, (256, 256, 128, 4, 2))]


@pytest.mark.parametrize("dt,n,t", FULL_SIZE, ids=["%s-%d" % (DT_NAMES[d], n) for d, n, _ in FULL_SIZE])
def test_full_size_sampled_rows(lib, dt, n, t):
    A, B = normal_operands(n)
    C, _ = run_gemm(lib, A, B, lib.cfg(n, n, n, *t, dtype=dt), dt)
    rows = S.sampled_rows(10, n, 128)
    ref = O.gemm_f64(A[rows], B)
    err = np.linalg.norm(C[rows] - ref) / np.linalg.norm(ref)
    assert err <= (2e-2 if dt == 1 else 6e-2), err
    assert np.isfinite(C).all()


def test_gemm_host_full_size_sampled_rows(lib):
    # the end-to-end call of the bench: host FP32 in and out, 8 row chunks
    n, t = 8192, (256, 256, 64, 4, 2)
    A, B = normal_operands(n)
    Ah = torch.from_numpy(A).pin_memory()
    Bh = torch.from_numpy(B).pin_memory()
    Ch = torch.full((n, n), float("nan"), dtype=torch.float32).pin_memory()
    c = lib.cfg(n, n, n, *t, dtype=1)
    ws = torch.empty(lib.pm_gemm_host_workspace(c, 8), dtype=torch.uint8, device="cuda")
    lib.pm_gemm_host(c, Ah, Bh, Ch, ws, 8)
    torch.cuda.synchronize()
    C = Ch.numpy()
    assert np.isfinite(C).all()
    rows = S.sampled_rows(11, n, 128)
    ref = O.gemm_f64(A[rows], B)
    assert np.linalg.norm(C[rows] - ref) / np.linalg.norm(ref) <= 2e-2


def test_gemm_autotune_picks_fastest_of_model_shortlist(lib):
    M = N = K = 2048
    A, B = S.gemm_operands(M, N, K, seed=2, dist="normal")
    ops = lib.GemmOperands(1, M, N, K)
    ops.prepare(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    C = torch.empty(M, N, dtype=torch.float32, device="cuda")
    th = O.prior_theta(lib.sm_count()).astype(np.float32).astype(np.float64)
    pick, timing = lib.pm_gemm_autotune(lib.cfg(M, N, K, dtype=1), 4, th, lib.sm_count(), ops.A_op, ops.B_op, C,
                                        ops.scales, warmup=2, reps=5)
    MNK = torch.tensor([M, N, K], dtype=torch.int32, device="cuda")
    picks = torch.empty(4 * 24, dtype=torch.uint8, device="cuda")
    t = torch.empty(4, dtype=torch.float32, device="cuda")
    lib.pm_autotune_topk(MNK, 1, 1, th, lib.sm_count(), 4, picks, t)
    short = [tuple(int(r[f]) for f in ("BM", "BN", "BK", "stages", "cta_group"))
             for r in picks.cpu().numpy().view(lib.CFG_DTYPE)]
    assert (pick.BM, pick.BN, pick.BK, pick.stages, pick.cta_group) in short
    assert timing["median_s"] > 0
    # the picked configuration computes the product correctly
    C2, _ = run_gemm(lib, A, B, pick, 1)
    ref = O.gemm_f64(A[:64], B)
    assert np.linalg.norm(C2[:64] - ref) / np.linalg.norm(ref) <= 2e-2


@pytest.mark.parametrize("dt,chunks,t", [(1, 3, (128, 256, 64, 4, 2)), (1, 1, (256, 256, 64, 4, 2)),
                                         (0, 4, (128, 128, 32, 3, 1)), (2, 4, (128, 256, 128, 3, 1)),
                                         (1, 7, (64, 128, 64, 4, 1))])
def test_gemm_host_pipeline_exact(lib, dt, chunks, t):
    # host FP32 in, host FP32 out, copies overlapped with compute in row chunks
    M, N, K = 1000, 768, 512
    A, B, ref = _int_case(M, N, K)
    Ah = torch.from_numpy(A).pin_memory()
    Bh = torch.from_numpy(B).pin_memory()
    Ch = torch.full((M, N), float("nan"), dtype=torch.float32).pin_memory()
    c = lib.cfg(M, N, K, *t, dtype=dt)
    ws = torch.empty(lib.pm_gemm_host_workspace(c, chunks), dtype=torch.uint8, device="cuda")
    for _ in range(2):                      # the second call reuses the staging buffers
        Ch.fill_(float("nan"))
        lib.pm_gemm_host(c, Ah, Bh, Ch, ws, chunks)
        torch.cuda.synchronize()
        C = Ch.numpy().astype(np.float64)
        if dt == 2:
            assert np.all(np.abs(C - ref) <= 2.0 ** -23 * np.abs(ref))
        else:
            assert np.array_equal(C, ref)


@pytest.mark.parametrize("dt,t", [(1, (256, 256, 64, 3, 1)), (1, (256, 256, 64, 4, 2)), (2, (256, 256, 128, 3, 1)),
                                  (2, (256, 256, 128, 4, 2))])
def test_split_accumulator_release_many_tiles_per_cta(lib, dt, t):
    # 256 x 256 tiles fill TMEM with one accumulator, so its two row blocks are
    # released separately (no FP32 tile that large fits shared memory);
    # 8192 x 8192 outputs give every CTA several tiles
    M = N = 8192
    K = 256
    A, B = S.integer_matrix(31, M, K), S.integer_matrix(32, K, N)
    C, _ = run_gemm(lib, A, B, lib.cfg(M, N, K, *t, dtype=dt), dt)
    rows = S.sampled_rows(33, M, 96)
    ref = O.gemm_f64(A[rows], B)
    if dt == 2:
        assert np.all(np.abs(C[rows] - ref) <= 2.0 ** -23 * np.abs(ref))
    else:
        assert np.array_equal(C[rows].astype(np.float64), ref)
