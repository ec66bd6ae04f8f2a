"""GPU parity of the grouped persistent GEMM (one launch over G problems with
uneven M, per-group tiles, captured in a CUDA graph) against the FP64 oracle."""
import itertools

import numpy as np
import pytest

import oracle as O
import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def stacked_operands(lib, A_list, B_list, N, K):
    """BF16 operands: A rows stacked, B_g transposed to [N, K] and stacked."""
    G = len(A_list)
    sum_m = sum(a.shape[0] for a in A_list)
    A_op = torch.empty(sum_m * K * 2, dtype=torch.uint8, device="cuda")
    B_op = torch.empty(G * N * K * 2, dtype=torch.uint8, device="cuda")
    row0 = 0
    for q, (A, B) in enumerate(zip(A_list, B_list)):
        M = A.shape[0]
        lib.pm_gemm_prepare(lib.PM_BF16, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), M, N, K,
                            A_op.data_ptr() + row0 * K * 2, B_op.data_ptr() + q * N * K * 2, None)
        row0 += M
    return A_op, B_op, sum_m


def run_grouped(lib, A_list, B_list, N, K, bm, bn, launch, graph=False):
    A_op, B_op, sum_m = stacked_operands(lib, A_list, B_list, N, K)
    C = torch.full((sum_m, N), float("nan"), dtype=torch.float32, device="cuda")
    Ms = [a.shape[0] for a in A_list]
    lib.pm_grouped_gemm_run(Ms, N, K, bm, bn, *launch, A_op, B_op, C)
    torch.cuda.synchronize()
    assert lib.pm_device_status(True) == lib.PM_OK
    if graph:
        C2 = torch.full_like(C, float("nan"))
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            lib.pm_grouped_gemm_run(Ms, N, K, bm, bn, *launch, A_op, B_op, C2, stream=s)
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        assert torch.equal(C, C2)
    return C.cpu().numpy()


def int_groups(Ms, N, K, seed=21):
    A_list = [S.integer_matrix(seed + q, m, K) for q, m in enumerate(Ms)]
    B_list = [S.integer_matrix(seed + 1000 + q, K, N) for q in range(len(Ms))]
    return A_list, B_list


@pytest.mark.parametrize("launch", list(itertools.product((64, 128), (2, 4), (1, 2))))
def test_grouped_exact_integer_mixed_tiles(lib, launch):
    Ms = [1, 16, 33, 100, 129, 256, 300, 77]
    N, K = 192, 320
    A_list, B_list = int_groups(Ms, N, K)
    sizes = (64, 128, 256)
    bm = [sizes[q % 3] for q in range(len(Ms))]
    bn = [sizes[(q // 3 + q) % 3] for q in range(len(Ms))]
    # drop (BM, BN) pairs the launch's ring cannot hold
    for q in range(len(Ms)):
        while not O.cfg_valid(bm[q], bn[q], launch[0], launch[1], launch[2], 1):
            bm[q] = max(64, bm[q] // 2) if bm[q] > 64 else bm[q]
            bn[q] = max(64, bn[q] // 2)
    C = run_grouped(lib, A_list, B_list, N, K, bm, bn, launch)
    row0 = 0
    for A, B in zip(A_list, B_list):
        m = A.shape[0]
        assert np.array_equal(C[row0:row0 + m].astype(np.float64), O.gemm_f64(A, B))
        row0 += m


def test_grouped_64_groups_reduced_with_graph(lib):
    # 64 groups, M log-uniform in [16, 4096] (seed 3), N = K = 1024, tiles
    # and launch from the GPU grouped autotuner; captured in a CUDA graph.
    Mg = S.grouped_m(64, 3)
    N = K = 1024
    th = O.prior_theta(lib.sm_count()).astype(np.float32).astype(np.float64)
    t, bm, bn, launch = lib.pm_grouped_autotune(Mg, N, K, 1, th, lib.sm_count())
    A_list = [S.matrix(3, int(m), K, "uniform", offset=q * 4096 * K) for q, m in enumerate(Mg)]
    B_list = [S.matrix(4, K, N, "uniform", offset=q * K * N) for q in range(64)]
    C = run_grouped(lib, A_list, B_list, N, K, bm, bn, launch, graph=True)
    row0 = 0
    for q, (A, B) in enumerate(zip(A_list, B_list)):
        m = A.shape[0]
        rows = S.sampled_rows(q, m, 8)
        ref = O.gemm_f64(A[rows], B)
        err = np.linalg.norm(C[row0 + rows] - ref) / np.linalg.norm(ref)
        assert err <= 2e-2, (q, err)
        row0 += m


def test_grouped_measured_autotune_picks_from_model_shortlist(lib):
    # the measured grouped autotuner times the model's k best launches; its
    # pick is one of them and computes the product exactly
    Ms = [int(m) for m in S.grouped_m(16, 5, lo=16, hi=1024)]
    N, K = 512, 1024
    A_list, B_list = int_groups(Ms, N, K, seed=41)
    A_op, B_op, sum_m = stacked_operands(lib, A_list, B_list, N, K)
    C = torch.full((sum_m, N), float("nan"), dtype=torch.float32, device="cuda")
    th = O.prior_theta(lib.sm_count())
    t_pred, bm, bn, launch, timing = lib.pm_grouped_gemm_autotune(Ms, N, K, th, lib.sm_count(), 4, A_op, B_op, C,
                                                                  warmup=1, reps=3)
    assert timing["median_s"] > 0 and t_pred > 0
    t_best, _, _, _ = lib.pm_grouped_autotune(Ms, N, K, lib.PM_BF16, th, lib.sm_count())
    assert t_pred >= t_best * (1 - 1e-6)                 # a shortlist member: never predicted better than the best
    C = run_grouped(lib, A_list, B_list, N, K, bm, bn, launch)
    row0 = 0
    for A, B in zip(A_list, B_list):
        assert np.array_equal(C[row0:row0 + A.shape[0]].astype(np.float64), O.gemm_f64(A, B))
        row0 += A.shape[0]


@pytest.mark.parametrize("launch", [(64, 3, 1), (64, 3, 2)])
def test_grouped_exact_integer_split_release(lib, launch):
    # every group in 256 x 256 tiles: one TMEM accumulator released by row block
    Ms = [300, 600, 900, 257, 1024, 2048, 513, 4096]
    N, K = 1024, 192
    A_list, B_list = int_groups(Ms, N, K, seed=61)
    G = len(Ms)
    C = run_grouped(lib, A_list, B_list, N, K, [256] * G, [256] * G, launch, graph=True)
    row0 = 0
    for A, B in zip(A_list, B_list):
        assert np.array_equal(C[row0:row0 + A.shape[0]].astype(np.float64), O.gemm_f64(A, B))
        row0 += A.shape[0]


def test_grouped_schedule_reorders_groups_exactly(lib):
    # tiles of four sizes in the caller's order small, large, medium, ...:
    # the launch lists them largest first and deals them in alternating
    # round-robin order; every group's product stays exact, on one SM
    # (cta_group 1) and on CTA pairs, and after graph replay
    Ms = [40, 700, 130, 2000, 64, 999, 257, 5]
    N, K = 640, 256
    A_list, B_list = int_groups(Ms, N, K, seed=81)
    bm = [64, 256, 128, 256, 64, 128, 128, 64]
    bn = [64, 256, 128, 128, 256, 256, 64, 128]
    for launch in ((64, 3, 1), (64, 3, 2)):
        b_m = [b if O.cfg_valid(b, n, *launch, 1) else 128 for b, n in zip(bm, bn)]
        C = run_grouped(lib, A_list, B_list, N, K, b_m, bn, launch, graph=True)
        row0 = 0
        for A, B in zip(A_list, B_list):
            assert np.array_equal(C[row0:row0 + A.shape[0]].astype(np.float64), O.gemm_f64(A, B))
            row0 += A.shape[0]
