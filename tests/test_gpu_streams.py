"""GPU checks of the concurrent-stream interference probe (Sec. III-A.6):
every stream's kernel computes its own result exactly while the streams
overlap, and the makespan is reported."""
import numpy as np
import pytest

import oracle as O
import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_streams", [1, 2, 3, 8])
@pytest.mark.parametrize("n", [1000, 2 ** 20 + 5])
def test_copy_on_concurrent_streams_bit_exact(lib, n_streams, n):
    src = [torch.from_numpy(S.uniform_pm1(40 + i, n)).cuda() for i in range(n_streams)]
    dst = [torch.full_like(x, float("nan")) for x in src]
    r = lib.pm_streams_run(lib.probe_args(lib.PM_PROBE_COPY, n=n), src, dst, warmup=1, reps=3)
    assert r["median_s"] > 0 and r["bytes"] == 8.0 * n * n_streams
    for a, b in zip(src, dst):
        assert torch.equal(a.view(torch.int32), b.view(torch.int32))


def test_triad_on_concurrent_streams_bit_exact(lib):
    n, k = 4099, 4
    b = [S.normal(50 + i, n) for i in range(k)]
    c = [S.uniform_pm1(60 + i, n) for i in range(k)]
    a_d = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(k)]
    lib.pm_streams_run(lib.probe_args(lib.PM_PROBE_TRIAD, n=n, scalar=3.0), a_d,
                       [torch.from_numpy(x).cuda() for x in b], [torch.from_numpy(x).cuda() for x in c],
                       warmup=0, reps=2)
    for i in range(k):
        assert np.array_equal(a_d[i].cpu().numpy().view(np.uint32), O.triad_f32(b[i], c[i], 3.0).view(np.uint32))


@pytest.mark.parametrize("ctas", [8, 76])
def test_mma_on_concurrent_streams_exact(lib, ctas):
    n, k = 1 << 12, 4
    outs = [torch.zeros(ctas, dtype=torch.int32, device="cuda") for _ in range(k)]
    args = lib.probe_args(lib.PM_PROBE_MMA, n=n, tile_r=256, tile_c=128, rows=1, cols=1, start=ctas)
    r = lib.pm_streams_run(args, outs, warmup=1, reps=3)
    for o in outs:
        assert np.all(o.cpu().numpy().view(np.float32) == O.mma_probe_value(n, 1))
    assert r["bytes"] == k * ctas * n * 2.0 * 128 * 256 * 16
    assert lib.pm_device_status(True) == lib.PM_OK


def test_shutdown_releases_and_recreates(lib):
    # streams, host pipeline and descriptor caches are released and re-created on demand
    n = 4099
    src = [torch.from_numpy(S.uniform_pm1(70 + i, n)).cuda() for i in range(3)]
    for _ in range(2):
        dst = [torch.full_like(x, float("nan")) for x in src]
        lib.pm_streams_run(lib.probe_args(lib.PM_PROBE_COPY, n=n), src, dst, warmup=0, reps=1)
        for a, b in zip(src, dst):
            assert torch.equal(a, b)
        A, B = S.integer_matrix(71, 200, 64), S.integer_matrix(72, 64, 96)
        c = lib.cfg(200, 96, 64, 128, 128, 64, 2, 1, lib.PM_BF16)
        ws = torch.empty(lib.pm_gemm_host_workspace(c, 2), dtype=torch.uint8, device="cuda")
        Ch = torch.empty(200, 96, dtype=torch.float32).pin_memory()
        lib.pm_gemm_host(c, torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory(), Ch, ws, 2)
        torch.cuda.synchronize()
        assert np.array_equal(Ch.numpy().astype(np.float64), O.gemm_f64(A, B))
        lib.pm_shutdown()
