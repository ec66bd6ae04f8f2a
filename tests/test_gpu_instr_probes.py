"""GPU checks of the Blackwell instruction probes (tcgen05.mma throughput,
mbarrier round trips, TMEM load/store bandwidth) and the host-link copy
probes, against closed forms in the oracle."""
import numpy as np
import pytest

import oracle as O
import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cg,M,N", [(1, 128, 256), (1, 128, 128), (1, 64, 256), (2, 256, 256), (2, 256, 128),
                                    (2, 128, 256)])
@pytest.mark.parametrize("dt", [0, 1, 2])
def test_mma_probe_accumulates_exactly(lib, cg, M, N, dt):
    n = 1000
    grid = 8
    out = torch.zeros(grid, dtype=torch.int32, device="cuda")
    r = lib.pm_probe_run(lib.probe_args(lib.PM_PROBE_MMA, n=n, tile_r=N, tile_c=M, rows=cg, cols=dt, start=grid),
                         out, warmup=1, reps=3)
    got = out.cpu().numpy().view(np.float32)
    assert np.all(got == O.mma_probe_value(n, dt)), got
    kin = {0: 8, 1: 16, 2: 32}[dt]
    assert r["bytes"] == (grid // cg) * n * 2.0 * M * N * kin


def test_mma_probe_full_chip_rate(lib):
    # all SMs, 128x256x16 BF16 per SM: reports FLOP/s; must exceed half the datasheet peak
    out = torch.zeros(lib.sm_count(), dtype=torch.int32, device="cuda")
    r = lib.pm_probe_run(lib.probe_args(lib.PM_PROBE_MMA, n=1 << 16, tile_r=256, tile_c=256, rows=2, cols=1),
                         out, warmup=2, reps=5)
    assert np.all(out.cpu().numpy().view(np.float32) == O.mma_probe_value(1 << 16, 1))
    assert r["bytes"] / r["median_s"] > 1.1e15


@pytest.mark.parametrize("n", [1, 2, 1000, 100000])
def test_mbar_probe_round_trips(lib, n):
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    r = lib.pm_probe_run(lib.probe_args(lib.PM_PROBE_MBAR, n=n), out, warmup=1, reps=3)
    assert r["final_index"] == n


@pytest.mark.parametrize("kind,store", [(9, False), (10, True)])
@pytest.mark.parametrize("iters", [1, 3, 257])
def test_tmem_probe_checksums(lib, kind, store, iters):
    sms = lib.sm_count()
    out = torch.zeros(sms * 256, dtype=torch.int32, device="cuda")
    lib.pm_probe_run(lib.probe_args(kind, n=iters), out, warmup=0, reps=1)
    got = out.cpu().numpy().view(np.uint32).reshape(sms, 256)
    assert np.array_equal(got, np.broadcast_to(O.tmem_probe_sums(iters, store), (sms, 256)))


@pytest.mark.parametrize("nbytes", [16, 1000, 1 << 26])
def test_host_link_probes_copy_bytes(lib, nbytes):
    src = torch.from_numpy(S.uniform_pm1(3, (nbytes + 3) // 4)).view(torch.uint8)[:nbytes].contiguous().pin_memory()
    dev = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    back = torch.zeros(nbytes, dtype=torch.uint8).pin_memory()
    r = lib.pm_probe_run(lib.probe_args(lib.PM_PROBE_H2D, n=nbytes), src, dev, warmup=1, reps=3)
    lib.pm_probe_run(lib.probe_args(lib.PM_PROBE_D2H, n=nbytes), dev, back, warmup=1, reps=3)
    assert torch.equal(src, back) and r["bytes"] == nbytes
