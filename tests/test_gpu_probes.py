"""GPU parity of the calibration probes against the CPU oracle (bit-exact)."""
import numpy as np
import pytest

import oracle as O
import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 3, 4, 1000, 2 ** 20 + 3, 2 ** 24, 2 ** 24 + 3, 2 ** 24 + 8195, 5 * 2 ** 23 + 1])
def test_copy_bit_exact(lib, n):
    a = torch.from_numpy(S.uniform_pm1(1, n)).cuda()
    b = torch.full_like(a, float("nan"))
    r = lib.pm_probe_run(lib.probe_args(lib.PM_PROBE_COPY, n=n), a, b, warmup=1, reps=3)
    assert r["bytes"] == 8 * n and r["median_s"] > 0
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))


@pytest.mark.parametrize("n", [1, 5, 4099, 2 ** 20 + 1])
def test_triad_bit_exact(lib, n):
    b = S.normal(1, n) * np.float32(100.0)
    c = S.uniform_pm1(2, n)
    s = 3.0
    a_dev = torch.empty(n, dtype=torch.float32, device="cuda")
    lib.pm_probe_run(lib.probe_args(lib.PM_PROBE_TRIAD, n=n, scalar=s), a_dev, torch.from_numpy(b).cuda(),
                     torch.from_numpy(c).cuda(), warmup=0, reps=2)
    ref = O.triad_f32(b, c, s)
    assert np.array_equal(a_dev.cpu().numpy().view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("nodes,hops,start", [(1, 10, 0), (256, 1000, 3), (4096, 4096, 7), (1 << 20, 100000, 12345)])
def test_pchase_final_index(lib, nodes, hops, start):
    buf = S.pchase_buffer(nodes, seed=1)
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    r = lib.pm_probe_run(lib.probe_args(lib.PM_PROBE_PCHASE, n=nodes, hops=hops, start=start),
                         torch.from_numpy(buf.view(np.int32)).cuda(), out, warmup=1, reps=2)
    # three launches, each continuing the walk of the previous one
    assert r["final_index"] == O.pchase(buf, 16, start, 3 * hops)
    lib.pm_probe_launch(lib.probe_args(lib.PM_PROBE_PCHASE, n=nodes, hops=hops, start=start),
                        torch.from_numpy(buf.view(np.int32)).cuda(), out)
    assert int(out.cpu().numpy()[0]) == O.pchase(buf, 16, start, hops)


@pytest.mark.parametrize("tile", [(64, 64), (128, 64), (128, 128), (256, 64), (256, 128), (8, 4), (200, 36)])
@pytest.mark.parametrize("shape", [(1000, 1004), (64, 64), (3, 20)])
def test_tma2d_copy_bit_exact(lib, tile, shape):
    rows, cols = shape
    src = torch.from_numpy(S.uniform_pm1(7, rows * cols).reshape(rows, cols)).cuda()
    dst = torch.full_like(src, float("nan"))
    lib.pm_probe_run(lib.probe_args(lib.PM_PROBE_TMA2D, rows=rows, cols=cols, tile_r=tile[0], tile_c=tile[1]),
                     src, dst, warmup=0, reps=2)
    assert torch.equal(src.view(torch.int32), dst.view(torch.int32))


def test_tma2d_full_size(lib):
    # 1 GiB FP32 matrix (16384 x 16384), the probe's full configuration
    src = torch.randn(16384, 16384, device="cuda")
    dst = torch.zeros_like(src)
    r = lib.pm_probe_run(lib.probe_args(lib.PM_PROBE_TMA2D, rows=16384, cols=16384, tile_r=128, tile_c=64),
                         src, dst, warmup=1, reps=3)
    assert torch.equal(src, dst)
    assert r["bytes"] == 2 ** 31


def test_watchdog_times_out_and_context_survives(lib):
    st = lib.pm_watchdog_selftest(100000)          # 0.1 s limit on a wait nothing completes
    assert st == lib.PM_ETIMEOUT
    assert lib.pm_device_status(True) == lib.PM_OK  # the self-test cleared its record
    x = torch.arange(1000, device="cuda", dtype=torch.float32)
    y = torch.empty_like(x)
    lib.pm_probe_run(lib.probe_args(lib.PM_PROBE_COPY, n=1000), x, y, warmup=0, reps=1)
    assert torch.equal(x, y)


@pytest.mark.parametrize("n", [1, 5, 4099, 2 ** 22 + 3])
def test_host_link_sm_copies_bit_exact(lib, n):
    # SM-driven copies through the device mapping of page-locked host memory
    h = torch.from_numpy(S.uniform_pm1(9, n)).pin_memory()
    d = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
    r = lib.pm_probe_run(lib.probe_args(lib.PM_PROBE_HOST_READ, n=n), h, d, warmup=1, reps=2)
    assert r["bytes"] == 4 * n
    assert torch.equal(d.cpu().view(torch.int32), h.view(torch.int32))
    back = torch.full((n,), float("nan"), dtype=torch.float32).pin_memory()
    lib.pm_probe_run(lib.probe_args(lib.PM_PROBE_HOST_WRITE, n=n), d, back, warmup=0, reps=1)
    torch.cuda.synchronize()
    assert torch.equal(back.view(torch.int32), h.view(torch.int32))


def test_host_link_probe_refuses_unpinned_memory(lib):
    d = torch.empty(1024, dtype=torch.float32, device="cuda")
    with pytest.raises(lib.PMError) as e:
        lib.pm_probe_run(lib.probe_args(lib.PM_PROBE_HOST_READ, n=1024), d, d, warmup=0, reps=1)
    assert e.value.status == lib.PM_EINVAL


@pytest.mark.parametrize("shape", [(1, 1), (2, 7), (3, 3), (37, 1000), (1000, 37), (1024, 1024), (4099, 2053),
                                   (5, 8), (9, 132), (17, 4100), (3, 256), (1, 64)])
def test_stencil_bit_exact(lib, shape):
    # widths that are multiples of 4 take the four-points-per-thread kernel
    rows, cols = shape
    x = S.uniform_pm1(21, rows * cols).reshape(rows, cols)
    src = torch.from_numpy(x).cuda()
    dst = torch.full_like(src, float("nan"))
    r = lib.pm_probe_run(lib.probe_args(lib.PM_PROBE_STENCIL, rows=rows, cols=cols), src, dst, warmup=1, reps=2)
    assert r["bytes"] == 8 * rows * cols
    assert np.array_equal(dst.cpu().numpy().view(np.uint32), O.stencil5_f32(x).view(np.uint32))


def test_timing_harness_records_clocks(lib):
    # Sec. V-B protocol: every measurement carries the clock and throttle
    # state; the harness reads the SM clock through NVML (read only) right
    # before its first timed launch and after its last one
    c = lib.pm_clock_sample()
    assert c is not None, lib.pm_last_error()
    assert 0 < c["sm_mhz"] <= c["sm_max_mhz"] and c["mem_mhz"] > 0 and c["power_w"] > 0
    n = 2 ** 26
    a = torch.empty(n, dtype=torch.float32, device="cuda").uniform_(-1, 1)
    b = torch.empty_like(a)
    r = lib.pm_probe_run(lib.probe_args(lib.PM_PROBE_COPY, n=n), a, b, warmup=2, reps=10)
    assert 0 < r["sm_mhz_begin"] <= r["sm_max_mhz"] and 0 < r["sm_mhz_end"] <= r["sm_max_mhz"]
    assert all(name in lib.CLOCK_REASONS.values() for name in r["clock_reasons"])
