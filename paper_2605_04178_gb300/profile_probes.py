"""Launch each HBM probe kernel a few times, for profilers (ncu) and quick timing.

    python -m paper_2605_04178_gb300.profile_probes --elems 67108864 --side 8192

STREAM copy and triad (a = b + 3 c) over --elems FP32 elements, the TMA 2D
tile copy of a --side x --side FP32 matrix in 64 x 64 tiles, and the
five-point stencil over the same matrix (values uniform[-1,1) drawn on the
device).  Each kernel gets --warmup untimed and --reps timed single launches
(CUDA events), in that order, through pm_probe_launch.  Prints the median time
and the bandwidth over the bytes each must move: 8 B per element for copy,
TMA copy and stencil, 12 B for triad.
"""
import argparse
import statistics


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--elems", type=int, default=2 ** 26)
    ap.add_argument("--side", type=int, default=8192)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args()

    import torch

    import paper_2605_04178_gb300 as pm
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1)
    n, side = args.elems, args.side
    a = torch.rand(n, device="cuda", generator=gen) * 2 - 1
    b = torch.rand(n, device="cuda", generator=gen) * 2 - 1
    c = torch.rand(n, device="cuda", generator=gen) * 2 - 1
    src = torch.rand(side, side, device="cuda", generator=gen) * 2 - 1
    dst = torch.empty_like(src)
    probes = (("copy", pm.probe_args(pm.PM_PROBE_COPY, n=n), (a, b, None), 8.0 * n),
              ("triad", pm.probe_args(pm.PM_PROBE_TRIAD, n=n, scalar=3.0), (a, b, c), 12.0 * n),
              ("tma2d 64x64", pm.probe_args(pm.PM_PROBE_TMA2D, rows=side, cols=side, tile_r=64, tile_c=64),
               (src, dst, None), 8.0 * side * side),
              ("stencil", pm.probe_args(pm.PM_PROBE_STENCIL, rows=side, cols=side), (src, dst, None),
               8.0 * side * side))
    for name, pa, bufs, nbytes in probes:
        for _ in range(args.warmup):
            pm.pm_probe_launch(pa, *bufs)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.reps)]
        for s, e in ev:
            s.record()
            pm.pm_probe_launch(pa, *bufs)
            e.record()
        torch.cuda.synchronize()
        if pm.pm_device_status(True) != pm.PM_OK:
            raise RuntimeError(pm.pm_last_error())
        ms = statistics.median(s.elapsed_time(e) for s, e in ev)
        print("%s: %.1f us, %.0f GB/s" % (name, ms * 1e3, nbytes / ms / 1e6))


if __name__ == "__main__":
    main()
