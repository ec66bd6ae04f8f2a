"""Run one GEMM configuration a few times, for profilers (ncu) and quick timing.

    python -m paper_2605_04178_gb300.profile_gemm --dtype fp8 --size 8192 --tile 256,256,128,3,1

Operands are seeded normal(0,1) FP32 drawn on the device and prepared into the
operand format once; then `--warmup` untimed and `--reps` timed launches of
the GEMM.  Prints the median time and TFLOP/s (CUDA events, one per launch).
"""
import argparse
import statistics


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--dtype", choices=("fp32", "bf16", "fp8"), default="bf16")
    ap.add_argument("--size", type=int, default=8192, help="M = N = K")
    ap.add_argument("--tile", default="256,256,64,4,2", help="BM,BN,BK,stages,cta_group")
    ap.add_argument("--tmem-a", type=int, default=0, help="1: TMEM strategy B")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args()

    import torch

    import paper_2605_04178_gb300 as pm
    dt = {"fp32": pm.PM_FP32, "bf16": pm.PM_BF16, "fp8": pm.PM_FP8E4M3}[args.dtype]
    n = args.size
    gen = torch.Generator(device="cuda")
    gen.manual_seed(2)
    A = torch.randn(n, n, device="cuda", generator=gen)
    B = torch.randn(n, n, device="cuda", generator=gen)
    ops = pm.GemmOperands(dt, n, n, n)
    ops.prepare(A, B)
    del A, B
    C = torch.empty(n, n, device="cuda")
    cfg = pm.cfg(n, n, n, *(int(v) for v in args.tile.split(",")), dtype=dt, tmem_a=args.tmem_a)
    for _ in range(args.warmup):
        ops.run(cfg, C)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.reps)]
    for s, e in ev:
        s.record()
        ops.run(cfg, C)
        e.record()
    torch.cuda.synchronize()
    if pm.pm_device_status(True) != pm.PM_OK:
        raise RuntimeError(pm.pm_last_error())
    ms = statistics.median(s.elapsed_time(e) for s, e in ev)
    print("%s %d^3 tile %s: %.3f ms, %.0f TFLOP/s" % (args.dtype, n, args.tile, ms, 2.0 * n ** 3 / ms / 1e9))


if __name__ == "__main__":
    main()
