"""Run one grouped BF16 GEMM launch a few times, for profilers (ncu) and quick timing.

    python -m paper_2605_04178_gb300.profile_grouped --groups 64 --n 4096 --k 4096

The grouped workload: G problems with M_g log-uniform in [16, 4096] (seed 3),
N = K fixed, a distinct B per group, BF16 operands drawn on the device (seed
3).  The per-group tiles and the launch (BK, stages, cta_group) are the
model's pick (pm_grouped_autotune under the calibrated literal parameters);
then `--warmup` untimed and `--reps` timed launches (CUDA events).  Prints the
median time, TFLOP/s and the GB/s over the bytes the launch must move (every
A_g and B_g once, every C_g written once).
"""
import argparse
import json
import os
import statistics


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--groups", type=int, default=64)
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--k", type=int, default=4096)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args()

    import torch

    import paper_2605_04178_gb300 as pm
    import synthetic as S
    with open(os.path.join(os.path.dirname(os.path.abspath(pm.__file__)), "theta_gb300.json")) as f:
        theta = json.load(f)["theta"]
    G, N, K = args.groups, args.n, args.k
    Mg = S.grouped_m(G, 3)
    sum_m = int(Mg.sum())
    _, bm, bn, launch = pm.pm_grouped_autotune(Mg, N, K, pm.PM_BF16, theta, pm.sm_count())
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    A = torch.randn(sum_m, K, device="cuda", generator=gen).to(torch.bfloat16)
    B = torch.empty(G * N, K, dtype=torch.bfloat16, device="cuda")
    for q in range(G):
        B[q * N:(q + 1) * N] = torch.randn(N, K, device="cuda", generator=gen).to(torch.bfloat16)
    C = torch.empty(sum_m, N, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        pm.pm_grouped_gemm_run(Mg, N, K, bm, bn, *launch, A, B, C)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.reps)]
    for s, e in ev:
        s.record()
        pm.pm_grouped_gemm_run(Mg, N, K, bm, bn, *launch, A, B, C)
        e.record()
    torch.cuda.synchronize()
    if pm.pm_device_status(True) != pm.PM_OK:
        raise RuntimeError(pm.pm_last_error())
    ms = statistics.median(s.elapsed_time(e) for s, e in ev)
    flops = sum(2.0 * int(m) * N * K for m in Mg)
    nbytes = sum(2.0 * (int(m) * K + N * K) + 4.0 * int(m) * N for m in Mg)
    print("grouped G=%d sum_M=%d N=%d K=%d launch %s: %.3f ms, %.0f TFLOP/s, %.0f GB/s"
          % (G, sum_m, N, K, launch, ms, flops / ms / 1e9, nbytes / ms / 1e6))


if __name__ == "__main__":
    main()
