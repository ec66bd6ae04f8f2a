"""Run the batched model kernels a few times, for profilers (ncu) and quick timing.

    python -m paper_2605_04178_gb300.profile_model --configs 1000000 --reading 0

The batch is the model-calibration workload: GEMM configurations with shapes
log-uniform in [16, 16384] rounded to 16, tiles uniform over the 180-point
space and dtypes uniform (seed 4).  Each round launches, in this order, the
forward (`model_predict_kernel`), the adjoint (`model_grad_kernel` and its
FP64 finish kernel) and the autotuner (`autotune_kernel`, the first
configs/180 shapes over all 180 tiles); `--warmup` untimed rounds, then
`--reps` timed ones.  Prints the median time of each and the configurations
per second (CUDA events on the launching stream).
"""
import argparse
import json
import os
import statistics


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--configs", type=int, default=10 ** 6)
    ap.add_argument("--reading", type=int, default=1, help="0 literal, 1 measured (default); each with its own calibration")
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args()

    import numpy as np
    import torch

    import paper_2605_04178_gb300 as pm
    import synthetic as S
    here = os.path.dirname(os.path.abspath(pm.__file__))
    name = "theta_gb300.json" if args.reading == pm.PM_READING_MEASURED else "theta_gb300_literal.json"
    with open(os.path.join(here, name)) as f:
        theta = json.load(f)["theta"]
    n_sm = pm.sm_count()
    nc = args.configs
    cf = S.model_config_batch(nc, seed=4)
    cf["kind"] = np.zeros(nc, dtype=np.int32)
    dev = pm.cfg_tensor(cf)
    t_out = torch.empty(nc, dtype=torch.float32, device="cuda")
    tm = torch.full((nc,), 1e-3, dtype=torch.float32, device="cuda")
    ws = torch.empty(pm.pm_model_grad_workspace(nc) // 8, dtype=torch.float64, device="cuda")
    go = torch.empty(pm.N_GRAD_OUT, dtype=torch.float64, device="cuda")
    ns = max(1, nc // 180)
    MNK = torch.from_numpy(np.stack([cf["M"], cf["N"], cf["K"]], 1)[:ns].astype(np.int32).ravel()).cuda()
    picks = torch.empty(ns * 24, dtype=torch.uint8, device="cuda")
    tp = torch.empty(ns, dtype=torch.float32, device="cuda")
    steps = (("forward", lambda: pm.pm_model_predict(dev, nc, theta, n_sm, t_out), nc),
             ("adjoint", lambda: pm.pm_model_grad(dev, nc, theta, n_sm, tm, ws, go), nc),
             ("autotune", lambda: pm.pm_autotune_pick(MNK, ns, pm.PM_BF16, theta, n_sm, picks, tp), ns * 180))
    pm.pm_model_set_reading(args.reading)
    try:
        for _ in range(args.warmup):
            for _, fn, _ in steps:
                fn()
        times = {k: [] for k, _, _ in steps}
        for _ in range(args.reps):
            for k, fn, _ in steps:
                s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s.record()
                fn()
                e.record()
                times[k].append((s, e))
        torch.cuda.synchronize()
    finally:
        pm.pm_model_set_reading(pm.PM_READING_MEASURED)
    for k, _, units in steps:
        ms = statistics.median(s.elapsed_time(e) for s, e in times[k])
        print("%s: %.2f us, %.1f G configurations/s" % (k, ms * 1e3, units / ms / 1e6))


if __name__ == "__main__":
    main()
