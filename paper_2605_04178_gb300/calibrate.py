"""Calibration of the stage-centric model against device-timed measurements
(arxiv 2605.04178, Sec. III-D: parameters from microbenchmarks, fitted to
measured kernel times with a train/holdout split; Sec. V-B protocol: warm-ups,
timed runs, median).

Pieces
  * measure_sweep(): the calibration table -- the FP32 GEMM at 512^3 over
    the FP32 tile space, the memory probes (copy/triad 2^20..2^30, TMA 2D tiles
    on a 1 GiB matrix, pointer chase 16 KB..1 GB) and the BF16/FP8 sweep (every valid BF16 and
    FP8 tile configuration at M = N = K in {1024..16384}), each timed on the
    device by the library's own harness (pm_gemm_bench / pm_probe_run).
  * measure_tmem_b(): the same GEMM classes under TMEM strategy B (A operand
    copied into tensor memory, Sec. III-A.1) over the strategy-B tile space.
  * measure_streams() / fit_tau_c(): the concurrent-stream term of Sec.
    III-A.6, T(N_c) = T(1) + (N_c - 1) tau_c, per workload class.
  * measure_segments() / fit_segments(): the generic roofline path (Sec.
    III-E): memory-bound, compute-bound, balanced and stencil segments,
    multi-kernel segments and segments with host transfers and syncs; one
    scale per class and an efficiency per precision, fitted with the model
    evaluated by pm_segment_predict.
  * StageModelLoss: torch.autograd.Function whose forward is the batched model
    on the GPU and whose backward is the hand-written adjoint kernel
    (pm_model_grad): mean squared log error and its gradient in theta.
  * fit(): L-BFGS over phi = ln(theta) with a weak pull to the prior.
  * report(): MAE per configuration family (train, holdout, all) and the
    model-picked tile against the exhaustively measured best.
The fitted parameters are written as a hardware parameter file (JSON), the
form the paper keeps per platform.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np
import torch

import paper_2605_04178_gb300 as pm
import synthetic as S

HERE = os.path.dirname(os.path.abspath(__file__))
THETA_PATH = os.path.join(HERE, "theta_gb300.json")                  # default (measured) reading
THETA_PATH_LITERAL = os.path.join(HERE, "theta_gb300_literal.json")  # the literal equations
REPORT_PATH = os.path.join(HERE, "data", "calib_report_gb300.json")
REPORT_PATH_LITERAL = os.path.join(HERE, "data", "calib_report_gb300_literal.json")
# Weight of the pull towards the prior in the fit.  The printed priors are
# B200 figures or guesses (D12), so the pull only regularises directions the
# table does not determine; at 1e-4 it held the fitted GEMM parameters near
# the priors (holdout MAE 4.7 -> 4.1 % for BF16 when lowered to 1e-6).
FIT_REG = 1e-6


def theta_path(reading: int) -> str:
    return THETA_PATH if reading == pm.PM_READING_MEASURED else THETA_PATH_LITERAL


def report_path(reading: int) -> str:
    return REPORT_PATH if reading == pm.PM_READING_MEASURED else REPORT_PATH_LITERAL
SWEEP_PATH = os.path.join(HERE, "data", "sweep_gb300.json")
FIELDS = ("M", "N", "K", "BM", "BN", "BK", "stages", "cta_group", "dtype", "kind", "tmem_a")


def prior_theta(n_sm: int, f_hz: float = 1.9e9, reading: int = pm.PM_READING_MEASURED) -> np.ndarray:
    """Parameter priors from the paper's printed values (Table "parameters",
    Sec. II-A sustained figures, Table "arch-params"); cycles at f_hz.  c_alpha
    puts alpha(2) at 0.85 under either overlap law of the reading; rho_L2
    starts at the peak-to-sustained HBM ratio and B_drain, like B_TMA, at the
    per-SM share of the sustained HBM rate (neither is printed)."""
    th = np.zeros(pm.N_PARAMS)
    th[0] = 5e-6
    th[1] = 6.8e12
    th[2] = 8.0e12
    th[3] = 64.0 * 2 ** 20
    th[4] = 420.0 / f_hz
    th[5] = th[1] / n_sm
    th[7] = 8192.0 * f_hz
    th[6] = th[7] / 2.0
    th[8] = 2.0 * th[7]
    th[9] = 12.0 / f_hz
    th[10] = 16e12
    th[11] = 8e12
    th[12] = 45.0 / f_hz
    th[13] = 100e-9
    th[14] = 1.0
    th[15] = 0.3 if reading == pm.PM_READING_LITERAL else 0.15
    th[16] = th[2] / th[1]
    th[17] = th[1] / n_sm
    return th


def clock_of(r: dict) -> dict:
    """The harness's clock record of one measurement (SM MHz before the first
    and after the last timed launch, the clock event reasons seen)."""
    return dict(sm_mhz_begin=r.get("sm_mhz_begin", 0), sm_mhz_end=r.get("sm_mhz_end", 0),
                clock_reasons=r.get("clock_reasons", []))


def family_of(r: dict) -> str:
    if "launch" in r and "G" in r:
        return "grouped"
    if r["kind"] == pm.PM_KIND_COPY or r["kind"] == pm.PM_KIND_TRIAD:
        return "stream"
    if r["kind"] == pm.PM_KIND_TMA2D:
        return "tma"
    fam = {0: "fp32", 1: "bf16", 2: "fp8"}[int(r["dtype"])]
    return fam + "_tmemB" if r.get("tmem_a", 0) else fam


# ------------------------------------------------------------------ measuring
def _valid(dt, t, tmem_a=0):
    bm, bn, bk, s, g = t
    try:
        pm.pm_gemm_run(pm.cfg(256, 256, 256, bm, bn, bk, s, g, dt, tmem_a=tmem_a), None, None, None)
    except pm.PMError as e:
        return e.status != pm.PM_EUNSUPPORTED
    return True


SETTLE_S = 5.0


def settle(seconds: float = SETTLE_S) -> None:
    """Leave the GPU idle for a few seconds.  After seconds of full-power work
    the SM clock stays capped for a while; short kernels timed in that window
    ran up to 30 % slow, so every block of short kernels that follows heavy
    work starts after this pause."""
    torch.cuda.synchronize()
    time.sleep(seconds)


def measure_sweep(shapes=(1024, 2048, 4096, 8192, 16384), dtypes=(1, 2), log=print) -> dict:
    """Device-timed calibration table (list of records) plus pointer-chase latencies."""
    torch.cuda.nvtx.range_push("measure_sweep")
    rows = []
    t0 = time.time()
    # FP32 (three-pass TF32) GEMM at 512^3 over the FP32 tile space
    A, B = S.gemm_operands(512, 512, 512, seed=0)
    ops = pm.GemmOperands(pm.PM_FP32, 512, 512, 512)
    ops.prepare(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    C = torch.empty(512, 512, dtype=torch.float32, device="cuda")
    for t in S.tile_space(0):
        if not _valid(0, t):
            continue
        r = ops.bench(pm.cfg(512, 512, 512, *t, dtype=0), C, warmup=10, reps=100)
        rows.append(dict(zip(FIELDS, (512, 512, 512, *t, 0, 0, 0)), t=r["median_s"], p25=r["p25_s"],
                         p75=r["p75_s"], **clock_of(r)))
    log("FP32 512^3 done (%d rows, %.0f s)" % (len(rows), time.time() - t0))
    # memory probes: copy / triad over 2^20 .. 2^30 FP32 elements
    nmax = 2 ** 30
    a = torch.from_numpy(S.uniform_pm1(1, nmax)).cuda()
    b = torch.empty_like(a)
    c = torch.from_numpy(S.uniform_pm1(1, nmax, offset=nmax)).cuda()
    for k in range(20, 31):
        n = 2 ** k
        for kind, pk in ((pm.PM_KIND_COPY, pm.PM_PROBE_COPY), (pm.PM_KIND_TRIAD, pm.PM_PROBE_TRIAD)):
            args = pm.probe_args(pk, n=n, scalar=3.0)
            r = pm.pm_probe_run(args, a, b, c, warmup=10, reps=100) if pk == pm.PM_PROBE_TRIAD else \
                pm.pm_probe_run(args, a, b, warmup=10, reps=100)
            rows.append(dict(M=n, N=0, K=0, BM=0, BN=0, BK=0, stages=0, cta_group=0, dtype=0, kind=kind,
                             t=r["median_s"], p25=r["p25_s"], p75=r["p75_s"], **clock_of(r)))
    del b, c
    # TMA 2D tiles over a 1 GiB FP32 matrix (16384 x 16384)
    src = a[: 16384 * 16384].view(16384, 16384)
    dst = torch.empty_like(src)
    for tr, tc in ((64, 64), (128, 64), (128, 128), (256, 64), (256, 128)):
        r = pm.pm_probe_run(pm.probe_args(pm.PM_PROBE_TMA2D, rows=16384, cols=16384, tile_r=tr, tile_c=tc),
                            src, dst, warmup=3, reps=20)
        rows.append(dict(M=16384, N=16384, K=0, BM=tr, BN=tc, BK=0, stages=0, cta_group=0, dtype=0,
                         kind=pm.PM_KIND_TMA2D, t=r["median_s"], p25=r["p25_s"], p75=r["p75_s"], **clock_of(r)))
    del a, src, dst
    torch.cuda.empty_cache()
    log("memory probes done (%.0f s)" % (time.time() - t0))
    # pointer chase: 16 KB .. 1 GB working sets, 64-byte node stride
    pchase = []
    for k in range(17):
        W = 16 * 1024 * 2 ** k
        nodes = W // 64
        buf = torch.from_numpy(S.pchase_buffer(nodes, seed=1).view(np.int32)).cuda()
        out = torch.zeros(1, dtype=torch.int32, device="cuda")
        hops = 2 ** 18
        # warm-up launches walk the whole cycle once where that is affordable,
        # so working sets that fit a cache level are timed resident; larger
        # ones are walked cold (every launch continues to new nodes)
        warm = min(-(-nodes // hops) + 1, 9)
        r = pm.pm_probe_run(pm.probe_args(pm.PM_PROBE_PCHASE, n=nodes, hops=hops, start=0), buf, out,
                            warmup=warm, reps=3)
        pchase.append(dict(W=W, hops=hops, ns_per_hop=1e9 * r["median_s"] / hops, final_index=r["final_index"]))
        del buf
    log("pointer chase done (%.0f s)" % (time.time() - t0))
    # Blackwell instruction probes (Sec. V-A (iii)-(iv)) and the host link (Eq. 15)
    instr = measure_instructions()
    log("instruction and host-link probes done (%.0f s)" % (time.time() - t0))
    streams = measure_streams()
    settle()
    log("concurrent-stream probes done (%.0f s)" % (time.time() - t0))
    # BF16 / FP8 sweep: every valid configuration at M = N = K = s
    for s in shapes:
        A, B = S.gemm_operands(s, s, s, seed=2, dist="normal")
        Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        del A, B
        C = torch.empty(s, s, dtype=torch.float32, device="cuda")
        reps = 100 if s <= 4096 else (40 if s <= 8192 else 20)
        for dt in dtypes:
            ops = pm.GemmOperands(dt, s, s, s)
            ops.prepare(Ad, Bd)
            for t in S.tile_space(dt):
                if not _valid(dt, t):
                    continue
                r = ops.bench(pm.cfg(s, s, s, *t, dtype=dt), C, warmup=10, reps=reps)
                rows.append(dict(zip(FIELDS, (s, s, s, *t, dt, 0, 0)), t=r["median_s"], p25=r["p25_s"],
                                 p75=r["p75_s"], **clock_of(r)))
            del ops
        del Ad, Bd, C
        torch.cuda.empty_cache()
        log("BF16/FP8 %d^3 done (%d rows, %.0f s)" % (s, len(rows), time.time() - t0))
    settle()
    rows += measure_tmem_b(shapes, dtypes, log)
    settle()
    props = torch.cuda.get_device_properties(0)
    segments = measure_segments(dict(rows=rows), log)
    settle()
    grouped = measure_grouped(grouped_theta(props.multi_processor_count, dict(instr=instr)),
                              props.multi_processor_count, log=log)
    torch.cuda.nvtx.range_pop()
    return dict(environment=environment(), device=props.name, n_sm=props.multi_processor_count, rows=rows, pchase=pchase, instr=instr,
                streams=streams, segments=segments, grouped=grouped,
                protocol="10 warm-ups; 100 timed runs (20-40 at 8192-16384, 20 for TMA), median of CUDA-event times; "
                         "grouped launches 3 warm-ups, median of 15")


def measure_tmem_b(shapes=(1024, 2048, 4096, 8192, 16384), dtypes=(1, 2), log=print) -> list:
    """GEMM rows under TMEM strategy B: FP32 512^3 and BF16/FP8 at M = N = K in
    `shapes`, every strategy-B tile, same protocol as the strategy-A rows."""
    rows = []
    t0 = time.time()
    cases = [(512, (0,))] + [(s, tuple(dtypes)) for s in shapes]
    for s, dts in cases:
        A, B = S.gemm_operands(s, s, s, seed=0 if s == 512 else 2, dist="uniform" if s == 512 else "normal")
        Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        del A, B
        C = torch.empty(s, s, dtype=torch.float32, device="cuda")
        reps = 100 if s <= 4096 else (40 if s <= 8192 else 20)
        for dt in dts:
            ops = pm.GemmOperands(dt, s, s, s)
            ops.prepare(Ad, Bd)
            for t in S.tile_space(dt):
                if not _valid(dt, t, 1):
                    continue
                r = ops.bench(pm.cfg(s, s, s, *t, dtype=dt, tmem_a=1), C, warmup=10, reps=reps)
                rows.append(dict(zip(FIELDS, (s, s, s, *t, dt, 0, 1)), t=r["median_s"], p25=r["p25_s"],
                                 p75=r["p75_s"], **clock_of(r)))
            del ops
        del Ad, Bd, C
        torch.cuda.empty_cache()
        log("strategy B shape %d done (%d rows, %.0f s)" % (s, len(rows), time.time() - t0))
    return rows


def measure_instructions() -> dict:
    """tcgen05.mma time per instruction by shape and dtype (all SMs issuing),
    mbarrier round trip, TMEM load/store bandwidth per SM, and copy-engine
    transfer times over the host link for Eq. 15."""
    n_sm = pm.sm_count()
    out = {"mma": [], "host": []}
    buf = torch.zeros(max(n_sm, 2) * 256, dtype=torch.int32, device="cuda")
    n = 1 << 15
    for dt in (0, 1, 2):
        for cg, M, N in ((1, 64, 256), (1, 128, 128), (1, 128, 256), (2, 128, 256), (2, 256, 128), (2, 256, 256)):
            r = pm.pm_probe_run(pm.probe_args(pm.PM_PROBE_MMA, n=n, tile_r=N, tile_c=M, rows=cg, cols=dt), buf,
                                warmup=2, reps=5)
            out["mma"].append(dict(dtype=dt, cta_group=cg, M=M, N=N, ns_per_instr=1e9 * r["median_s"] / n,
                                   tflops=r["bytes"] / r["median_s"] / 1e12))
    r = pm.pm_probe_run(pm.probe_args(pm.PM_PROBE_MBAR, n=1 << 16), buf, warmup=1, reps=5)
    out["mbar_round_trip_ns"] = 1e9 * r["median_s"] / (1 << 16)
    for kind, name in ((pm.PM_PROBE_TMEM_LD, "tmem_ld"), (pm.PM_PROBE_TMEM_ST, "tmem_st")):
        r = pm.pm_probe_run(pm.probe_args(kind, n=256), buf, warmup=1, reps=5)
        out[name + "_bytes_per_s_per_sm"] = r["bytes"] / r["median_s"] / n_sm
    for k in range(12, 31, 2):
        nb = 1 << k
        h = torch.empty(nb, dtype=torch.uint8).pin_memory()
        d = torch.empty(nb, dtype=torch.uint8, device="cuda")
        r1 = pm.pm_probe_run(pm.probe_args(pm.PM_PROBE_H2D, n=nb), h, d, warmup=2, reps=10)
        r2 = pm.pm_probe_run(pm.probe_args(pm.PM_PROBE_D2H, n=nb), d, h, warmup=2, reps=10)
        # the same transfers driven by the SMs through the host mapping (no copy engine)
        r3 = pm.pm_probe_run(pm.probe_args(pm.PM_PROBE_HOST_READ, n=nb // 4), h, d, warmup=2, reps=10)
        r4 = pm.pm_probe_run(pm.probe_args(pm.PM_PROBE_HOST_WRITE, n=nb // 4), d, h, warmup=2, reps=10)
        out["host"].append(dict(bytes=nb, h2d_s=r1["median_s"], d2h_s=r2["median_s"], h2d_sm_s=r3["median_s"],
                                d2h_sm_s=r4["median_s"]))
        del h, d
    out["eq15"] = fit_eq15(out["host"])
    return out


STREAM_COUNTS = (1, 2, 3, 4, 6, 8)


def pchase_levels(pchase, l1_bytes: float, l2_bytes: float) -> dict:
    """Three-level latency step L(W) from the pointer chase: the median ns/hop
    of the working sets well inside each level (W <= L1/2; 2 L1 <= W <= L2/2;
    W >= 4 L2), with the capacities of the device."""
    W = np.array([p["W"] for p in pchase], dtype=np.float64)
    ns = np.array([p["ns_per_hop"] for p in pchase], dtype=np.float64)
    out = dict(l1_bytes=float(l1_bytes), l2_bytes=float(l2_bytes))
    for name, m in (("l1_ns", W <= l1_bytes / 2), ("l2_ns", (W >= 2 * l1_bytes) & (W <= l2_bytes / 2)),
                    ("dram_ns", W >= 4 * l2_bytes)):
        out[name] = float(np.median(ns[m])) if m.any() else None
        out[name.replace("_ns", "_points")] = int(m.sum())
    return out


def fit_tau_c(counts, times) -> dict:
    """Least-squares tau_c of T(N_c) = T(1) + (N_c - 1) tau_c (Sec. III-A.6),
    with T(1) the measured single-stream time, and the MAE of that law over
    the N_c > 1 points."""
    counts = np.asarray(counts, dtype=np.float64)
    times = np.asarray(times, dtype=np.float64)
    t1 = float(times[counts == 1][0])
    x = counts - 1.0
    tau = float(np.sum(x * (times - t1)) / np.sum(x * x))
    pred = t1 + x * tau
    m = counts > 1
    return dict(T1_s=t1, tau_c_s=tau, tau_over_T1=tau / t1,
                mae_pct=float(np.mean(np.abs(pred[m] - times[m]) / times[m]) * 100.0))


def measure_streams(counts=STREAM_COUNTS) -> dict:
    """Makespan of N_c concurrent copies of one probe kernel on N_c streams:
    a bandwidth-bound triad that fills the GPU, a launch-bound small copy, and
    tcgen05.mma streams that occupy an eighth of the SMs or all of them."""
    n_sm = pm.sm_count()
    k = max(counts)
    out = {}
    nt = 1 << 24
    a = [torch.empty(nt, dtype=torch.float32, device="cuda") for _ in range(k)]
    b = [torch.empty(nt, dtype=torch.float32, device="cuda").uniform_(-1, 1) for _ in range(k)]
    c = [torch.empty(nt, dtype=torch.float32, device="cuda").uniform_(-1, 1) for _ in range(k)]
    mma = [torch.zeros(n_sm, dtype=torch.int32, device="cuda") for _ in range(k)]
    classes = {
        "triad_2^24_per_stream": (pm.probe_args(pm.PM_PROBE_TRIAD, n=nt, scalar=3.0), (a, b, c)),
        "copy_2^16_per_stream": (pm.probe_args(pm.PM_PROBE_COPY, n=1 << 16), (b, a, None)),
        "mma_bf16_%d_ctas_per_stream" % (n_sm // 8): (
            pm.probe_args(pm.PM_PROBE_MMA, n=1 << 13, tile_r=256, tile_c=128, rows=1, cols=1, start=n_sm // 8),
            (mma, None, None)),
        "mma_bf16_%d_ctas_per_stream" % n_sm: (
            pm.probe_args(pm.PM_PROBE_MMA, n=1 << 13, tile_r=256, tile_c=128, rows=1, cols=1, start=n_sm),
            (mma, None, None)),
    }
    for name, (args, (x0, x1, x2)) in classes.items():
        times = []
        for nc in counts:
            r = pm.pm_streams_run(args, x0[:nc], x1[:nc] if x1 else None, x2[:nc] if x2 else None, warmup=5,
                                  reps=30)
            times.append(r["median_s"])
        out[name] = dict(counts=list(counts), t_s=times, fit=fit_tau_c(counts, times))
    return out


def fit_eq15(host_rows) -> dict:
    """Least-squares fit of Eq. 15, T = S / B_dir + tau, per direction
    (weighted by 1/T so small and large transfers count alike)."""
    res = {}
    S_ = np.array([r["bytes"] for r in host_rows], dtype=np.float64)
    for d in ("h2d", "d2h", "h2d_sm", "d2h_sm"):
        if not all((d + "_s") in r for r in host_rows):
            continue
        T = np.array([r[d + "_s"] for r in host_rows], dtype=np.float64)
        A = np.stack([S_ / T, 1.0 / T], 1)          # rows scaled by 1/T: S/T * (1/B) + (1/T) * tau = 1
        coef, *_ = np.linalg.lstsq(A, np.ones_like(T), rcond=None)
        inv_b, tau = coef
        pred = S_ * inv_b + tau
        res[d] = dict(B_eff=1.0 / inv_b, tau_s=tau, mae_pct=float(np.mean(np.abs(pred - T) / T) * 100))
    return res


def probe_priors(instr: dict, n_sm: int, f_hz: float = 1.9e9, reading: int = pm.PM_READING_MEASURED) -> np.ndarray:
    """Priors with the probe measurements in place of the paper's printed
    values where a probe measures the parameter itself (Sec. V-A: parameters
    come from microbenchmarks): R_TC^SM per precision from the back-to-back
    tcgen05.mma rate (one SM, M = 128, N = 256), L_mbar from half an mbarrier
    round trip, TMEM read/write bandwidth per SM from the TMEM probes.  L_mma
    keeps the printed instruction latency (the probe measures throughput)."""
    th = prior_theta(n_sm, f_hz, reading)
    for dt, j in ((0, 6), (1, 7), (2, 8)):
        m = [x for x in instr["mma"] if x["dtype"] == dt and x["cta_group"] == 1 and x["M"] == 128 and x["N"] == 256]
        if m:
            th[j] = m[0]["tflops"] * 1e12 / n_sm
    th[12] = 0.5 * instr["mbar_round_trip_ns"] * 1e-9
    th[10] = instr["tmem_ld_bytes_per_s_per_sm"]
    th[11] = instr["tmem_st_bytes_per_s_per_sm"]
    return th


# ------------------------------------------------------------ autograd + fit
class StageModelLoss(torch.autograd.Function):
    """L(theta) = mean_i (ln T_hat_i(theta) - ln T_i)^2 on the GPU; the backward
    pass returns the gradient from the hand-written adjoint kernel.  A float64
    t_meas selects the all-FP64 evaluation (pm_model_grad_f64)."""

    @staticmethod
    def forward(ctx, theta, cfg_dev, n, t_meas_dev, n_sm, workspace):
        out = torch.empty(pm.N_GRAD_OUT, dtype=torch.float64, device=cfg_dev.device)
        grad_fn = pm.pm_model_grad_f64 if t_meas_dev.dtype == torch.float64 else pm.pm_model_grad
        grad_fn(cfg_dev, n, theta.detach().cpu().numpy(), n_sm, t_meas_dev, workspace, out)
        o = out.cpu()
        ctx.save_for_backward(o[1:].clone().to(theta.dtype))
        return o[0].to(theta.dtype)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None, None, None, None, None


class GroupedLoss(torch.autograd.Function):
    """Sum over grouped launches of (ln T_hat - ln T)^2, T_hat the stage
    model's makespan of the launch's schedule (pm_grouped_grad, FP64 on the
    GPU); the backward pass returns the sum of the makespans' gradients."""

    @staticmethod
    def forward(ctx, theta, grouped, n_sm):
        th = theta.detach().cpu().numpy()
        total, grad = 0.0, np.zeros(pm.N_PARAMS)
        for r in grouped:
            t_hat, g = pm.pm_grouped_grad(r["M"], r["N"], r["K"], r["bm"], r["bn"], *r["launch"], pm.PM_BF16, th,
                                          n_sm)
            res = math.log(t_hat) - math.log(r["t"])
            total += res * res
            grad += 2.0 * res * g / t_hat
        ctx.save_for_backward(torch.tensor(grad, dtype=theta.dtype))
        return torch.tensor(total, dtype=theta.dtype)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None, None


class GpuObjective:
    """Binds a calibration table to the GPU loss: call with theta (float64
    tensor).  rows: configuration records (pm_cfg fields and the measured t);
    grouped: measured grouped launches (the grouped family), each one term of the mean
    like a configuration."""

    def __init__(self, rows, n_sm, grouped=()):
        self.n = len(rows)
        cols = {f: np.array([r.get(f, 0) for r in rows], dtype=np.int64) for f in FIELDS}
        self.cfg = pm.cfg_tensor(cols)
        self.t = torch.tensor([r["t"] for r in rows], dtype=torch.float64, device="cuda")
        self.ws = torch.empty(pm.pm_model_grad_workspace(self.n) // 8 + 1, dtype=torch.float64, device="cuda")
        self.n_sm = n_sm
        self.grouped = list(grouped)

    def __call__(self, theta):
        loss = StageModelLoss.apply(theta, self.cfg, self.n, self.t, self.n_sm, self.ws)
        if not self.grouped:
            return loss
        n_g = len(self.grouped)
        return (self.n * loss + GroupedLoss.apply(theta, self.grouped, self.n_sm)) / (self.n + n_g)

    def predict(self, theta) -> np.ndarray:
        out = torch.empty(self.n, dtype=torch.float32, device="cuda")
        pm.pm_model_predict(self.cfg, self.n, np.asarray(theta, dtype=np.float64), self.n_sm, out)
        return out.cpu().numpy().astype(np.float64)

    def predict_grouped(self, theta) -> np.ndarray:
        return predict_grouped(self.grouped, theta, self.n_sm)


def predict_grouped(grouped, theta, n_sm) -> np.ndarray:
    """The stage model's makespan (pm_grouped_predict) of each grouped launch."""
    return np.array([pm.pm_grouped_predict(r["M"], r["N"], r["K"], r["bm"], r["bn"], *r["launch"], pm.PM_BF16,
                                           np.asarray(theta, dtype=np.float64), n_sm) for r in grouped])


# Parameter pairs (lo, hi) the fit keeps ordered, theta[lo] <= theta[hi]:
# Eq. 16 blends from the peak bandwidth for small working sets down to the
# sustained one, so B_peak >= B_sus.  With B_sus above B_peak the blend never
# beats the B_peak floor, B_sus and w0 drop out of the memory-probe times and
# (under the literal reading, where nothing else uses them) their gradient is
# zero: a dead region a descent method cannot leave.
ORDERED = ((1, 2),)


def fit(objective, theta0, prior=None, reg=1e-4, iters=500, rounds=3, log=None, ordered=ORDERED, order_weight=1.0,
        polish=8):
    """Minimise objective(theta) + reg * ||ln theta - ln prior||^2 over phi = ln theta:
    L-BFGS, restarted `rounds` times from its own end point, then up to
    `polish` Newton steps (newton_polish).  A one-sided penalty
    order_weight * max(0, phi_lo - phi_hi)^2 per pair in `ordered` steers the
    fit out of regions the model's ordering assumptions exclude; it is zero
    wherever the ordering holds, so it does not move an admissible optimum."""
    theta0 = np.asarray(theta0, dtype=np.float64)
    prior = theta0 if prior is None else np.asarray(prior, dtype=np.float64)
    phi = torch.tensor(np.log(theta0), dtype=torch.float64, requires_grad=True)
    phi_p = torch.tensor(np.log(prior), dtype=torch.float64)
    trace = []

    def total(p):
        loss = objective(torch.exp(p)) + reg * torch.sum((p - phi_p) ** 2)
        for lo, hi in ordered:
            loss = loss + order_weight * torch.clamp(p[lo] - p[hi], min=0.0) ** 2
        return loss

    opt = torch.optim.LBFGS([phi], lr=1.0, max_iter=iters, tolerance_grad=1e-12, tolerance_change=1e-15,
                            history_size=50, line_search_fn="strong_wolfe")

    def closure():
        opt.zero_grad()
        loss = total(phi)
        loss.backward()
        trace.append(float(loss.item()))
        return loss

    for _ in range(rounds):
        opt.step(closure)

    def value_grad(p_np):
        p = torch.tensor(p_np, dtype=torch.float64, requires_grad=True)
        loss = total(p)
        loss.backward()
        return float(loss.item()), p.grad.numpy().copy()

    phi_np = newton_polish(value_grad, phi.detach().numpy().copy(), steps=polish, trace=trace)
    if log:
        log("fit: %d evaluations, loss %.4g -> %.4g" % (len(trace), trace[0], trace[-1]))
    return np.exp(phi_np), trace


def newton_polish(value_grad, phi, steps=8, h=1e-4, rcond=1e-12, trace=None):
    """Newton steps on a smooth piece of the objective, from phi.  The
    Hessian is the central difference of the gradient (2 x 16 gradient
    evaluations; the GPU objective gives loss and gradient only), made
    symmetric; directions with eigenvalues at or below rcond x the largest
    (unidentifiable combinations of parameters, or negative curvature) are
    left alone.  Each step is halved until the loss decreases; the polish
    stops when no step decreases it.  L-BFGS crawls along the objective's
    badly conditioned directions (Eq. 16's B_peak and w0 are seen only
    through the smallest memory probes); a few Newton steps finish them."""
    n = len(phi)
    L, g = value_grad(phi)
    for _ in range(steps):
        H = np.empty((n, n))
        for j in range(n):
            e = np.zeros(n)
            e[j] = h
            H[:, j] = (value_grad(phi + e)[1] - value_grad(phi - e)[1]) / (2 * h)
        H = 0.5 * (H + H.T)
        w, V = np.linalg.eigh(H)
        keep = w > rcond * max(w.max(), 0.0)
        if not keep.any():
            break
        step = -V[:, keep] @ ((V[:, keep].T @ g) / w[keep])
        t, moved = 1.0, False
        while t >= 1.0 / 1024:
            L2, g2 = value_grad(phi + t * step)
            if L2 < L:
                phi, L, g, moved = phi + t * step, L2, g2, True
                break
            t *= 0.5
        if trace is not None:
            trace.append(L)
        if not moved:
            break
    return phi


def split(n: int, holdout: float = 0.2, seed: int = 6):
    """Seeded train/holdout split (Sec. III-D recommends a holdout)."""
    order = np.argsort(S.splitmix64(seed, n), kind="stable")
    k = int(round(n * holdout))
    hold = np.zeros(n, dtype=bool)
    hold[order[:k]] = True
    return ~hold, hold


def mae_by_family(rows, t_pred, mask=None) -> dict:
    out = {}
    fam = np.array([family_of(r) for r in rows])
    t = np.array([r["t"] for r in rows])
    ape = np.abs(t_pred - t) / t * 100.0
    if mask is None:
        mask = np.ones(len(rows), dtype=bool)
    for f in sorted(set(fam)):
        m = (fam == f) & mask
        if m.any():
            out[f] = dict(n=int(m.sum()), mae_pct=float(ape[m].mean()), median_ape_pct=float(np.median(ape[m])),
                          max_ape_pct=float(ape[m].max()))
    out["all"] = dict(n=int(mask.sum()), mae_pct=float(ape[mask].mean()))
    return out


def roofline_mae(rows, peaks) -> dict:
    """Naive roofline with datasheet peaks (Sec. V-A context): max(FLOPs/P, bytes/B)."""
    fam = np.array([family_of(r) for r in rows])
    t = np.array([r["t"] for r in rows])
    pred = np.zeros(len(rows))
    for i, r in enumerate(rows):
        if r["kind"] in (pm.PM_KIND_COPY, pm.PM_KIND_TRIAD):
            pred[i] = (8.0 if r["kind"] == pm.PM_KIND_COPY else 12.0) * r["M"] / peaks["hbm"]
        elif r["kind"] == pm.PM_KIND_TMA2D:
            pred[i] = 8.0 * r["M"] * r["N"] / peaks["hbm"]
        else:
            e = {0: 4.0, 1: 2.0, 2: 1.0}[r["dtype"]]
            P = {0: peaks["tf32"], 1: peaks["bf16"], 2: peaks["fp8"]}[r["dtype"]]
            flops = 2.0 * r["M"] * r["N"] * r["K"]
            bytes_ = e * (r["M"] * r["K"] + r["N"] * r["K"]) + 4.0 * r["M"] * r["N"]
            pred[i] = max(flops / P, bytes_ / peaks["hbm"])
    ape = np.abs(pred - t) / t * 100
    return {f: float(ape[fam == f].mean()) for f in sorted(set(fam))} | {"all": float(ape.mean())}


def autotune_vs_best(rows, theta, n_sm) -> list:
    """For each measured GEMM shape: the model's pick (GPU autotuner) against the
    fastest measured configuration."""
    out = []
    gem = [r for r in rows if r["kind"] == pm.PM_KIND_GEMM and not r.get("tmem_a", 0)]
    keys = sorted(set((r["M"], r["N"], r["K"], r["dtype"]) for r in gem))
    for (M, N, K, dt) in keys:
        cand = {(r["BM"], r["BN"], r["BK"], r["stages"], r["cta_group"]): r["t"] for r in gem
                if (r["M"], r["N"], r["K"], r["dtype"]) == (M, N, K, dt)}
        MNK = torch.tensor([M, N, K], dtype=torch.int32, device="cuda")
        picks = torch.empty(24, dtype=torch.uint8, device="cuda")
        tp = torch.empty(1, dtype=torch.float32, device="cuda")
        pm.pm_autotune_pick(MNK, 1, dt, theta, n_sm, picks, tp)
        p = picks.cpu().numpy().view(pm.CFG_DTYPE)[0]
        pick = (int(p["BM"]), int(p["BN"]), int(p["BK"]), int(p["stages"]), int(p["cta_group"]))
        best = min(cand, key=cand.get)
        flops = 2.0 * M * N * K
        out.append(dict(M=M, N=N, K=K, dtype=dt, pick=pick, t_pick=cand.get(pick), best=best, t_best=cand[best],
                        t_pred=float(tp.item()), pick_over_best=cand.get(pick, math.inf) / cand[best],
                        tflops_pick=flops / cand.get(pick, math.inf) / 1e12, tflops_best=flops / cand[best] / 1e12))
    return out


def two_sm_report(rows) -> dict:
    """Measured CTA-pair speedup (Sec. V reports 1.28-1.30x on B200): per GEMM
    shape and dtype, the fastest one-SM tile's time over the fastest pair
    tile's, and the median over tiles that exist in both forms."""
    out = {}
    gem = [r for r in rows if r["kind"] == pm.PM_KIND_GEMM and not r.get("tmem_a", 0)]
    for dt in sorted(set(r["dtype"] for r in gem)):
        best_ratio, same = [], []
        for M in sorted(set(r["M"] for r in gem if r["dtype"] == dt)):
            cand = [r for r in gem if r["dtype"] == dt and r["M"] == M]
            t1 = [r["t"] for r in cand if r["cta_group"] == 1]
            t2 = [r["t"] for r in cand if r["cta_group"] == 2]
            if t1 and t2:
                best_ratio.append(min(t1) / min(t2))
            by_tile = {(r["BM"], r["BN"], r["BK"], r["stages"], r["cta_group"]): r["t"] for r in cand}
            same += [by_tile[k[:4] + (1,)] / v for k, v in by_tile.items() if k[4] == 2 and k[:4] + (1,) in by_tile]
        if best_ratio:
            out[("fp32", "bf16", "fp8")[dt]] = dict(best_single_over_best_pair=[round(x, 3) for x in best_ratio],
                                                    median_same_tile_speedup=float(np.median(same)) if same else None)
    return out


def environment() -> dict:
    """Where the measurements and the fit ran: GPU, driver and runtime versions, host."""
    import subprocess
    props = torch.cuda.get_device_properties(0)
    driver = None
    try:
        driver = subprocess.run(["nvidia-smi", "--query-gpu=driver_version", "--format=csv,noheader", "-i", "0"],
                                capture_output=True, text=True, timeout=30).stdout.strip() or None
    except (OSError, subprocess.SubprocessError):
        pass
    return dict(gpu=props.name, sm_count=props.multi_processor_count, total_memory=props.total_memory,
                driver=driver, torch=torch.__version__, torch_cuda=torch.version.cuda,
                host_cores=os.cpu_count(), host_machine=os.uname().machine)


def tmem_strategy_report(rows, t_pred) -> list:
    """Per GEMM shape with strategy-B rows: the fastest measured tile of each
    TMEM strategy and what the model predicts for the two (Sec. III-A.1: B
    relieves shared memory but adds TMEM traffic)."""
    out = []
    keys = sorted(set((r["M"], r["dtype"]) for r in rows if r["kind"] == pm.PM_KIND_GEMM and r.get("tmem_a", 0)))
    for (M, dt) in keys:
        best = {}
        for ta in (0, 1):
            idx = [i for i, r in enumerate(rows) if r["kind"] == pm.PM_KIND_GEMM and r["M"] == M and
                   r["dtype"] == dt and r.get("tmem_a", 0) == ta]
            if not idx:
                break
            i = min(idx, key=lambda j: rows[j]["t"])
            ip = min(idx, key=lambda j: t_pred[j])
            best[ta] = dict(tile=[rows[i][f] for f in ("BM", "BN", "BK", "stages", "cta_group")], t=rows[i]["t"],
                            t_pred_of_best=float(t_pred[i]), model_pick_t=rows[ip]["t"])
        if len(best) == 2:
            out.append(dict(M=M, dtype=dt, A=best[0], B=best[1], measured_B_over_A=best[1]["t"] / best[0]["t"],
                            predicted_B_over_A=best[1]["t_pred_of_best"] / best[0]["t_pred_of_best"]))
    return out


def save_theta(theta, meta, path=THETA_PATH):
    with open(path, "w") as f:
        json.dump(dict(theta=[float(v) for v in theta], **meta), f, indent=1)


def load_theta(path=THETA_PATH):
    with open(path) as f:
        return np.array(json.load(f)["theta"], dtype=np.float64)


# ---------------------------------------------------------- generic segments
SEG_FIELDS = ("flops", "bytes", "working_set", "h2d_bytes", "d2h_bytes", "cls", "precision", "kernels", "syncs",
              "execs", "streams")
SEG_CLASS_NAMES = ("memory", "compute", "balanced", "stencil")


def _seg(name, t, **kw):
    r = dict(name=name, t=float(t), flops=0.0, bytes=0.0, working_set=0.0, h2d_bytes=0.0, d2h_bytes=0.0, cls=0,
             precision=pm.PM_BF16, kernels=1, syncs=0, execs=1)
    r.update(kw)
    return r


def _events_median(fn, warmup=3, reps=20):
    for _ in range(warmup):
        fn()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t = []
    for _ in range(reps):
        s.record()
        fn()
        e.record()
        e.synchronize()
        t.append(s.elapsed_time(e) * 1e-3)
    return float(np.median(t))


def measure_segments(table, log=print) -> dict:
    """Measured workload segments for the generic path: the table's copy/triad
    rows (memory) and fastest GEMM tile per shape and dtype (compute), grouped
    GEMMs (balanced), the five-point stencil (stencil), copy-triad chains
    (multi-kernel) and triads wrapped in host transfers and a sync."""
    rows = []
    for r in table["rows"]:
        if r["kind"] in (pm.PM_KIND_COPY, pm.PM_KIND_TRIAD):
            n = r["M"]
            b = (8.0 if r["kind"] == pm.PM_KIND_COPY else 12.0) * n
            rows.append(_seg("copy" if r["kind"] == pm.PM_KIND_COPY else "triad", r["t"], cls=0,
                             precision=pm.PM_FP32, flops=0.0 if r["kind"] == pm.PM_KIND_COPY else 2.0 * n, bytes=b,
                             working_set=b))
    best = {}
    for r in table["rows"]:
        if r["kind"] == pm.PM_KIND_GEMM and not r.get("tmem_a", 0):
            key = (r["M"], r["N"], r["K"], r["dtype"])
            if key not in best or r["t"] < best[key]["t"]:
                best[key] = r
    for (M, N, K, dt), r in sorted(best.items()):
        e = {0: 8.0, 1: 2.0, 2: 1.0}[dt]                   # operand bytes per element (FP32: hi and lo)
        b = e * (M * K + N * K) + 4.0 * M * N
        rows.append(_seg("gemm_%d_%s" % (M, ("fp32", "bf16", "fp8")[dt]), r["t"], cls=1, precision=dt,
                         flops=2.0 * M * N * K, bytes=b, working_set=b))
    n_sm = pm.sm_count()
    theta = prior_theta(n_sm)
    # balanced: grouped GEMMs, launch from the measured grouped autotuner
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    for G, seed, NK in ((64, 3, 1024), (64, 3, 2048), (64, 3, 4096), (16, 5, 2048), (16, 5, 4096)):
        Mg = S.grouped_m(G, seed)
        sum_m = int(Mg.sum())
        A = torch.randn(sum_m, NK, device="cuda", generator=gen).to(torch.bfloat16)
        B = torch.randn(G * NK, NK, device="cuda", generator=gen).to(torch.bfloat16)
        C = torch.empty(sum_m, NK, dtype=torch.float32, device="cuda")
        _, bm, bn, launch, _ = pm.pm_grouped_gemm_autotune(Mg, NK, NK, theta, n_sm, 4, A, B, C, warmup=2, reps=5)
        t = _events_median(lambda: pm.pm_grouped_gemm_run(Mg, NK, NK, bm, bn, *launch, A, B, C))
        flops = float(sum(2.0 * m * NK * NK for m in Mg))
        b = float(sum(2.0 * (m * NK + NK * NK) + 4.0 * m * NK for m in Mg))
        rows.append(_seg("grouped_G%d_NK%d" % (G, NK), t, cls=2, precision=pm.PM_BF16, flops=flops, bytes=b,
                         working_set=b, grouped=dict(M=[int(m) for m in Mg], NK=NK, bm=[int(v) for v in bm],
                                                     bn=[int(v) for v in bn], launch=[int(v) for v in launch])))
        del A, B, C
    # stencil: five-point stencil grids
    for side in (1024, 2048, 4096, 8192, 16384):
        x = torch.empty(side * side, dtype=torch.float32, device="cuda").uniform_(-1, 1)
        y = torch.empty_like(x)
        r = pm.pm_probe_run(pm.probe_args(pm.PM_PROBE_STENCIL, rows=side, cols=side), x, y, warmup=5, reps=30)
        rows.append(_seg("stencil_%d" % side, r["median_s"], cls=3, precision=pm.PM_FP32,
                         flops=6.0 * side * side, bytes=8.0 * side * side, working_set=8.0 * side * side))
        del x, y
    settle()
    # multi-kernel memory segments: copy -> triad (-> copy) on shared buffers
    for k in (20, 24, 27):
        n = 1 << k
        a = torch.empty(n, dtype=torch.float32, device="cuda")
        b = torch.empty(n, dtype=torch.float32, device="cuda").uniform_(-1, 1)
        c = torch.empty(n, dtype=torch.float32, device="cuda").uniform_(-1, 1)
        cp = pm.probe_args(pm.PM_PROBE_COPY, n=n)
        tr = pm.probe_args(pm.PM_PROBE_TRIAD, n=n, scalar=3.0)
        t2 = _events_median(lambda: (pm.pm_probe_launch(cp, b, a), pm.pm_probe_launch(tr, a, b, c)))
        t3 = _events_median(lambda: (pm.pm_probe_launch(cp, b, a), pm.pm_probe_launch(tr, a, b, c),
                                     pm.pm_probe_launch(cp, a, c)))
        rows.append(_seg("copy+triad_2^%d" % k, t2, cls=0, precision=pm.PM_FP32, kernels=2, flops=2.0 * n,
                         bytes=20.0 * n, working_set=12.0 * n))
        rows.append(_seg("copy+triad+copy_2^%d" % k, t3, cls=0, precision=pm.PM_FP32, kernels=3, flops=2.0 * n,
                         bytes=28.0 * n, working_set=12.0 * n))
        del a, b, c
    # host segments: H2D of b, triad, D2H of a, one synchronisation (host clock)
    for k in (20, 24, 27):
        n = 1 << k
        hb = torch.empty(n, dtype=torch.float32).pin_memory()
        hb.uniform_(-1, 1)
        ha = torch.empty(n, dtype=torch.float32).pin_memory()
        a = torch.empty(n, dtype=torch.float32, device="cuda")
        b = torch.empty(n, dtype=torch.float32, device="cuda")
        c = torch.empty(n, dtype=torch.float32, device="cuda").uniform_(-1, 1)
        h2d = pm.probe_args(pm.PM_PROBE_H2D, n=4 * n)
        d2h = pm.probe_args(pm.PM_PROBE_D2H, n=4 * n)
        tr = pm.probe_args(pm.PM_PROBE_TRIAD, n=n, scalar=3.0)
        ts = []
        for i in range(13):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pm.pm_probe_launch(h2d, hb, b)
            pm.pm_probe_launch(tr, a, b, c)
            pm.pm_probe_launch(d2h, a, ha)
            torch.cuda.synchronize()
            if i >= 3:
                ts.append(time.perf_counter() - t0)
        rows.append(_seg("h2d+triad+d2h_2^%d" % k, float(np.median(ts)), cls=0, precision=pm.PM_FP32, flops=2.0 * n,
                         bytes=12.0 * n, working_set=12.0 * n, h2d_bytes=4.0 * n, d2h_bytes=4.0 * n, syncs=1))
        del ha, hb, a, b, c
    # tau_sync: a synchronisation with nothing in flight, host clock
    torch.cuda.synchronize()
    ts = []
    for _ in range(2000):
        t0 = time.perf_counter()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    log("segments measured: %d" % len(rows))
    return dict(rows=rows, tau_sync_s=float(np.median(ts)))


# Grouped problems of the grouped family (the 64-group recipe at several sizes): number of
# groups, seed of M_g = round(exp(U[ln 16, ln 4096])), N = K.
GROUPED_PROBLEMS = ((64, 3, 1024), (64, 3, 2048), (64, 3, 4096), (16, 5, 2048), (16, 5, 4096), (32, 9, 1024))


def measure_grouped(theta, n_sm, problems=GROUPED_PROBLEMS, warmup=3, reps=15, log=print) -> list:
    """Grouped family: every launch-level candidate of the grouped autotuner (its
    per-group tiles under theta) of each grouped BF16 problem, timed as one
    persistent launch (CUDA events, median of `reps`), operands drawn on the
    device from a seeded generator."""
    rows = []
    for G, seed, NK in problems:
        Mg = [int(m) for m in S.grouped_m(G, seed)]
        sum_m = sum(Mg)
        gen = torch.Generator(device="cuda")
        gen.manual_seed(seed)
        A = torch.randn(sum_m, NK, device="cuda", generator=gen).to(torch.bfloat16)
        B = torch.randn(G * NK, NK, device="cuda", generator=gen).to(torch.bfloat16)
        C = torch.empty(sum_m, NK, dtype=torch.float32, device="cuda")
        for t_pred, bm, bn, launch in pm.pm_grouped_candidates(Mg, NK, NK, pm.PM_BF16, theta, n_sm):
            if not math.isfinite(t_pred):
                continue
            run = lambda: pm.pm_grouped_gemm_run(Mg, NK, NK, bm, bn, *launch, A, B, C)
            ts = _events_times(run, warmup, reps)
            rows.append(dict(family="grouped", G=G, seed=seed, M=Mg, N=NK, K=NK, bm=bm, bn=bn,
                             launch=list(launch), t=float(np.median(ts)), p25=float(np.percentile(ts, 25)),
                             p75=float(np.percentile(ts, 75))))
        del A, B, C
        torch.cuda.empty_cache()
        log("grouped G=%d N=K=%d: %d launches" % (G, NK, sum(1 for r in rows if r["G"] == G and r["N"] == NK)))
    return rows


def _events_times(fn, warmup, reps) -> list:
    for _ in range(warmup):
        fn()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        a.record()
        fn()
        b.record()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) * 1e-3 for a, b in ev]


def grouped_theta(n_sm, table) -> np.ndarray:
    """The theta whose grouped-autotuner candidates are measured: the
    calibrated file of the measured reading if there is one, else the probe
    priors."""
    if os.path.exists(THETA_PATH):
        th = load_theta(THETA_PATH)
        if th.size == pm.N_PARAMS:
            return th
    return probe_priors(table["instr"], n_sm) if table.get("instr") else prior_theta(n_sm)


def grouped_autotune_report(grouped, theta, n_sm) -> list:
    """Per grouped problem: the stage model's own pick (pm_grouped_autotune)
    against the fastest measured launch candidate."""
    out = []
    for key in sorted(set((r["G"], r["seed"], r["N"]) for r in grouped)):
        cand = [r for r in grouped if (r["G"], r["seed"], r["N"]) == key]
        best = min(cand, key=lambda r: r["t"])
        _, bm, bn, launch = pm.pm_grouped_autotune(cand[0]["M"], key[2], key[2], pm.PM_BF16, theta, n_sm)
        pick = [r for r in cand if tuple(r["launch"]) == tuple(launch) and list(r["bm"]) == list(bm)
                and list(r["bn"]) == list(bn)]
        out.append(dict(G=key[0], seed=key[1], N=key[2], K=key[2], pick_launch=list(launch),
                        best_launch=best["launch"], t_best=best["t"], t_pick=pick[0]["t"] if pick else None,
                        pick_over_best=pick[0]["t"] / best["t"] if pick else None))
    return out


def grouped_family(seg_table, theta, n_sm) -> dict:
    """Grouped GEMM family: the stage model's makespan (pm_grouped_predict)
    of each measured grouped launch against its time."""
    out = []
    for r in seg_table["rows"]:
        gq = r.get("grouped")
        if not gq:
            continue
        t_pred = pm.pm_grouped_predict(gq["M"], gq["NK"], gq["NK"], gq["bm"], gq["bn"], *gq["launch"], pm.PM_BF16,
                                       theta, n_sm)
        out.append(dict(name=r["name"], t=r["t"], pred=t_pred, ape_pct=abs(t_pred - r["t"]) / r["t"] * 100.0))
    if not out:
        return {}
    return dict(n=len(out), mae_pct=float(np.mean([x["ape_pct"] for x in out])), rows=out)


def _seg_predict(rows, theta, psi, n_sm):
    return pm.pm_segment_predict(pm.segment_array({f: np.array([r.get(f, 1 if f == "execs" else 0) for r in rows])
                                                   for f in SEG_FIELDS}), theta, psi, n_sm)


def _fit_1d(rows, theta, psi, n_sm, idx, lo=1e-3, hi=1e3):
    """psi[idx] minimising the squared log error over rows (golden section on ln psi[idx])."""
    t = np.array([r["t"] for r in rows])
    a, b = math.log(lo), math.log(hi)
    g = (math.sqrt(5.0) - 1.0) / 2.0

    def f(x):
        p = psi.copy()
        p[idx] = math.exp(x)
        return float(np.sum((np.log(_seg_predict(rows, theta, p, n_sm)) - np.log(t)) ** 2))

    c, d = b - g * (b - a), a + g * (b - a)
    fc, fd = f(c), f(d)
    for _ in range(80):
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - g * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + g * (b - a)
            fd = f(d)
    return math.exp(0.5 * (a + b))


def stream_segments(name: str, n_sm: int):
    """The concurrent-stream probe classes of measure_streams as generic-path
    segments (one launch per stream), or None for a class the generic path
    cannot describe: the MMA probe on an eighth of the SMs runs at a fraction
    of the chip's rate, which a full-chip roofline has no term for."""
    if name.startswith("triad_2^"):
        n = 1 << int(name.split("^")[1].split("_")[0])
        return dict(flops=2.0 * n, bytes=12.0 * n, working_set=12.0 * n, cls=pm.PM_SEG_MEMORY,
                    precision=pm.PM_FP32, kernels=1)
    if name.startswith("copy_2^"):
        n = 1 << int(name.split("^")[1].split("_")[0])
        return dict(flops=0.0, bytes=8.0 * n, working_set=8.0 * n, cls=pm.PM_SEG_MEMORY, precision=pm.PM_FP32,
                    kernels=1)
    if name == "mma_bf16_%d_ctas_per_stream" % n_sm:
        # the probe: n_sm CTAs x 2^13 tcgen05.mma of 128 x 256 x 16 (BF16)
        return dict(flops=float(n_sm) * (1 << 13) * 2.0 * 128 * 256 * 16, bytes=0.0, working_set=0.0,
                    cls=pm.PM_SEG_COMPUTE, precision=pm.PM_BF16, kernels=1)
    return None


def fit_stream_interference(streams: dict, theta, psi, n_sm) -> dict:
    """kappa_launch and kappa per class of the generic path's concurrent-stream
    term (Sec. III-A.6: N_c concurrent copies add (N_c - 1) tau_c), with
    tau_c = kappa_launch * launches + kappa_class * roofline term, by least
    squares on the measured makespan increments T(N_c) - T(1) of the probe
    classes (kappa >= 0).  The balanced class takes the compute kappa and the
    stencil class the memory one (no probe of their own).  Returns psi with
    entries 12-16 filled, and per class the makespans the generic path then
    predicts (its own single-stream time plus the term) with their MAE."""
    psi = np.array(psi, dtype=np.float64)
    cases = []
    for name, v in streams.items():
        seg = stream_segments(name, n_sm)
        if seg is None:
            continue
        base = dict(seg, streams=1)
        one = _seg_predict([base], theta, np.concatenate([psi[:12], np.zeros(5)]), n_sm)[0]
        launches = seg["kernels"] * float(theta[0])
        roof = one - launches
        cases.append((name, seg, np.array(v["counts"], dtype=np.float64), np.array(v["t_s"]), launches, roof))
    if not cases:
        psi[12:17] = 1.0
        return dict(psi=psi.tolist(), classes={})
    # unknowns x = (kappa_launch, kappa_memory, kappa_compute)
    rows_a, rows_b = [], []
    for _, seg, counts, t, launches, roof in cases:
        t1 = t[counts == 1][0]
        for c, tc in zip(counts, t):
            if c > 1:
                k = c - 1.0
                a = [k * launches, k * roof if seg["cls"] == pm.PM_SEG_MEMORY else 0.0,
                     k * roof if seg["cls"] == pm.PM_SEG_COMPUTE else 0.0]
                w = 1.0 / tc                                   # relative errors
                rows_a.append([x * w for x in a])
                rows_b.append((tc - t1) * w)
    A, b = np.array(rows_a), np.array(rows_b)
    active = [j for j in range(3) if np.any(A[:, j] != 0.0)]
    x = np.zeros(3)
    while active:
        sol = np.linalg.lstsq(A[:, active], b, rcond=None)[0]
        if np.all(sol >= 0.0):
            x[active] = sol
            break
        active.remove(active[int(np.argmin(sol))])            # drop the most negative, refit (kappa >= 0)
    psi[16] = x[0]
    psi[12] = psi[15] = x[1]                                   # memory, stencil
    psi[13] = psi[14] = x[2]                                   # compute, balanced
    out = {}
    for name, seg, counts, t, _, _ in cases:
        pred = _seg_predict([dict(seg, streams=int(c)) for c in counts], theta, psi, n_sm)
        m = counts > 1
        out[name] = dict(counts=counts.tolist(), t_s=t.tolist(), pred_s=pred.tolist(),
                         mae_pct=float(np.mean(np.abs(pred[m] - t[m]) / t[m]) * 100.0),
                         single_stream_ape_pct=float(abs(pred[0] - t[0]) / t[0] * 100.0))
    return dict(psi=psi.tolist(), kappa_launch=float(x[0]), kappa_memory=float(x[1]), kappa_compute=float(x[2]),
                classes=out)


def fit_segments(seg_table, theta, n_sm, eq15=None, streams=None) -> dict:
    """psi of the generic path: host link from the Eq. 15 fit, tau_sync measured,
    one scale per class and an efficiency per precision (BF16's fixed at 1)
    fitted to the measured segments; MAE per class in-sample and leave-one-out;
    the concurrent-stream entries from the stream probes (fit_stream_interference)."""
    rows = seg_table["rows"]
    psi = np.ones(pm.N_PSI)
    if eq15:
        psi[7], psi[8] = eq15["h2d"]["B_eff"], eq15["h2d"]["tau_s"]
        psi[9], psi[10] = eq15["d2h"]["B_eff"], eq15["d2h"]["tau_s"]
    else:
        psi[7], psi[8], psi[9], psi[10] = 2.0e11, 4e-6, 2.0e11, 4e-6
    psi[11] = seg_table["tau_sync_s"]

    def fit(rows_, psi_):
        p = psi_.copy()
        comp = [r for r in rows_ if r["cls"] == pm.PM_SEG_COMPUTE and r["precision"] == pm.PM_BF16]
        for c in (0, 2, 3):
            rc = [r for r in rows_ if r["cls"] == c]
            if rc:
                p[c] = _fit_1d(rc, theta, p, n_sm, c)
        if comp:
            p[1] = _fit_1d(comp, theta, p, n_sm, 1)
        for prec in (pm.PM_FP32, pm.PM_FP8E4M3):
            rp = [r for r in rows_ if r["cls"] == pm.PM_SEG_COMPUTE and r["precision"] == prec]
            if rp:
                p[4 + prec] = _fit_1d(rp, theta, p, n_sm, 4 + prec)
        return p

    psi = fit(rows, psi)
    t = np.array([r["t"] for r in rows])
    pred = _seg_predict(rows, theta, psi, n_sm)
    ape = np.abs(pred - t) / t * 100.0
    # leave-one-out: refit without each row, predict it
    loo = np.zeros(len(rows))
    for i in range(len(rows)):
        p_i = fit(rows[:i] + rows[i + 1:], psi)
        loo[i] = abs(_seg_predict([rows[i]], theta, p_i, n_sm)[0] - t[i]) / t[i] * 100.0
    by_class = {}
    for c, name in enumerate(SEG_CLASS_NAMES):
        m = np.array([r["cls"] == c for r in rows])
        if m.any():
            by_class[name] = dict(n=int(m.sum()), mae_pct=float(ape[m].mean()), loo_mae_pct=float(loo[m].mean()))
    extra = {}
    for name, sel in (("multi_kernel", lambda r: r["kernels"] > 1), ("host_transfers", lambda r: r["h2d_bytes"] > 0)):
        m = np.array([sel(r) for r in rows])
        if m.any():
            extra[name] = dict(n=int(m.sum()), mae_pct=float(ape[m].mean()), loo_mae_pct=float(loo[m].mean()))
    interference = fit_stream_interference(streams or {}, theta, psi, n_sm)
    psi = np.array(interference["psi"])
    return dict(psi=psi.tolist(), by_class=by_class, by_feature=extra, all=dict(
        n=len(rows), mae_pct=float(ape.mean()), loo_mae_pct=float(loo.mean())),
        rows=[dict(name=r["name"], t=r["t"], pred=float(pp)) for r, pp in zip(rows, pred)],
        streams=interference)


def main():
    import argparse
    ap = argparse.ArgumentParser(description="measure the calibration table and fit the stage model")
    ap.add_argument("--measure", action="store_true")
    ap.add_argument("--measure-instr", action="store_true", help="re-measure only the instruction/host probes")
    ap.add_argument("--measure-tmem-b", action="store_true", help="re-measure only the strategy-B GEMM rows")
    ap.add_argument("--measure-streams", action="store_true", help="re-measure only the concurrent-stream probes")
    ap.add_argument("--measure-segments", action="store_true", help="re-measure only the generic-path segments")
    ap.add_argument("--measure-grouped", action="store_true", help="re-measure only the grouped launches")
    ap.add_argument("--reading", type=int, default=pm.PM_READING_MEASURED,
                    help="0: literal equations; 1: readings measured on the kernels (default)")
    ap.add_argument("--sweep", default=SWEEP_PATH)
    ap.add_argument("--out", default=None, help="theta file (default: theta_gb300.json, or _literal for reading 0)")
    ap.add_argument("--report", default=None, help="report file (default: data/calib_report_gb300.json, or _literal)")
    ap.add_argument("--shapes", default="1024,2048,4096,8192,16384")
    args = ap.parse_args()
    if args.out is None:
        args.out = theta_path(args.reading)
    if args.report is None:
        args.report = report_path(args.reading)
    n_sm = pm.sm_count()
    pm.pm_model_set_reading(args.reading)
    if args.measure:
        table = measure_sweep(tuple(int(s) for s in args.shapes.split(",")))
        os.makedirs(os.path.dirname(args.sweep), exist_ok=True)
        with open(args.sweep, "w") as f:
            json.dump(table, f)
    with open(args.sweep) as f:
        table = json.load(f)
    if args.measure_instr:
        table["instr"] = measure_instructions()
    if args.measure_tmem_b:
        settle()
        table["rows"] = [r for r in table["rows"] if not r.get("tmem_a", 0)] + \
            measure_tmem_b(tuple(int(s) for s in args.shapes.split(",")))
    if args.measure_streams:
        table["streams"] = measure_streams()
    if args.measure_segments:
        settle()
        table["segments"] = measure_segments(table)
    if args.measure_grouped:
        settle()
        table["grouped"] = measure_grouped(grouped_theta(n_sm, table), n_sm)
    if (args.measure_instr or args.measure_tmem_b or args.measure_streams or args.measure_segments or
            args.measure_grouped):
        with open(args.sweep, "w") as f:
            json.dump(table, f)
    rows = table["rows"]
    grouped = table.get("grouped", [])
    train, hold = split(len(rows))
    gtrain, ghold = split(len(grouped)) if grouped else (np.zeros(0, bool), np.zeros(0, bool))
    th_paper = prior_theta(n_sm, reading=args.reading)
    th0 = probe_priors(table["instr"], n_sm, reading=args.reading) if "instr" in table else th_paper
    obj = GpuObjective([r for r, m in zip(rows, train) if m], n_sm, [r for r, m in zip(grouped, gtrain) if m])
    theta, trace = fit(obj, th0, reg=FIT_REG, log=print)
    allobj = GpuObjective(rows, n_sm, grouped)
    # every measured row (configurations, then grouped launches) with its prediction
    all_rows = rows + grouped
    hold_all = np.concatenate([hold, ghold])
    train_all = np.concatenate([train, gtrain])

    def predict_all(th):
        return np.concatenate([allobj.predict(th), allobj.predict_grouped(th) if grouped else np.zeros(0)])

    pred0, pred_all = predict_all(th0), predict_all(theta)
    pred = pred_all[:len(rows)]
    rep = dict(reading=args.reading, n_rows=len(all_rows), n_train=int(train_all.sum()),
               n_holdout=int(hold_all.sum()),
               loss_trace=[float(x) for x in trace], theta=theta.tolist(), prior=th0.tolist(),
               environment=environment(), two_sm=two_sm_report(rows),
               per_config=[dict(family=family_of(r), cfg=[r.get(f, 0) for f in FIELDS], t=r["t"], pred=float(p),
                                holdout=bool(h)) for r, p, h in zip(rows, pred, hold)],
               per_grouped=[dict(G=r["G"], seed=r["seed"], N=r["N"], launch=r["launch"], t=r["t"], pred=float(p),
                                 holdout=bool(h)) for r, p, h in zip(grouped, pred_all[len(rows):], ghold)],
               mae_paper_prior=mae_by_family(all_rows, predict_all(th_paper)),
               mae_prior=mae_by_family(all_rows, pred0), mae_train=mae_by_family(all_rows, pred_all, train_all),
               mae_holdout=mae_by_family(all_rows, pred_all, hold_all), mae_all=mae_by_family(all_rows, pred_all),
               grouped_autotune=grouped_autotune_report(grouped, theta, n_sm) if grouped else [],
               roofline_mae=roofline_mae(rows, dict(hbm=8.0e12, bf16=2.25e15, fp8=4.5e15, tf32=1.1e15)),
               autotune=autotune_vs_best(rows, theta, n_sm), pchase=table.get("pchase"),
               instr=table.get("instr"), tmem_strategy=tmem_strategy_report(rows, pred),
               streams=table.get("streams"))
    if table.get("pchase"):
        props = torch.cuda.get_device_properties(0)
        rep["pchase_levels"] = pchase_levels(table["pchase"],
                                             getattr(props, "shared_memory_per_multiprocessor", 0) or 256 * 1024,
                                             getattr(props, "L2_cache_size", 0) or 128 * 2 ** 20)
    if table.get("segments"):
        # the generic path's roofline uses the measured peak rates (instruction
        # probe), not the stage model's fitted per-step rates
        theta_generic = theta.copy()
        theta_generic[6:9] = th0[6:9]
        rep["segments"] = fit_segments(table["segments"], theta_generic, n_sm, (table.get("instr") or {}).get("eq15"),
                                       table.get("streams"))
        rep["segments"]["theta"] = theta_generic.tolist()
        rep["grouped_segments"] = grouped_family(table["segments"], theta, n_sm)
    meta = dict(device=table.get("device"), n_sm=n_sm, fitted_on=os.path.basename(args.sweep),
                reading=args.reading, mae_holdout=rep["mae_holdout"])
    if rep.get("segments"):
        meta["segment_psi"] = rep["segments"]["psi"]        # generic path: class scales, efficiencies, host link
        meta["segment_theta"] = rep["segments"]["theta"]    # theta with the probe-measured peak rates
    save_theta(theta, meta, args.out)
    if args.report:
        with open(args.report, "w") as f:
            json.dump(rep, f, indent=1)
    print(json.dumps({k: rep[k] for k in ("mae_paper_prior", "mae_prior", "mae_holdout", "mae_all", "roofline_mae")},
                     indent=1))
    if rep.get("instr"):
        print(json.dumps({k: v for k, v in rep["instr"].items() if k not in ("host",)}, indent=1))
    for a in rep["autotune"]:
        print("autotune %(M)d dt=%(dtype)d pick=%(pick)s best=%(best)s pick/best=%(pick_over_best).3f "
              "TFLOP/s pick %(tflops_pick).0f best %(tflops_best).0f" % a)
    if rep.get("pchase_levels"):
        pl = rep["pchase_levels"]
        print("pointer chase levels: L1 %s ns, L2 %s ns, DRAM %s ns (capacities %.0f KB, %.0f MB)" % (
            pl["l1_ns"], pl["l2_ns"], pl["dram_ns"], pl["l1_bytes"] / 1024, pl["l2_bytes"] / 2 ** 20))
    for a in rep["grouped_autotune"]:
        print("grouped autotune G=%(G)d N=K=%(N)d pick=%(pick_launch)s best=%(best_launch)s pick/best=%(pick_over_best)s"
              % a)
    if rep.get("segments"):
        sg = rep["segments"]
        print("generic path psi %s" % ["%.3g" % v for v in sg["psi"]])
        for name, v in list(sg["by_class"].items()) + list(sg["by_feature"].items()):
            print("segments %-14s n=%2d MAE %.1f %% (leave-one-out %.1f %%)" % (name, v["n"], v["mae_pct"],
                                                                            v["loo_mae_pct"]))
    for name, v in (rep.get("streams") or {}).items():
        print("streams %s: T(N_c) %s s, tau_c %.3g s (%.2f T1), additive-law MAE %.1f %%" % (
            name, ["%.3g" % x for x in v["t_s"]], v["fit"]["tau_c_s"], v["fit"]["tau_over_T1"], v["fit"]["mae_pct"]))
    si = (rep.get("segments") or {}).get("streams") or {}
    if si.get("classes"):
        print("generic path, concurrent streams: kappa_launch %.3g, kappa_memory %.3g, kappa_compute %.3g" % (
            si["kappa_launch"], si["kappa_memory"], si["kappa_compute"]))
        for name, v in si["classes"].items():
            print("  %s: predicted T(N_c) %s s, MAE %.1f %% (single stream %.1f %%)" % (
                name, ["%.3g" % x for x in v["pred_s"]], v["mae_pct"], v["single_stream_ape_pct"]))
    for r in rep["tmem_strategy"]:
        print("TMEM strategy %d dt=%d: best A %s %.3g s, best B %s %.3g s, measured B/A %.3f, predicted %.3f" % (
            r["M"], r["dtype"], r["A"]["tile"], r["A"]["t"], r["B"]["tile"], r["B"]["t"], r["measured_B_over_A"],
            r["predicted_B_over_A"]))


if __name__ == "__main__":
    main()
