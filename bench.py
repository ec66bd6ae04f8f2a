"""Benchmark of the GB300 hot path of the stage-centric performance model
(arxiv 2605.04178): the model-autotuned BF16 GEMM C = A.B at M = N = K = 8192.

One step = one launch of the tcgen05 GEMM in the tile configuration the
model's GPU autotuner picked for this shape (the pick is made once, before
timing).  `value` is whole-job TFLOP/s (2MNK per step per GPU) with the
operands already in HBM; `e2e` is the same metric through the public C-ABI
calls from pinned host FP32 buffers (H2D of A and B, operand preparation,
GEMM, D2H of C inside the timed region).  Secondary figures on the same line:
the HBM probes, the batched model and its adjoint, and the autotuner.

--impl reference times the CPU FP64 oracle (the reference of this build) on a
bounded row sample of the same GEMM, on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "model MAE % vs measured; autotuned GEMM TFLOP/s % of peak vs exhaustive best"
M = N = K = 8192
SEED = 2


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, dist=None, device: str = "cpu") -> float:
    """The largest of one value per rank (the job's time is its slowest replica)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, seconds: float, world: int, dist=None, device: str = "cpu"):
    """Whole-job rate of independent replicas: every rank does units_per_rank
    in its own time; the job takes the slowest rank's time (max over ranks)
    and does world x units.  Returns (rate in units/s, max seconds)."""
    t = max_over_ranks(seconds, dist, device)
    return world * units_per_rank / t, t


def _measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """Clock and throttle record of a timed region, read through the
    library's read-only NVML query (pm_clock_sample): one sample right before
    the region starts and one right after it has completed (mark()), and a
    poll every `period_s` in between, so even a region of a few milliseconds
    carries at least two samples."""

    def __init__(self, pm, period_s: float = 0.01):
        self.pm = pm
        self.period = period_s
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _poll(self):
        while not self._stop.is_set():
            c = self.pm.pm_clock_sample()
            if c is not None:
                self.samples.append(c)
            self._stop.wait(self.period)

    def start(self):
        self._t = threading.Thread(target=self._poll, daemon=True)
        self._t.start()

    def mark(self):
        c = self.pm.pm_clock_sample()
        if c is not None:
            self.samples.append(c)
        return c

    def stop(self):
        self._stop.set()
        if self._t is not None:
            self._t.join(timeout=2)

    def summary(self, begin=None, end=None):
        """Median SM clock, the maximum SM clock, the reasons seen and the
        largest power draw over the samples between the begin and end marks
        (all samples if either mark is missing)."""
        sel = list(self.samples)
        if begin is not None and end is not None:
            sel = [c for c in sel if begin["host_time_s"] <= c["host_time_s"] <= end["host_time_s"]]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "source": "NVML unavailable"}
        reasons = sorted(set(r for c in sel for r in c["reasons"]) - {"gpu_idle"})
        return {"sm_mhz": statistics.median(c["sm_mhz"] for c in sel), "sm_max_mhz": max(c["sm_max_mhz"] for c in sel),
                "sm_mhz_begin": sel[0]["sm_mhz"], "sm_mhz_end": sel[-1]["sm_mhz"],
                "power_w_max": max(c["power_w"] for c in sel), "reasons": reasons, "samples": len(sel),
                "source": "NVML read-only queries through pm_clock_sample: marks before and after the timed region, "
                          "%.0f ms poll between" % (self.period * 1e3)}


BURST_LIMIT_S = 1.0


def roofline_peak(peaks: dict, timed_s: float):
    """The measured bf16 peak that matches a timed region: cuBLAS's burst
    figure for a region shorter than BURST_LIMIT_S (the clock has not yet
    settled under the power cap), its sustained 4 s figure for longer ones."""
    burst = float(peaks.get("bf16_tflops", 1900.0))
    sustained = float(peaks.get("bf16_tflops_sustained", 1700.0))
    return (burst, "burst") if timed_s < BURST_LIMIT_S else (sustained, "sustained")


def _cpu_gemm_rate(A, B, rows_per_step: int, steps: int, warmup: int, keep: bool = True):
    """Oracle FP64 GEMM on sampled rows; returns (TFLOP/s, seconds, rows, the rows computed or None
    when keep is False: a long reference run would otherwise hold every step's rows)."""
    import numpy as np

    import oracle as O
    import synthetic as S
    Mr = A.shape[0]
    for i in range(warmup):
        O.gemm_f64(A[(i * rows_per_step) % Mr:(i * rows_per_step) % Mr + rows_per_step], B)
    t0 = time.perf_counter()
    out = []
    for i in range(steps):
        r0 = (i * rows_per_step) % (Mr - rows_per_step + 1)
        c = O.gemm_f64(A[r0:r0 + rows_per_step], B)
        if keep:
            out.append(c)
    dt = time.perf_counter() - t0
    flops = 2.0 * rows_per_step * B.shape[0] * B.shape[1] * steps
    return flops / dt / 1e12, dt, rows_per_step * steps, (np.concatenate(out) if keep else None)


def _omp_threads(n=None):
    """Sets (when n is given) and returns the OpenMP thread count of the
    oracle's runtime (libgomp); None when libgomp cannot be loaded.  The
    torch.distributed launcher exports OMP_NUM_THREADS=1 to every rank, which
    would leave the one working rank of the reference arm on one core."""
    import ctypes
    try:
        gomp = ctypes.CDLL("libgomp.so.1")
    except OSError:
        return None
    if n is not None:
        gomp.omp_set_num_threads(int(n))
    return int(gomp.omp_get_max_threads())


def run_reference(args):
    rank, world, _ = _dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            dist.destroy_process_group()
            return
    import numpy as np

    import oracle as O
    import synthetic as S
    O.build()
    rows_per_step = 8
    n_rows = rows_per_step * 64
    B = S.matrix(SEED, K, N, "normal", M * K)
    A = S.matrix(SEED, n_rows, K, "normal", 0)          # the first n_rows rows of A
    threads = _omp_threads(os.cpu_count() or 1)
    tflops, dt, rows, _ = _cpu_gemm_rate(A, B, rows_per_step, args.steps, args.warmup, keep=False)
    cores = threads or os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": tflops, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        # the GPU arm's workload, computed by the oracle on a row sample of the same operands
        "config": {"workload": "bf16_gemm_8192^3_model_autotuned", "M": M, "N": N, "K": K,
                   "inputs": "A,B ~ N(0,1) seed 2 (the same FP32 matrices), FP64 arithmetic",
                   "rows_per_step": rows_per_step, "parallelism": "single"},
        "cpu_baseline": {"value": tflops, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": "%d rows x 8192 x 8192 FP64 per step (C = A.B definition, OpenMP)" % rows_per_step,
                         "cpu_model": _cpu_model()},
        "e2e": {"value": tflops, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line))
    sys.stdout.flush()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def run_gpu(args):
    import numpy as np
    import torch

    rank, world, local = _dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2605_04178_gb300 import build as B_
    B_.build()
    import paper_2605_04178_gb300 as pm
    import synthetic as S
    from paper_2605_04178_gb300.calibrate import prior_theta

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    peaks, peak_src = _measured_peaks()
    n_sm = pm.sm_count()
    theta = prior_theta(n_sm).astype(np.float32).astype(np.float64)
    calib = os.path.join(ROOT, "paper_2605_04178_gb300", "theta_gb300.json")
    theta_src = "prior"
    if os.path.exists(calib):
        with open(calib) as f:
            theta = np.array(json.load(f)["theta"], dtype=np.float64)
        theta_src = "calibrated"
    stream = torch.cuda.current_stream()

    # ------------------------------------------------------------- operands
    A_h = S.matrix(SEED, M, K, "normal", 0)
    B_h = S.matrix(SEED, K, N, "normal", M * K)
    A_pin = torch.from_numpy(A_h).pin_memory()
    B_pin = torch.from_numpy(B_h).pin_memory()
    A_d, B_d = A_pin.cuda(), B_pin.cuda()
    ops = pm.GemmOperands(pm.PM_BF16, M, N, K)
    ops.prepare(A_d, B_d)
    C = torch.empty(M, N, dtype=torch.float32, device="cuda")
    flops = 2.0 * M * N * K

    # ------------------------------------------------------ model-driven pick
    # the model alone (argmin over the 180-point space, on the GPU) and the
    # library's autotuner (the model's 8 best tiles timed on the device)
    MNK = torch.tensor([M, N, K], dtype=torch.int32, device="cuda")
    picks = torch.empty(24, dtype=torch.uint8, device="cuda")
    t_pred = torch.empty(1, dtype=torch.float32, device="cuda")
    pm.pm_autotune_pick(MNK, 1, pm.PM_BF16, theta, n_sm, picks, t_pred)
    p = picks.cpu().numpy().view(pm.CFG_DTYPE)[0]
    model_pick = tuple(int(p[k]) for k in ("BM", "BN", "BK", "stages", "cta_group"))
    if args.cfg:
        pick = tuple(int(v) for v in args.cfg.split(","))
    else:
        tuned, _ = pm.pm_gemm_autotune(pm.cfg(M, N, K, dtype=pm.PM_BF16), 8, theta, n_sm, ops.A_op, ops.B_op, C,
                                       ops.scales)
        pick = (tuned.BM, tuned.BN, tuned.BK, tuned.stages, tuned.cta_group)
    cfg = pm.cfg(M, N, K, *pick, dtype=pm.PM_BF16)


    # ------------------------------------------------- device-resident steps
    clocks = ClockSampler(pm)
    clocks.start()
    for _ in range(args.warmup):
        ops.run(cfg, C)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
    barrier()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    mark0 = clocks.mark()
    start.record(stream)
    for i in range(args.steps):
        ev[2 * i].record(stream)
        ops.run(cfg, C)
        ev[2 * i + 1].record(stream)
    end.record(stream)
    barrier()
    mark1 = clocks.mark()
    clocks.stop()
    ms_total = start.elapsed_time(end)
    per_launch = [ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(args.steps)]
    rate, t_max = replica_throughput(flops * args.steps, ms_total * 1e-3, world, dist, "cuda")
    ms_total = t_max * 1e3
    ms_step = ms_total / args.steps
    value = rate / 1e12
    kern_ms = statistics.mean(per_launch)
    achieved = flops / (kern_ms * 1e-3) / 1e12
    # a short timed region is a burst (clock not yet capped): cuBLAS's burst
    # figure is its peak; seconds of back-to-back launches run under the power
    # cap, where cuBLAS's sustained figure is the peak.  Both fractions are
    # reported; frac is the one that matches the region's length.
    peak, peak_kind = roofline_peak(peaks, ms_total * 1e-3)
    peak_burst = float(peaks.get("bf16_tflops", 1900.0))
    peak_sustained = float(peaks.get("bf16_tflops_sustained", 1700.0))
    C_h = C.cpu().numpy()

    # ------------------------------------------------------ end-to-end steps
    C_pin = torch.empty(M, N, dtype=torch.float32).pin_memory()
    e2e_steps = max(3, min(100, args.steps // 50))

    ws_host = torch.empty(pm.pm_gemm_host_workspace(cfg, args.e2e_chunks), dtype=torch.uint8, device="cuda")

    def e2e_step():
        # one public call: pinned host FP32 A, B in, host FP32 C out, the host
        # link overlapped with conversion and GEMM in row chunks
        pm.pm_gemm_host(cfg, A_pin, B_pin, C_pin, ws_host, chunks=args.e2e_chunks)
        torch.cuda.current_stream().synchronize()

    for _ in range(2):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    barrier()
    e2e_rate, e2e_s = replica_throughput(flops * e2e_steps, time.perf_counter() - t0, world, dist, "cuda")
    e2e_value = e2e_rate / 1e12

    # exhaustive search at this shape (every valid BF16 tile, same protocol for
    # all, including the model's pick) and the model's error on those times
    exhaustive = None
    if not args.skip_exhaustive:
        import synthetic as S_
        meas = {}
        for t in S_.tile_space(pm.PM_BF16):
            try:
                r = ops.bench(pm.cfg(M, N, K, *t, dtype=pm.PM_BF16), C, warmup=3, reps=15)
            except pm.PMError as e:
                if e.status == pm.PM_EUNSUPPORTED:
                    continue
                raise
            meas[t] = r["median_s"]
        tiles = sorted(meas)
        cols = {f: np.array(v) for f, v in zip(("BM", "BN", "BK", "stages", "cta_group"), zip(*tiles))}
        cols.update(M=np.full(len(tiles), M), N=np.full(len(tiles), N), K=np.full(len(tiles), K),
                    dtype=np.full(len(tiles), pm.PM_BF16), kind=np.zeros(len(tiles)))
        pred = torch.empty(len(tiles), dtype=torch.float32, device="cuda")
        pm.pm_model_predict(pm.cfg_tensor(cols), len(tiles), theta, n_sm, pred)
        pred = pred.cpu().numpy().astype(np.float64)
        tm = np.array([meas[t] for t in tiles])
        best = min(meas, key=meas.get)
        exhaustive = {"configs": len(meas), "best_tile": dict(zip(("BM", "BN", "BK", "stages", "cta_group"), best)),
                      "best_tflops": flops / meas[best] / 1e12, "pick_tflops": flops / meas[pick] / 1e12,
                      "pick_over_best_time": meas[pick] / meas[best],
                      "model_only_tile": dict(zip(("BM", "BN", "BK", "stages", "cta_group"), model_pick)),
                      "model_only_over_best_time": meas[model_pick] / meas[best],
                      "model_mae_pct": float(np.mean(np.abs(pred - tm) / tm) * 100.0),
                      "protocol": "3 warm-ups, median of 15 CUDA-event timed launches per tile"}
        # the same under the literal equations with their own calibration
        calib_l = os.path.join(ROOT, "paper_2605_04178_gb300", "theta_gb300_literal.json")
        if os.path.exists(calib_l):
            with open(calib_l) as f:
                theta_l = np.array(json.load(f)["theta"], dtype=np.float64)
            pred_m = torch.empty(len(tiles), dtype=torch.float32, device="cuda")
            pm.pm_model_set_reading(pm.PM_READING_LITERAL)
            try:
                pm.pm_autotune_pick(MNK, 1, pm.PM_BF16, theta_l, n_sm, picks, t_pred)
                pm.pm_model_predict(pm.cfg_tensor(cols), len(tiles), theta_l, n_sm, pred_m)
                torch.cuda.synchronize()
            finally:
                pm.pm_model_set_reading(pm.PM_READING_MEASURED)
            pq = picks.cpu().numpy().view(pm.CFG_DTYPE)[0]
            mp = tuple(int(pq[k]) for k in ("BM", "BN", "BK", "stages", "cta_group"))
            pm_np = pred_m.cpu().numpy().astype(np.float64)
            exhaustive["literal_reading"] = {
                "model_only_tile": dict(zip(("BM", "BN", "BK", "stages", "cta_group"), mp)),
                "model_only_over_best_time": meas[mp] / meas[best] if mp in meas else None,
                "model_mae_pct": float(np.mean(np.abs(pm_np - tm) / tm) * 100.0)}
        # TMEM strategy B (A operand copied into tensor memory) over its tile
        # space at the same shape: fastest of each strategy, measured and predicted
        measB = {}
        for t in S_.tile_space(pm.PM_BF16):
            try:
                r = ops.bench(pm.cfg(M, N, K, *t, dtype=pm.PM_BF16, tmem_a=1), C, warmup=3, reps=15)
            except pm.PMError as e:
                if e.status == pm.PM_EUNSUPPORTED:
                    continue
                raise
            measB[t] = r["median_s"]
        tilesB = sorted(measB)
        colsB = {f: np.array(v) for f, v in zip(("BM", "BN", "BK", "stages", "cta_group"), zip(*tilesB))}
        colsB.update(M=np.full(len(tilesB), M), N=np.full(len(tilesB), N), K=np.full(len(tilesB), K),
                     dtype=np.full(len(tilesB), pm.PM_BF16), kind=np.zeros(len(tilesB)),
                     tmem_a=np.ones(len(tilesB)))
        predB = torch.empty(len(tilesB), dtype=torch.float32, device="cuda")
        pm.pm_model_predict(pm.cfg_tensor(colsB), len(tilesB), theta, n_sm, predB)
        predB = predB.cpu().numpy().astype(np.float64)
        tB = np.array([measB[t] for t in tilesB])
        bestB = min(measB, key=measB.get)
        iA, iB = tiles.index(best), tilesB.index(bestB)
        same = [t for t in tilesB if t in meas]
        exhaustive["tmem_strategy_b"] = {
            "configs": len(measB), "best_tile": dict(zip(("BM", "BN", "BK", "stages", "cta_group"), bestB)),
            "best_tflops": flops / measB[bestB] / 1e12, "measured_best_B_over_best_A": measB[bestB] / meas[best],
            "predicted_best_B_over_best_A": predB[iB] / pred[iA],
            "median_B_over_A_same_tile": float(np.median([measB[t] / meas[t] for t in same])),
            "model_mae_pct": float(np.mean(np.abs(predB - tB) / tB) * 100.0)}

    extra = {}
    if not args.skip_extra:
        extra = secondary(pm, S, theta, n_sm, peaks)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "bf16_gemm_8192^3_model_autotuned", "M": M, "N": N, "K": K,
                       "inputs": "A,B ~ N(0,1) seed 2, FP32 -> BF16 K-major operands",
                       "tile": dict(zip(("BM", "BN", "BK", "stages", "cta_group"), pick)),
                       "autotune": ("tile given by --cfg" if args.cfg else
                                    "model top-8 tiles (GPU) timed on the device, fastest kept"),
                       "theta": theta_src, "l2": "operands 256 MB > 129 MB L2, no flush",
                       "parallelism": "replicas" if world > 1 else "single"},
            "pct_of_peak": 100.0 * achieved / peak,
            "pct_of_datasheet_dense_bf16": 100.0 * achieved / 2250.0,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "peak_source": "%s bf16 %s (%s); chosen by the timed region's length (%.3f s; burst below "
                                        "%.1f s)" % (peak_src, peak_kind,
                                                     "cuBLAS 8192^3 best of 10" if peak_kind == "burst" else
                                                     "cuBLAS 8192^3 back to back for 4 s", ms_total * 1e-3,
                                                     BURST_LIMIT_S),
                         "peak_burst": peak_burst, "frac_vs_burst": achieved / peak_burst,
                         "peak_sustained": peak_sustained, "frac_vs_sustained": achieved / peak_sustained,
                         "kernel": "gemm_kernel<1 or 2, bf16>", "kernel_ms": kern_ms},
            "e2e": {"value": e2e_value, "unit": "TFLOP/s", "h2d_bytes_per_step": 4 * (M * K + K * N),
                    "d2h_bytes_per_step": 4 * M * N, "call": "pm_gemm_host, %d row chunks" % args.e2e_chunks,
                    "ms_per_step": 1e3 * e2e_s / e2e_steps},
            "gpu_launches": args.steps,
            "clocks": clocks.summary(mark0, mark1),
        }
        if exhaustive is not None:
            line["exhaustive"] = exhaustive
            line["vs_exhaustive_best"] = 1.0 / exhaustive["pick_over_best_time"]
            # the model's own argmin (no timing) against the exhaustive best,
            # beside the timed shortlist's pick
            line["model_only_over_best_time"] = exhaustive["model_only_over_best_time"]
            line["shortlist_over_best_time"] = exhaustive["pick_over_best_time"]
        calib_rep = os.path.join(ROOT, "paper_2605_04178_gb300", "data", "calib_report_gb300.json")
        if theta_src == "calibrated" and os.path.exists(calib_rep):
            with open(calib_rep) as f:
                rep = json.load(f)
            line["model_mae_pct_holdout"] = {k: round(v["mae_pct"], 2) for k, v in rep["mae_holdout"].items()}
        calib_lit = os.path.join(ROOT, "paper_2605_04178_gb300", "data", "calib_report_gb300_literal.json")
        if os.path.exists(calib_lit):
            with open(calib_lit) as f:
                rep = json.load(f)
            line["model_mae_pct_holdout_literal_reading"] = {k: round(v["mae_pct"], 2)
                                                             for k, v in rep["mae_holdout"].items()}
        line.update(extra)
        if not args.skip_cpu and world == 1:
            # the oracle on the host cores (one GPU only): rows 0..47 of the same
            # product, which also gives the GPU result's error on those rows
            threads = _omp_threads(os.cpu_count() or 1)
            tfl, dt, rows, ref = _cpu_gemm_rate(A_h[:64], B_h, 8, 6, 1)
            err = float(np.linalg.norm(C_h[:48] - ref) / np.linalg.norm(ref))
            line["cpu_baseline"] = {"value": tfl, "unit": "TFLOP/s", "cores": threads or os.cpu_count(),
                                    "kind": "oracle",
                                    "sample": "6 x 8 rows of the 8192^3 GEMM in FP64 (%.1f s)" % dt,
                                    "cpu_model": _cpu_model()}
            line["bf16_rel_frobenius_error_rows0_47"] = err
            line["cpu_baseline"]["per_config"] = _cpu_per_config()
        line["roofline"]["traffic"] = _traffic_from_profile(pick)
        print(json.dumps(line))
        sys.stdout.flush()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def _cpu_per_config() -> dict:
    """The oracle, as it stands, timed on the host cores on a bounded sample of
    each workload the bench reports on the GPU (a few seconds in all)."""
    import ctypes

    import numpy as np

    import oracle as O
    import synthetic as S

    def best(fn, reps=3):
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        return min(ts)

    out = {}
    # FP64 GEMM 512^3 (the definition), all host cores and one thread
    A, B = S.gemm_operands(512, 512, 512, seed=0)
    O.gemm_f64(A, B)
    t_all = best(lambda: O.gemm_f64(A, B))
    c1 = {"GFLOPps_all_cores": 2 * 512 ** 3 / t_all / 1e9, "ms_all_cores": t_all * 1e3}
    try:
        gomp = ctypes.CDLL("libgomp.so.1")
        gomp.omp_set_num_threads(1)
        try:
            t_one = best(lambda: O.gemm_f64(A, B), 1)
        finally:
            gomp.omp_set_num_threads(os.cpu_count() or 1)
        c1.update(GFLOPps_one_thread=2 * 512 ** 3 / t_one / 1e9, ms_one_thread=t_one * 1e3)
    except OSError:
        pass
    out["fp64_gemm_512"] = c1
    # triad (one rounding, one thread) and copy over 2^26 FP32
    n = 2 ** 26
    b = S.uniform_pm1(1, n)
    c = S.uniform_pm1(1, n, offset=n)
    t_tr = best(lambda: O.triad_f32(b, c, 3.0))
    dst = np.empty_like(b)
    t_cp = best(lambda: np.copyto(dst, b))
    out["stream_2pow26"] = {"n": n, "triad_GBps_one_thread": 12.0 * n / t_tr / 1e9,
                              "copy_GBps": 8.0 * n / t_cp / 1e9}
    # pointer chase over 256 MB, 2^20 dependent loads
    nodes = (256 << 20) // 64
    buf = S.pchase_buffer(nodes, seed=1)
    hops = 2 ** 20
    t_pc = best(lambda: O.pchase(buf, 16, 0, hops), 2)
    out["pchase_256MB"] = {"ns_per_hop": t_pc / hops * 1e9}
    del b, c, dst, buf
    # per-group sampled rows of the 64-group grouped GEMM (8 groups x 8 rows, N = K = 4096)
    Bg = S.matrix(3, 4096, 4096, "normal", 0)
    Ag = S.matrix(3, 8, 4096, "normal", 4096 * 4096)
    t_g = best(lambda: [O.gemm_f64(Ag, Bg) for _ in range(8)], 2)
    out["grouped_rows"] = {"GFLOPps": 8 * 2 * 8 * 4096 * 4096 / t_g / 1e9, "sample": "8 groups x 8 rows"}
    # FP64 model with its dual-number gradient over 2e5 configurations
    nc = 200000
    cf = S.model_config_batch(nc, seed=4)
    cf["kind"] = np.zeros(nc, dtype=np.int32)
    th = O.prior_theta(152)
    t_m = best(lambda: O.model_batch(cf, th, 152), 2)
    t_mg = best(lambda: O.model_batch(cf, th, 152, grad=True), 2)
    out["model_2e5"] = {"forward_Mcfg_per_s": nc / t_m / 1e6, "forward_grad_Mcfg_per_s": nc / t_mg / 1e6,
                            "sample": "%d configurations" % nc}
    return out


def _cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (model name, else implementer/part)."""
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
    except OSError:
        return platform.machine()
    for key in ("model name", "Model", "CPU part"):
        for line in info.splitlines():
            if line.startswith(key) and ":" in line:
                return "%s %s" % (platform.machine(), line.split(":", 1)[1].strip())
    return platform.machine()


def _kernel_source_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("pm_gemm.cu", "pm_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2605_04178_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic_from_profile(pick):
    """DRAM bytes per launch from the committed ncu summary of this tile, if the
    kernel source has not changed since that capture (else None)."""
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "gemm_kernel_bf16_8192_*.md"))):
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith(("#", "|", " ")):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("tile") == ",".join(str(v) for v in pick) and kv.get("source_sha") == _kernel_source_sha():
            return float(kv["traffic_bytes"])
    return None


def secondary(pm, S, theta, n_sm, peaks):
    """HBM probes, batched model forward/adjoint and autotuner throughput."""
    import numpy as np
    import torch
    out = {}
    n = 2 ** 28
    a = torch.empty(n, dtype=torch.float32, device="cuda").uniform_(-1, 1)
    b = torch.empty_like(a)
    c = torch.empty_like(a).uniform_(-1, 1)
    r_copy = pm.pm_probe_run(pm.probe_args(pm.PM_PROBE_COPY, n=n), a, b, warmup=10, reps=50)
    r_triad = pm.pm_probe_run(pm.probe_args(pm.PM_PROBE_TRIAD, n=n, scalar=3.0), a, b, c, warmup=10, reps=50)
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    out["probes"] = {
        "copy_GBps": r_copy["bytes"] / r_copy["median_s"] / 1e9,
        "triad_GBps": r_triad["bytes"] / r_triad["median_s"] / 1e9,
        "n_elems": n, "hbm_peak_GBps": hbm,
    }
    out["probes"]["copy_frac"] = out["probes"]["copy_GBps"] / hbm
    out["probes"]["triad_frac"] = out["probes"]["triad_GBps"] / hbm
    # TMA 2D tile copy of a 1 GiB FP32 matrix (64 x 64 tiles): 2 GiB moved
    src = a[: 16384 * 16384].view(16384, 16384)
    dst = b[: 16384 * 16384].view(16384, 16384)
    r_tma = pm.pm_probe_run(pm.probe_args(pm.PM_PROBE_TMA2D, rows=16384, cols=16384, tile_r=64, tile_c=64),
                            src, dst, warmup=3, reps=20)
    out["probes"]["tma2d_64x64_GBps"] = r_tma["bytes"] / r_tma["median_s"] / 1e9
    out["probes"]["tma2d_frac"] = out["probes"]["tma2d_64x64_GBps"] / hbm
    del a, b, c, src, dst
    # pointer chase over a 256 MB working set (DRAM level), 64-byte node stride
    nodes = (256 << 20) // 64
    buf = torch.from_numpy(S.pchase_buffer(nodes, seed=1).view(np.int32)).cuda()
    res = torch.zeros(1, dtype=torch.int32, device="cuda")
    hops = 2 ** 18
    r_pc = pm.pm_probe_run(pm.probe_args(pm.PM_PROBE_PCHASE, n=nodes, hops=hops, start=0), buf, res, warmup=2, reps=3)
    out["probes"]["pchase_256MB_ns_per_hop"] = 1e9 * r_pc["median_s"] / hops
    del buf
    # FP32 (three-pass TF32) GEMM 512^3 in its fixed tile, and the
    # stage model's prediction for that launch (calibrated theta, measured reading)
    A1 = torch.from_numpy(S.matrix(0, 512, 512, "uniform", 0)).cuda()
    B1 = torch.from_numpy(S.matrix(0, 512, 512, "uniform", 512 * 512)).cuda()
    ops1 = pm.GemmOperands(pm.PM_FP32, 512, 512, 512)
    ops1.prepare(A1, B1)
    C1 = torch.empty(512, 512, dtype=torch.float32, device="cuda")
    c1 = pm.cfg(512, 512, 512, 128, 128, 32, 2, 1, dtype=pm.PM_FP32)
    r1 = ops1.bench(c1, C1, warmup=10, reps=100)
    p1 = torch.empty(1, dtype=torch.float32, device="cuda")
    pm.pm_model_predict(pm.cfg_tensor({k: np.array([v]) for k, v in dict(
        M=512, N=512, K=512, BM=128, BN=128, BK=32, stages=2, cta_group=1, dtype=0, kind=0).items()}),
        1, theta, n_sm, p1)
    out["fp32_gemm_512"] = {"workload": "fp32_gemm_512^3_128x128x32_s2_g1", "gpu_us": r1["median_s"] * 1e6,
                      "TFLOPps": 2 * 512 ** 3 / r1["median_s"] / 1e12, "model_pred_us": float(p1.item()) * 1e6,
                      "model_ape_pct": abs(float(p1.item()) - r1["median_s"]) / r1["median_s"] * 100}
    # the same launch under the literal equations with their own calibration
    calib_l = os.path.join(ROOT, "paper_2605_04178_gb300", "theta_gb300_literal.json")
    if os.path.exists(calib_l):
        with open(calib_l) as f:
            theta_l = np.array(json.load(f)["theta"], dtype=np.float64)
        pm.pm_model_set_reading(pm.PM_READING_LITERAL)
        try:
            pm.pm_model_predict(pm.cfg_tensor({k: np.array([v]) for k, v in dict(
                M=512, N=512, K=512, BM=128, BN=128, BK=32, stages=2, cta_group=1, dtype=0, kind=0).items()}),
                1, theta_l, n_sm, p1)
            torch.cuda.synchronize()
        finally:
            pm.pm_model_set_reading(pm.PM_READING_MEASURED)
        out["fp32_gemm_512"]["model_pred_us_literal_reading"] = float(p1.item()) * 1e6
        out["fp32_gemm_512"]["model_ape_pct_literal_reading"] = abs(float(p1.item()) - r1["median_s"]) / r1["median_s"] * 100
    del A1, B1, C1, ops1
    # batched model over 1e6 configurations: forward and adjoint
    nc = 10 ** 6
    cf = S.model_config_batch(nc, seed=4)
    cf["kind"] = np.zeros(nc, dtype=np.int32)
    dev = pm.cfg_tensor(cf)
    t_out = torch.empty(nc, dtype=torch.float32, device="cuda")
    tm = torch.ones(nc, dtype=torch.float32, device="cuda") * 1e-3
    ws = torch.empty(pm.pm_model_grad_workspace(nc) // 8, dtype=torch.float64, device="cuda")
    go = torch.empty(pm.N_GRAD_OUT, dtype=torch.float64, device="cuda")
    MNK = torch.from_numpy(np.stack([cf["M"], cf["N"], cf["K"]], 1)[: nc // 180].astype(np.int32).ravel()).cuda()
    picks = torch.empty((nc // 180) * 24, dtype=torch.uint8, device="cuda")
    tp = torch.empty(nc // 180, dtype=torch.float32, device="cuda")

    def timeit(fn, reps=50):
        for _ in range(5):
            fn()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(reps):
            fn()
        e.record()
        torch.cuda.synchronize()
        return s.elapsed_time(e) / reps * 1e-3

    t_f = timeit(lambda: pm.pm_model_predict(dev, nc, theta, n_sm, t_out))
    t_g = timeit(lambda: pm.pm_model_grad(dev, nc, theta, n_sm, tm, ws, go))
    t_a = timeit(lambda: pm.pm_autotune_pick(MNK, nc // 180, 1, theta, n_sm, picks, tp))
    # grouped GEMM: 64 problems, M_g log-uniform in [16, 4096] (seed 3), N = K = 4096, BF16,
    # tiles and launch from the grouped autotuner (the model's 4 best launches timed, fastest kept), one
    # persistent launch replayed from a CUDA graph
    Mg = S.grouped_m(64, 3)
    Ng = Kg = 4096
    t_model, _, _, model_launch = pm.pm_grouped_autotune(Mg, Ng, Kg, pm.PM_BF16, theta, n_sm)
    sum_m = int(Mg.sum())
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    A_g = torch.randn(sum_m, Kg, device="cuda", generator=gen).to(torch.bfloat16)
    B_g = torch.empty(64 * Ng, Kg, dtype=torch.bfloat16, device="cuda")
    for q in range(64):
        B_g[q * Ng:(q + 1) * Ng] = torch.randn(Ng, Kg, device="cuda", generator=gen).to(torch.bfloat16)
    C_g = torch.empty(sum_m, Ng, dtype=torch.float32, device="cuda")
    t_gp, gbm, gbn, glaunch, _ = pm.pm_grouped_gemm_autotune(Mg, Ng, Kg, theta, n_sm, 4, A_g, B_g, C_g,
                                                             warmup=2, reps=5)
    side = torch.cuda.Stream()
    pm.pm_grouped_gemm_run(Mg, Ng, Kg, gbm, gbn, *glaunch, A_g, B_g, C_g)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        pm.pm_grouped_gemm_run(Mg, Ng, Kg, gbm, gbn, *glaunch, A_g, B_g, C_g, stream=side)
    t_grp = timeit(graph.replay, reps=20)
    gflops = float(sum(2.0 * m * Ng * Kg for m in Mg))
    gbytes = float(sum(2.0 * (m * Kg + Ng * Kg) + 4.0 * m * Ng for m in Mg))
    out["grouped"] = {"groups": 64, "sum_M": sum_m, "N": Ng, "K": Kg, "launch": dict(zip(("BK", "stages", "cta_group"),
                                                                                          glaunch)),
                      "autotune": "model top-4 launches timed, fastest kept",
                      "model_only_launch": dict(zip(("BK", "stages", "cta_group"), model_launch)),
                      "ms": t_grp * 1e3, "TFLOPps": gflops / t_grp / 1e12, "GBps": gbytes / t_grp / 1e9,
                      "predicted_ms": t_gp * 1e3, "ape_pct": abs(t_gp - t_grp) / t_grp * 100,
                      "flop_frac": gflops / (float(peaks.get("bf16_tflops", 1900.0)) * 1e12) / t_grp,
                      "byte_frac": gbytes / (float(peaks.get("hbm_gbs", 6800.0)) * 1e9) / t_grp,
                      "roofline_frac": max(gflops / (float(peaks.get("bf16_tflops", 1900.0)) * 1e12),
                                           gbytes / (float(peaks.get("hbm_gbs", 6800.0)) * 1e9)) / t_grp}
    del A_g, B_g, C_g, graph
    # FP8 e4m3 GEMM 8192^3 (per-tensor scales from the amax pass), in the tile the
    # library's autotuner picks (the model's 8 best tiles timed), 20 timed launches;
    # its peak is the measured BF16 burst peak times the nominal FP8/BF16 ratio of 2
    n8 = 8192
    gen.manual_seed(2)
    A8 = torch.randn(n8, n8, device="cuda", generator=gen)
    B8 = torch.randn(n8, n8, device="cuda", generator=gen)
    ops8 = pm.GemmOperands(pm.PM_FP8E4M3, n8, n8, n8)
    ops8.prepare(A8, B8)
    del A8, B8
    C8 = torch.empty(n8, n8, dtype=torch.float32, device="cuda")
    tuned8, _ = pm.pm_gemm_autotune(pm.cfg(n8, n8, n8, dtype=pm.PM_FP8E4M3), 8, theta, n_sm, ops8.A_op, ops8.B_op,
                                    C8, ops8.scales)
    tile8 = (tuned8.BM, tuned8.BN, tuned8.BK, tuned8.stages, tuned8.cta_group)
    r8 = ops8.bench(pm.cfg(n8, n8, n8, *tile8, dtype=pm.PM_FP8E4M3), C8, warmup=5, reps=20)
    p8 = torch.empty(1, dtype=torch.float32, device="cuda")
    pm.pm_model_predict(pm.cfg_tensor({k: np.array([v]) for k, v in dict(
        M=n8, N=n8, K=n8, BM=tile8[0], BN=tile8[1], BK=tile8[2], stages=tile8[3], cta_group=tile8[4],
        dtype=pm.PM_FP8E4M3, kind=0).items()}), 1, theta, n_sm, p8)
    fp8_peak = 2.0 * float(peaks.get("bf16_tflops", 1900.0))
    tf8 = 2.0 * n8 ** 3 / r8["median_s"] / 1e12
    out["fp8_gemm_8192"] = {"workload": "fp8_e4m3_gemm_8192^3_model_autotuned",
                            "tile": dict(zip(("BM", "BN", "BK", "stages", "cta_group"), tile8)),
                            "autotune": "model top-8 tiles (GPU) timed on the device, fastest kept",
                            "ms": r8["median_s"] * 1e3, "TFLOPps": tf8, "peak_TFLOPps": fp8_peak,
                            "peak_source": "measured bf16 burst x 2 (nominal FP8/BF16 dense ratio)",
                            "frac": tf8 / fp8_peak, "model_pred_ms": float(p8.item()) * 1e3,
                            "model_ape_pct": abs(float(p8.item()) - r8["median_s"]) / r8["median_s"] * 100,
                            "sm_mhz_begin": r8["sm_mhz_begin"], "sm_mhz_end": r8["sm_mhz_end"],
                            "clock_reasons": r8["clock_reasons"], "timing": "median of 20 launches after 5 warm-ups"}
    del C8, ops8
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    out["model"] = {"configs": nc, "forward_Mcfg_per_s": nc / t_f / 1e6, "forward_us": t_f * 1e6,
                    "adjoint_Mcfg_per_s": nc / t_g / 1e6, "adjoint_us": t_g * 1e6,
                    "autotune_Mcfg_per_s": (nc // 180) * 180 / t_a / 1e6, "autotune_us": t_a * 1e6,
                    "forward_GBps": 28.0 * nc / t_f / 1e9}
    # 10^8 configurations (the 10^6 batch repeated on the device): the asymptotic
    # rates, and the forward's fraction of the 28 B/configuration HBM floor
    big = 100
    dev_big = dev.repeat(big)
    nb = nc * big
    t_big = torch.empty(nb, dtype=torch.float32, device="cuda")
    tm_big = torch.full((nb,), 1e-3, dtype=torch.float32, device="cuda")
    ws_big = torch.empty(pm.pm_model_grad_workspace(nb) // 8, dtype=torch.float64, device="cuda")
    t_fb = timeit(lambda: pm.pm_model_predict(dev_big, nb, theta, n_sm, t_big), reps=10)
    t_gb = timeit(lambda: pm.pm_model_grad(dev_big, nb, theta, n_sm, tm_big, ws_big, go), reps=10)
    out["model"].update({"configs_large": nb, "forward_large_Mcfg_per_s": nb / t_fb / 1e6,
                         "adjoint_large_Mcfg_per_s": nb / t_gb / 1e6,
                         "forward_large_hbm_frac": 28.0 * nb / t_fb / 1e9 / hbm,
                         "adjoint_large_hbm_frac": 28.0 * nb / t_gb / 1e9 / hbm})
    del dev_big, t_big, tm_big, ws_big
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cfg", default=None, help="override the tile: BM,BN,BK,stages,cta_group")
    ap.add_argument("--skip-extra", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--skip-exhaustive", action="store_true")
    ap.add_argument("--e2e-chunks", type=int, default=8)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
