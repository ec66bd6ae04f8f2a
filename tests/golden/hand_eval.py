"""Hand evaluation of the stage-centric model for the oracle's pins.

A plain, scalar restatement of the model of arxiv 2605.04178 for a handful of
configurations: the Blackwell stage equations (Sec. III-A, Eqs. 2-8), the
roofline floor of Sec. II-A and the working-set bandwidth of Eq. 16, under
both sets of readings of the points the paper leaves open.  It imports
neither the oracle nor the library: it is an independent second
transcription, written top to bottom in the order of the paper's equations,
so a transcription slip in either one shows up as a mismatch.

Run `python tests/golden/hand_eval.py` to rewrite hand_rows.json beside it;
tests/test_oracle_golden.py checks that the file is current and that this
script reproduces the golden row printed with the model's definition
(1.438600e-05 s for the FP32 512^3 launch, etc.), and tests/test_oracle_model.py
reads its values.

Units: seconds, bytes, bytes/s, FLOP/s.  Parameters theta, by index:
  0 T_launch, 1 B_sus, 2 B_peak, 3 w0, 4 L_TMA, 5 B_TMA per SM,
  6/7/8 R_TC per SM (TF32/BF16/FP8), 9 L_mma, 10/11 TMEM read/write bandwidth
  per SM, 12 L_mbar, 13 L_alloc + L_dealloc, 14 S_2SM, 15 c_alpha,
  16 rho_L2 (the measured reading's L2-resident TMA speed-up), 17 B_drain (the
  measured reading's per-SM drain rate of a single-buffered accumulator).
"""
import json
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "hand_rows.json")

LITERAL, MEASURED = 0, 1


def printed_prior(n_sm, f_hz=1.9e9, reading=LITERAL):
    """Priors from the paper's printed values: launch 5 us (Sec. V-B, 5-12 us),
    sustained/peak HBM 6.8/8 TB/s (Sec. II-A, Table "arch-params"), w0 = 64 MiB
    (Eq. 16), L_TMA 420 cycles, tcgen05.mma 12 cycles, mbarrier 45 cycles
    (Table "parameters"), TMEM 16/8 TB/s read/write (Table "parameters"),
    BF16 8192 FLOP per cycle per SM (the dense datasheet rate), TF32 half and
    FP8 twice that, TMEM management 100 ns, S_2SM 1, c_alpha for alpha(2) =
    0.85, rho_L2 the peak-to-sustained HBM ratio, B_drain the per-SM share of
    the sustained HBM rate (like B_TMA).  Cycles are converted at f_hz."""
    bf16 = 8192.0 * f_hz
    return [
        5e-6,                      # 0 T_launch
        6.8e12,                    # 1 B_sus
        8.0e12,                    # 2 B_peak
        64.0 * 1024 * 1024,        # 3 w0
        420.0 / f_hz,              # 4 L_TMA
        6.8e12 / n_sm,             # 5 B_TMA per SM: the sustained HBM rate shared by the SMs
        bf16 / 2.0,                # 6 R_TC TF32
        bf16,                      # 7 R_TC BF16
        2.0 * bf16,                # 8 R_TC FP8
        12.0 / f_hz,               # 9 L_mma
        16e12,                     # 10 TMEM read
        8e12,                      # 11 TMEM write
        45.0 / f_hz,               # 12 L_mbar
        100e-9,                    # 13 TMEM alloc + dealloc
        1.0,                       # 14 S_2SM
        0.3 if reading == LITERAL else 0.15,   # 15 c_alpha
        8.0e12 / 6.8e12,           # 16 rho_L2
        6.8e12 / n_sm,             # 17 B_drain per SM
    ]


def up(a, b):
    return -(-a // b)


def gemm_time(th, n_sm, reading, M, N, K, BM, BN, BK, stages, cta_group, dtype):
    """T_hat of one GEMM launch (TMEM strategy A), step by step."""
    e = {0: 4.0, 1: 2.0, 2: 1.0}[dtype]          # operand bytes
    n_pass = 3.0 if dtype == 0 else 1.0           # three TF32 passes for FP32
    l = 2.0 if dtype == 0 else 1.0                # FP32 loads a hi and a lo plane
    R = th[{0: 6, 1: 7, 2: 8}[dtype]]
    k_instr = {0: 8, 1: 16, 2: 32}[dtype]
    g = cta_group

    K_tiles = up(K, BK)
    if reading == LITERAL:
        tiles = up(M, BM) * up(N, BN)
    else:
        tiles = g * up(M, g * BM) * up(N, BN)     # a pair covers 2 BM rows
    conc = n_sm if g == 1 else 2 * (n_sm // 2)
    waves = up(tiles, conc)

    # Eq. 2: accumulator bytes read and written per K-step, plus the MMA latency
    D = 4.0 * BM * BN
    if reading == LITERAL:
        mmas = 1.0
    else:
        mmas = n_pass * (BK // k_instr) * up(BM, 128)
    T_TMEM = D / th[10] + mmas * th[9] + D / th[11]
    # Eq. 3 (and Eq. 6's S_2SM for a pair).  Literal: TMEM management
    # amortised per K-step.  Measured: it is paid once per launch (below), and
    # a 64-row tile on one SM takes the tensor time of 128 rows.
    S = 1.0 if g == 1 else th[14]
    if reading == LITERAL:
        T_c = n_pass * 2.0 * BM * BN * BK / (R * S) + T_TMEM + th[13] / K_tiles
    else:
        rows = 128 if (g == 1 and BM < 128) else BM
        T_c = n_pass * 2.0 * rows * BN * BK / (R * S) + T_TMEM

    # Eq. 4 with P = 1: each CTA loads its A rows and 1/g of the B tile
    b_step = l * e * BK * (BM + BN / g)
    working_set = l * e * (M * K + N * K) + 4.0 * M * N
    B_TMA = th[5]
    if reading == MEASURED and th[3] > 0:
        # loads that hit in L2 arrive faster: rho_L2 for a resident working
        # set, falling to 1 with Eq. 16's exponential shape
        B_TMA = th[5] * (1.0 + (th[16] - 1.0) * math.exp(-working_set / th[3]))
    T_tma = th[4] + b_step / B_TMA

    # Eq. 7: overlap from the ring depth
    T_sync = 2.0 * th[12]                         # full and empty barrier
    depth = stages if reading == LITERAL else stages - 1
    one_minus_alpha = min(max(th[15] / depth, 0.0), 1.0)
    if reading == LITERAL:
        T_io = one_minus_alpha * T_tma + T_sync
    else:
        T_io = one_minus_alpha * T_tma

    # Eq. 8
    T_step = max(T_c, T_io) + T_sync
    if reading == MEASURED:
        # O_misc: s stages cycle through load, MMAs and barriers
        T_step = max(T_step, (T_tma + T_c + T_sync) / stages)

    # writeback of the FP32 tile, then the kernel total; the measured reading's
    # launch includes the TMEM allocation and release of the persistent CTAs.
    # Measured reading: a kernel that cannot hold two accumulators in the 512
    # TMEM columns (two of ceil(BM/128) BN columns; BN/2 for 64 rows per CTA of
    # a pair) drains each tile before the next one starts, at B_drain per SM.
    T_store = th[4] + 4.0 * BM * BN / th[5]
    acc_cols = BN / 2 if (BM < 128 and g == 2) else up(BM, 128) * BN
    if reading == MEASURED and 2 * acc_cols > 512:
        T_store += 4.0 * BM * BN / th[17]
    launch = th[0] if reading == LITERAL else th[0] + th[13]
    T_stage = launch + waves * (K_tiles * T_step + T_store)

    # naive roofline floor (Sec. II-A)
    flops = n_pass * 2.0 * M * N * K
    T_roof = launch + max(flops / (n_sm * R * S), working_set / th[2])
    return max(T_stage, T_roof)


def stream_time(th, kind, n):
    """Copy (kind 1, 8 B per element) or triad (kind 2, 12 B): Eq. 16 with
    W = the bytes moved, floored by the peak rate."""
    beta = (8.0 if kind == 1 else 12.0) * n
    B = th[1] if th[3] <= 0 else th[1] + (th[2] - th[1]) * math.exp(-beta / th[3])
    return max(th[0] + beta / B, th[0] + beta / th[2])


# The configurations pinned; the first four GEMM rows and the three stream
# rows carry the golden values printed with the model's definition.
CONFIG_ROWS = [
    dict(M=512, N=512, K=512, BM=128, BN=128, BK=32, stages=2, cta_group=1, dtype=0),
    dict(M=8192, N=8192, K=8192, BM=128, BN=256, BK=64, stages=4, cta_group=1, dtype=1),
    dict(M=8192, N=8192, K=8192, BM=128, BN=256, BK=128, stages=4, cta_group=1, dtype=2),
    dict(M=16384, N=16384, K=16384, BM=128, BN=128, BK=64, stages=2, cta_group=1, dtype=1),
    dict(M=2 ** 30, kind=1),
    dict(M=2 ** 30, kind=2),
    dict(M=2 ** 20, kind=1),
]
# Load-bound rows (T_io > T_c) that pin the overlap law of Eq. 7: c_alpha = 0.9.
LOAD_BOUND_ROWS = [dict(M=4096, N=4096, K=4096, BM=128, BN=64, BK=128, stages=s, cta_group=1, dtype=1)
                   for s in (4, 6)]
# Rows whose 256 x 256 accumulator fills the TMEM columns (one buffer): they
# pin the measured reading's drain term (one SM and a CTA pair, BF16 and FP8).
SINGLE_BUFFER_ROWS = [dict(M=8192, N=8192, K=8192, BM=256, BN=256, BK=64, stages=3, cta_group=1, dtype=1),
                      dict(M=8192, N=8192, K=8192, BM=256, BN=256, BK=128, stages=3, cta_group=1, dtype=2),
                      dict(M=8192, N=8192, K=8192, BM=256, BN=256, BK=64, stages=4, cta_group=2, dtype=1)]


def row_time(th, n_sm, reading, row):
    if row.get("kind", 0) != 0:
        return stream_time(th, row["kind"], row["M"])
    return gemm_time(th, n_sm, reading, row["M"], row["N"], row["K"], row["BM"], row["BN"], row["BK"],
                     row["stages"], row["cta_group"], row["dtype"])


def compute():
    n_sm = 160
    out = dict(n_sm=n_sm, f_hz=1.9e9, config_rows=CONFIG_ROWS, load_bound_rows=LOAD_BOUND_ROWS,
               single_buffer_rows=SINGLE_BUFFER_ROWS, prior={}, config_times={}, load_bound_times={},
               load_bound_times_no_blend={}, single_buffer_times={})
    for reading, name in ((LITERAL, "literal"), (MEASURED, "measured")):
        th = printed_prior(n_sm, reading=reading)
        out["prior"][name] = th
        out["config_times"][name] = [row_time(th, n_sm, reading, r) for r in CONFIG_ROWS]
        out["single_buffer_times"][name] = [row_time(th, n_sm, reading, r) for r in SINGLE_BUFFER_ROWS]
        lb = list(th)
        lb[15] = 0.9
        out["load_bound_times"][name] = [row_time(lb, n_sm, reading, r) for r in LOAD_BOUND_ROWS]
        lb[3] = 0.0                                   # w0 <= 0: no working-set blend
        out["load_bound_times_no_blend"][name] = [row_time(lb, n_sm, reading, r) for r in LOAD_BOUND_ROWS]
    return out


def main():
    with open(OUT, "w") as f:
        json.dump(compute(), f, indent=1)
        f.write("\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
