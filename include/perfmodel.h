/*
 * perfmodel.h -- C ABI of libperfmodel.so, the GB300 (sm_103a) hot path of the
 * stage-centric performance model of arxiv 2605.04178 ("Microbenchmark-Driven
 * Analytical Performance Modeling Across Modern GPU Architectures").
 *
 * Conventions shared by every entry point
 *  - Pointers named *_dev are CUDA device pointers on the current device; the
 *    caller allocates and owns them.  Pointers named *_host are host memory.
 *    The library keeps only a small per-device cache (TMA descriptors of the
 *    last call, the watchdog word) and never frees caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Entry points documented "async" only enqueue work; those
 *    documented "synchronises" wait for their stream before returning.
 *  - Matrices are row-major.  Times are seconds.
 *  - Every entry point returns a pm_status.  On failure nothing is launched
 *    unless the status is PM_ECUDA/PM_ETIMEOUT (reported after the fact), and
 *    pm_last_error() gives a message.  No entry point aborts the process.
 *  - Device-side waits (mbarrier pipelines) are bounded by a watchdog; on
 *    expiry the kernel records PM_ETIMEOUT in a device word, releases its
 *    tensor memory and returns.  Synchronising entry points report it;
 *    asynchronous ones report it through pm_device_status().
 */
#ifndef PERFMODEL_H
#define PERFMODEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PM_OK = 0,
  PM_EINVAL = -1,        /* bad argument: null pointer, size, alignment */
  PM_EUNSUPPORTED = -2,  /* configuration outside the valid tile space */
  PM_ECUDA = -3,         /* a CUDA runtime/driver call failed */
  PM_ETIMEOUT = -4,      /* a device-side wait hit the watchdog limit */
  PM_ENOMEM = -5         /* workspace (caller-provided or built-in) too small */
} pm_status;

/* Operand precisions of the GEMM family (Sec. II: 5th-gen tensor cores take
 * TF32, BF16 and FP8; FP32 accumulation in TMEM, Sec. III-A.1).  PM_FP32 runs
 * three TF32 passes (hi*hi + hi*lo + lo*hi) so the product keeps FP32 accuracy. */
typedef enum { PM_FP32 = 0, PM_BF16 = 1, PM_FP8E4M3 = 2 } pm_dtype;

/* Workload kinds the model predicts: the GEMM family and the calibration
 * probes of Sec. V-A (memory copy/triad through Eq. 16, TMA tile copy). */
typedef enum { PM_KIND_GEMM = 0, PM_KIND_COPY = 1, PM_KIND_TRIAD = 2, PM_KIND_TMA2D = 3 } pm_kind;

/* One workload configuration (24 bytes, 8-byte aligned arrays).
 *  GEMM : C[M,N] = A[M,K] B[K,N]; tile BM x BN x BK per CTA, `stages` deep
 *         shared-memory ring, cta_group 1 (one SM) or 2 (CTA pair, the pair
 *         covers 2*BM x BN), dtype a pm_dtype.  These are the model inputs of
 *         Sec. III-E (b_M, b_N, b_K, K_tiles, bytes per CTA; P = 1).
 *         tmem_a selects the TMEM strategy of Sec. III-A.1: 0 = A (only the
 *         accumulators in TMEM, both operands read from shared memory),
 *         1 = B (each stage's A tile also copied into TMEM by tcgen05.cp and
 *         read from there by the MMAs).
 *  COPY/TRIAD: M = FP32 elements.  TMA2D: M x N FP32 matrix in BM x BN tiles.
 *  Probe kinds take tmem_a = 0.
 * Valid GEMM tile space: BM, BN in {64,128,256}; BK in {32,64} (FP32) or
 * {64,128} (BF16, FP8); stages 2..6; cta_group 1..2; stages * stage bytes
 * <= 227 KiB - 2 KiB where stage bytes = l*e*BK*(BM + BN/cta_group) with e the
 * element size and l = 2 for FP32 (hi and lo), else 1; ceil(BM/128)*BN <= 512
 * TMEM columns (the 256 KB TMEM limit of Sec. III-A.1).  Strategy B further
 * needs cta_group 1, BM >= 128 and ceil(BM/128)*(BN + stages*l*BK*e/4) <= 512
 * columns (accumulator plus the A ring in TMEM). */
typedef struct {
  int32_t M, N, K;
  int16_t BM, BN, BK;
  int8_t stages, cta_group, dtype, kind;
  int16_t tmem_a;        /* TMEM strategy: 0 = A, 1 = B */
} pm_cfg;

/* Model parameters theta, SI units (Sec. III-A and Eq. 16):
 *  0 T_launch   1 B_sus      2 B_peak     3 w0          4 L_TMA      5 B_TMA/SM
 *  6 R_TC tf32  7 R_TC bf16  8 R_TC fp8   9 L_mma      10 BW_TMEM_rd 11 BW_TMEM_wr
 * 12 L_mbar    13 L_alloc+L_dealloc      14 S_2SM      15 c_alpha
 * 16 rho_L2 (measured reading only: TMA load speed-up of an L2-resident
 *    working set, Sec. III-A.2)
 * 17 B_drain/SM (measured reading only: rate at which a tile's accumulator
 *    is drained when the kernel keeps one accumulator buffer, Sec. III-A.5)
 * with the overlap law alpha(stages) = clamp(1 - c_alpha/stages, 0, 1) (the
 * measured reading: clamp(1 - c_alpha/(stages - 1), 0, 1)). */
#define PM_NPARAMS 18
typedef struct { float v[PM_NPARAMS]; } pm_params;

/* Readings of the points the paper leaves open in the stage model:
 *  PM_READING_LITERAL: the equations as printed -- L_mma once per K-step
 *    (Eq. 2), alpha = 1 - c_alpha/stages, T_sync in both Eq. 7 and Eq. 8,
 *    TMEM management amortised over the K-steps (Sec. III-A.5);
 *  PM_READING_MEASURED (default): readings measured on this library's
 *    kernels -- L_mma once per tensor-pipe instruction of the K-step
 *    (BK/k_instr per 128-row block per pass, plus strategy B's copies),
 *    alpha = 1 - c_alpha/(stages-1), T_sync once per K-step (Eq. 8), O_misc
 *    of Eq. 8 = the bubble of the s-deep ring (T_step >= (T_tma + T_c +
 *    T_sync)/s), the TMA bandwidth scaled by an L2-residency factor
 *    rho(W) = 1 + (rho_L2 - 1) exp(-W/w0) over the launch's working set W
 *    (operands and C; Sec. III-A.2 notes that L2 hits change B_TMA; the
 *    shape of Eq. 16's blend), the TMEM management paid once per launch (a
 *    persistent CTA allocates tensor memory once: T_launch + L_alloc+L_dealloc
 *    starts every GEMM launch), and a one-SM tile of 64 rows at the tensor
 *    time of 128 rows (an M = 64 tcgen05.mma on one SM takes as long as an
 *    M = 128 one), and T_store + 4 BM BN / B_drain per tile of a launch whose
 *    accumulator cannot be double-buffered in the 512 TMEM columns (twice
 *    ceil(BM/128) BN columns, BN/2 for 64 rows per CTA of a pair, plus
 *    strategy B's A copy per stage, above 512): its next tile waits for the
 *    drain, which two buffers hide.  A grouped launch is single-buffered when
 *    any group's tile is.
 * The setting is process-wide and read by every model entry point at launch;
 * fit theta under the reading it will be used with. */
typedef enum { PM_READING_LITERAL = 0, PM_READING_MEASURED = 1 } pm_reading;
pm_status pm_model_set_reading(int32_t reading);
int32_t pm_model_reading(void);

/* ------------------------------------------------------------------ probes */
/* Calibration microbenchmarks (Sec. V-A; STREAM-style copy and triad for the
 * memory-bound class; TMA copy latency and bandwidth by tile size; pointer
 * chase after Mei & Chu as cited in Sec. III-B).
 *  PM_PROBE_COPY  : buf1[i] = buf0[i], n FP32 elements (16-byte aligned buffers).
 *  PM_PROBE_TRIAD : buf0[i] = fmaf(scalar, buf2[i], buf1[i]) (one rounding).
 *  PM_PROBE_TMA2D : buf1 = buf0, an rows x cols FP32 matrix moved in
 *                   tile_r x tile_c tiles by TMA loads and TMA stores through
 *                   a shared-memory ring (cols*4 bytes a multiple of 16).
 *  PM_PROBE_PCHASE: j = buf0[j * 16] for `hops` hops from `start` by one
 *                   thread (nodes 64 bytes apart, n nodes); the final j is
 *                   written to ((uint32_t*)buf1)[0].  start = 0xFFFFFFFF
 *                   resumes from the node in buf1[0]; pm_probe_run resumes
 *                   this way on every launch after its first, so repeated
 *                   runs walk new nodes rather than re-walk cached ones and
 *                   final_index is the node after (warmup + reps) * hops hops. */
/* Blackwell instruction and host-link probes (Sec. V-A (i), (iii), (iv); Eq. 15):
 *  PM_PROBE_MMA    : one CTA (cta_group 1) or CTA pair (2) per SM issues n
 *                    (<= 2^19) back-to-back tcgen05.mma of one shape from
 *                    operands equal to 1.0 into one TMEM accumulator; rows =
 *                    cta_group, cols = pm_dtype, tile_c = instruction M (64/128
 *                    for one SM, 128/256 for a pair), tile_r = N (16..256, step
 *                    16), start = CTAs (0 = one per SM).  ((uint32_t*)buf0)[cta]
 *                    = bits of D[0][0] = n * k (k = 8 TF32, 16 BF16, 32 FP8).
 *                    result.bytes holds the launch's FLOPs.
 *  PM_PROBE_MBAR   : two threads of different warps pass a token through two
 *                    mbarriers n times; final_index = completed round trips.
 *  PM_PROBE_TMEM_LD: every SM fills 128 lanes x 512 columns of TMEM with
 *                    lane*512 + column; 8 warps (warp w: lanes 32*(w%4).., columns
 *                    256*(w/4)..) read their part n times with tcgen05.ld;
 *                    ((uint32_t*)buf0)[sm*256 + thread] = the sum of everything
 *                    that thread read (mod 2^32).
 *  PM_PROBE_TMEM_ST: n passes of tcgen05.st writing lane*512 + column + pass,
 *                    then one read pass; buf0 as above (sum of the last pass).
 *  PM_PROBE_H2D / PM_PROBE_D2H: cudaMemcpyAsync of n bytes from buf0 to buf1
 *                    (host memory pinned for full speed).
 *  PM_PROBE_HOST_READ / PM_PROBE_HOST_WRITE: the SMs copy n FP32 elements from
 *                    buf0 to buf1 through the device mapping of CUDA
 *                    page-locked host memory (buf0 host for READ, buf1 host
 *                    for WRITE; no copy engine); PM_EINVAL if the host buffer
 *                    is not such memory.  result.bytes = 4n.
 *  PM_PROBE_STENCIL: buf1 = five-point stencil of the rows x cols FP32 grid
 *                    buf0 (distinct buffers): interior points
 *                    0.5 x + 0.125 ((up + down) + (left + right)), each
 *                    operation rounded separately; border points copied.
 *                    result.bytes = 8 rows cols (one read, one write). */
typedef enum {
  PM_PROBE_COPY = 1, PM_PROBE_TRIAD = 2, PM_PROBE_TMA2D = 3, PM_PROBE_PCHASE = 4, PM_PROBE_H2D = 5,
  PM_PROBE_D2H = 6, PM_PROBE_MMA = 7, PM_PROBE_MBAR = 8, PM_PROBE_TMEM_LD = 9, PM_PROBE_TMEM_ST = 10,
  PM_PROBE_HOST_READ = 11, PM_PROBE_HOST_WRITE = 12, PM_PROBE_STENCIL = 13
} pm_probe_kind;

typedef struct {
  int32_t kind;          /* pm_probe_kind */
  int32_t tile_r, tile_c;/* TMA2D tile (rows, cols), each in [8, 256] */
  uint32_t start;        /* PCHASE start node */
  int64_t n;             /* COPY/TRIAD elements; PCHASE nodes */
  int64_t rows, cols;    /* TMA2D matrix */
  int64_t hops;          /* PCHASE hops */
  float scalar;          /* TRIAD s */
  int32_t reserved;
} pm_probe_args;

typedef struct {
  double median_s, p25_s, p75_s, min_s;   /* per-launch device time */
  double bytes;                           /* algorithmic bytes per launch */
  uint32_t final_index;                   /* PCHASE result */
  /* Clock record of the timed region (Sec. V-B protocol: clocks and throttle
   * state recorded with every measurement): SM clock read through NVML just
   * before the first timed launch and just after the last one completed, the
   * maximum SM clock, and the OR of the NVML clock event reasons seen at
   * both reads (0x4 software power cap, 0x8 hardware slowdown, 0x20
   * software thermal slowdown, 0x40 hardware thermal slowdown, 0x80 power
   * brake).  Zero when NVML cannot be read. */
  uint32_t sm_mhz_begin, sm_mhz_end, sm_max_mhz;
  uint64_t clock_reasons;
} pm_probe_result;                        /* 64 bytes */

/* One read-only NVML sample of the current CUDA device (matched by PCI bus
 * id): SM, maximum SM and memory clocks, board power, clock event reasons
 * (bitmask as in pm_probe_result), and the host's monotonic time.  Changes
 * no GPU setting.  PM_EUNSUPPORTED when the driver's NVML library cannot be
 * loaded or does not know the device. */
typedef struct {
  uint32_t sm_mhz, sm_max_mhz, mem_mhz, power_mw;
  uint64_t reasons;
  double host_time_s;
} pm_clock;                               /* 32 bytes */

pm_status pm_clock_sample(pm_clock* out);

/* Concurrent-stream interference probe (Sec. III-A.6: N_c concurrent streams
 * add (N_c - 1) tau_c to the single-stream time).  Launches the probe
 * `per_stream` (PM_PROBE_COPY, PM_PROBE_TRIAD or PM_PROBE_MMA) once on each of
 * n_streams (1..8) library-owned non-blocking streams, stream i on buffers
 * buf0[i], buf1[i], buf2[i] (host arrays of n_streams device pointers; buf1
 * may be NULL for MMA, buf2 is needed for TRIAD only).  All streams are
 * released by one event on `stream` and joined back on it; each rep's time is
 * the makespan between those two events.  `warmup` untimed then `reps` timed
 * reps; result as for pm_probe_run with bytes (FLOPs for MMA) summed over the
 * streams.  The streams are created on first use per device and kept until
 * process exit.  Synchronises `stream`. */
pm_status pm_streams_run(const pm_probe_args* per_stream, int32_t n_streams, void* const* buf0, void* const* buf1,
                         void* const* buf2, int warmup, int reps, void* stream, pm_probe_result* out);

/* One probe launch on `stream` (async). */
pm_status pm_probe_launch(const pm_probe_args* args, void* buf0, void* buf1, void* buf2, void* stream);

/* `warmup` untimed then `reps` timed launches, each bracketed by CUDA events
 * on `stream`; fills *out with median and quartiles (Sec. V-B protocol:
 * 10 warm-ups, 100 runs, median).  Synchronises. */
pm_status pm_probe_run(const pm_probe_args* args, void* buf0, void* buf1, void* buf2, int warmup, int reps,
                       void* stream, pm_probe_result* out);

/* ---------------------------------------------------------------- GEMM */
/* Bytes of the operand buffers pm_gemm_prepare writes: A_op holds A as
 * dtype [M,K] (FP32: hi then lo, 2*M*K floats), B_op holds B transposed to
 * [N,K] (K-major, FP32: hi then lo), `scales_dev` 4 floats. */
pm_status pm_gemm_operand_bytes(int32_t dtype, int32_t M, int32_t N, int32_t K, size_t* a_bytes, size_t* b_bytes);

/* Operand preparation (async): casts row-major FP32 A [M,K] and B [K,N]
 * into the tensor-core operand formats.  BF16: round to nearest even.
 * FP8 e4m3: per-tensor scale s = 448/max|X| (FP32 division), codes
 * RNE-saturated from s*X; scales_dev[0] = s_A, scales_dev[1] = s_B.
 * FP32: hi = tf32_rn(X), lo = tf32_rn(X - hi).  scales_dev (4 floats) is
 * required for FP8 and ignored otherwise. */
pm_status pm_gemm_prepare(int32_t dtype, const float* A_dev, const float* B_dev, int32_t M, int32_t N, int32_t K,
                          void* A_op_dev, void* B_op_dev, float* scales_dev, void* stream);

/* C[M,N] (FP32, row-major, leading dimension N) = A B with the tile
 * configuration `cfg` (kind PM_KIND_GEMM), from the operands written by
 * pm_gemm_prepare.  FP8 results are multiplied by 1/(s_A s_B) read from
 * scales_dev.  The kernel is the paper's pipeline (Fig. "cta-exec-model"):
 * TMA -> shared-memory ring -> tcgen05.mma -> TMEM -> epilogue, one
 * persistent CTA (or CTA pair) per SM.  Async.  Requires K*e % 16 == 0. */
pm_status pm_gemm_run(const pm_cfg* cfg, const void* A_op_dev, const void* B_op_dev, float* C_dev,
                      const float* scales_dev, void* stream);

/* Timing harness for the GEMM (Sec. V-B protocol): `warmup` untimed then
 * `reps` timed pm_gemm_run launches, each bracketed by CUDA events on
 * `stream`; result fields as for pm_probe_run (bytes = algorithmic operand
 * and result bytes of one launch).  Synchronises; reports PM_ETIMEOUT if a
 * device wait expired during the runs. */
pm_status pm_gemm_bench(const pm_cfg* cfg, const void* A_op_dev, const void* B_op_dev, float* C_dev,
                        const float* scales_dev, int warmup, int reps, void* stream, pm_probe_result* out);

/* End-to-end GEMM from host memory: C_host[M,N] = A_host[M,K] B_host[K,N]
 * (FP32 row-major; pinned host memory lets the copies overlap), in the tile
 * configuration `cfg`.  B is copied and converted first; A then moves in
 * `chunks` row chunks on a copy stream, each chunk is converted and
 * multiplied while the next is in flight, and each finished C chunk is copied
 * back on a third stream (FP8 uses one chunk: its per-tensor scale needs all
 * of A).  The work is ordered after prior work on `stream` and `stream` waits
 * for its completion, so the call is async with respect to `stream`.
 * ws_dev: pm_gemm_host_workspace bytes, 256-byte aligned, owned by the
 * caller.  One device per calling host thread. */
pm_status pm_gemm_host_workspace(const pm_cfg* cfg, int32_t chunks, size_t* bytes);
pm_status pm_gemm_host(const pm_cfg* cfg, const float* A_host, const float* B_host, float* C_host, void* ws_dev,
                       size_t ws_bytes, int32_t chunks, void* stream);

/* Grouped BF16 GEMM in one persistent launch: G problems C_g[M_g,N] =
 * A_g[M_g,K] B_g[K,N].  A_op_dev stacks the A_g as bf16 [sum M_g, K]; B_op_dev
 * stacks the B_g transposed, bf16 [G*N, K]; C_dev stacks C_g, FP32
 * [sum M_g, N].  Group g uses tile BM_host[g] x BN_host[g]; BK, stages and
 * cta_group are per launch.  Tiles are listed group by group and tile t runs
 * on CTA t mod (number of CTAs).  Async; capturable in a CUDA graph after one
 * uncaptured call with the same shapes (which builds the descriptors). */
pm_status pm_grouped_gemm_run(int32_t G, const int32_t* M_host, int32_t N, int32_t K, const int16_t* BM_host,
                              const int16_t* BN_host, int32_t BK, int32_t stages, int32_t cta_group,
                              const void* A_op_dev, const void* B_op_dev, float* C_dev, void* stream);

/* --------------------------------------------------------------- model */
/* Stage-model prediction T_hat (FP32 seconds) for n configurations (any
 * kind) on the GPU: Eqs. 2-8 for GEMM tiles with persistent-CTA waves and the
 * naive roofline as a floor; Eq. 16 for copy/triad; the TMA tile model for
 * TMA2D.  cfgs_dev: n pm_cfg; t_out_dev: n floats.  A record the model cannot
 * evaluate (a non-positive size, an unknown kind, dtype or cta_group, or a
 * cta_group 2 pair when n_sm < 2: a pair needs two SMs) gets NaN.  Async. */
pm_status pm_model_predict(const pm_cfg* cfgs_dev, int64_t n, const pm_params* theta_host, int32_t n_sm,
                           float* t_out_dev, void* stream);

/* Scratch the gradient needs: partial sums of 1 + PM_NPARAMS doubles per block. */
pm_status pm_model_grad_workspace(int64_t n, size_t* bytes);

/* Calibration objective of Sec. III-D (parameters fitted to measured times):
 *   L = (1/n) sum_i (ln T_hat_i - ln T_i)^2 and dL/dtheta (PM_NPARAMS values),
 * from a hand-written adjoint of the model (ties of max() go to the first
 * argument, the alpha clamp has zero slope outside (0,1)).  Per-block partial
 * sums go to workspace_dev (pm_model_grad_workspace bytes) and are reduced in
 * FP64 in a fixed order; out_dev receives 1 + PM_NPARAMS doubles
 * {L, dL/dtheta_0 .. dL/dtheta_16}.
 * Async. */
pm_status pm_model_grad(const pm_cfg* cfgs_dev, int64_t n, const pm_params* theta_host, int32_t n_sm,
                        const float* t_meas_dev, void* workspace_dev, size_t workspace_bytes, double* out_dev,
                        void* stream);

/* pm_model_grad evaluated entirely in FP64 (parameters, per-configuration
 * model and adjoint, log residuals), for the calibration fit: the FP32
 * objective is piecewise flat at the 1e-7 level, which stalls the line
 * searches of a quasi-Newton fit near its optimum.  theta_host: PM_NPARAMS doubles
 * in the pm_params order; t_meas_dev: n doubles (8-byte aligned); workspace
 * and output as for pm_model_grad.  Async. */
pm_status pm_model_grad_f64(const pm_cfg* cfgs_dev, int64_t n, const double* theta_host, int32_t n_sm,
                            const double* t_meas_dev, void* workspace_dev, size_t workspace_bytes, double* out_dev,
                            void* stream);

/* The k predicted-fastest valid configurations per shape (k <= 16), sorted
 * by predicted time: picks_dev n*k pm_cfg, t_pred_dev n*k floats.  Entries
 * past the number of valid configurations have BM = 0 and t = +inf.  Async. */
pm_status pm_autotune_topk(const int32_t* MNK_dev, int64_t n, int32_t dtype, const pm_params* theta_host,
                           int32_t n_sm, int32_t k, pm_cfg* picks_dev, float* t_pred_dev, void* stream);

/* Model-pruned measured autotuning of one GEMM shape: the model's top-k
 * configurations (pm_autotune_topk) are each timed with pm_gemm_bench on the
 * caller's operands and the fastest is returned in *pick_out (its timing in
 * *pick_time_out, nullable).  `shape` gives M, N, K and dtype.  The paper's
 * autotuning guidance (Sec. VI) ranks tiles by the model; timing a short list
 * absorbs the model's residual error at ~k/180 of an exhaustive search's cost.
 * Allocates a few hundred bytes of device scratch (stream-ordered).
 * Synchronises. */
pm_status pm_gemm_autotune(const pm_cfg* shape, int32_t k, const pm_params* theta_host, int32_t n_sm,
                           const void* A_op_dev, const void* B_op_dev, float* C_dev, const float* scales_dev,
                           int warmup, int reps, void* stream, pm_cfg* pick_out, pm_probe_result* pick_time_out);

/* pm_model_grad without any device allocation, for callers that cannot
 * allocate device memory when they need the gradient (a host program that
 * links only this library and owns no CUDA allocator, a runtime held to a
 * fixed device-memory budget).  The paper has no counterpart: this is an
 * interface convenience of this library.  Same inputs and output as
 * pm_model_grad, minus the workspace: the per-block partial sums go to a
 * fixed 622,592-byte array inside the library, present on every GPU that
 * loads it until the process exits.  At most 1,048,576 configurations per
 * call; larger n returns PM_ENOMEM with a message and launches nothing.
 * It launches the same grid as pm_model_grad, so its output is bit-identical
 * to pm_model_grad's for the same inputs.  The first call on a device looks
 * up that array's device address (cudaGetSymbolAddress, no allocation) and
 * caches it; make that first call outside any stream capture, and call
 * pm_shutdown before a device reset (it forgets the cached address).  All
 * calls share the array: calls whose kernels overlap on the GPU race and must
 * be serialised by the caller (one stream, or events).  Nothing needs
 * clearing between calls: each call writes every partial record it reads.
 * Async. */
pm_status pm_model_grad_noalloc(const pm_cfg* cfgs_dev, int64_t n, const pm_params* theta_host, int32_t n_sm,
                                const float* t_meas_dev, double* out_dev, void* stream);

/* Autotuner (Sec. III-B adaptive tile selection; Sec. VI autotuning
 * guidance): for each of n shapes (MNK_dev: n x {M,N,K} int32) evaluates the
 * model over the 180-point tile space of `dtype` and picks the fastest valid
 * configuration; ties go to the first in lexicographic (BM, BN, BK, stages,
 * cta_group) order; with n_sm < 2 pairs (cta_group 2) are not candidates.
 * picks_dev: n pm_cfg; t_pred_dev: n floats.  Async. */
pm_status pm_autotune_pick(const int32_t* MNK_dev, int64_t n, int32_t dtype, const pm_params* theta_host,
                           int32_t n_sm, pm_cfg* picks_dev, float* t_pred_dev, void* stream);

/* Stage-model makespan of one grouped launch with given per-group tiles
 * (the grouped reading of Eq. 8, exact for pm_grouped_gemm_run's static
 * schedule: per group tau_g = K_tiles T_step_g + T_store_g; the launch lists
 * the groups largest tile (BM x BN) first, ties in the caller's order, and
 * deals the listed tiles to the n_conc workers round by round, the worker
 * order reversed on odd rounds when G > 1; T_hat = launch + max_w sum of the
 * worker's tau, launch = T_launch, plus L_alloc + L_dealloc under the
 * measured reading).  Host arrays of G entries (G <= 1024); *t_pred_host in
 * seconds, NaN for a cta_group 2 launch when n_sm < 2.  Allocates a few KB
 * of stream-ordered device scratch.  Synchronises. */
pm_status pm_grouped_predict(int32_t G, const int32_t* M_host, int32_t N, int32_t K, const int16_t* BM_host,
                             const int16_t* BN_host, int32_t BK, int32_t stages, int32_t cta_group, int32_t dtype,
                             const pm_params* theta_host, int32_t n_sm, float* t_pred_host, void* stream);

/* pm_grouped_predict in FP64 with the makespan's gradient, for the
 * calibration fit's grouped rows (Sec. III-D): the busiest worker's tiles
 * (the first such worker on ties) carry the gradient, each through the
 * adjoint of its K-steps and writeback.  theta_host: PM_NPARAMS doubles;
 * out_host: 1 + PM_NPARAMS doubles {T_hat, dT_hat/dtheta_0 ..}.  Errors as
 * pm_grouped_predict.  Synchronises. */
pm_status pm_grouped_grad(int32_t G, const int32_t* M_host, int32_t N, int32_t K, const int16_t* BM_host,
                          const int16_t* BN_host, int32_t BK, int32_t stages, int32_t cta_group, int32_t dtype,
                          const double* theta_host, int32_t n_sm, double* out_host, void* stream);

/* Grouped autotuner: for each launch-level (BK, stages, cta_group), each
 * group takes the (BM, BN) minimising tiles_g * (K_tiles T_step_g + T_store_g);
 * the launch whose static schedule (pm_grouped_predict) has the smallest
 * makespan wins.  Results to host: BM_out_host/BN_out_host (G each), launch_out_host
 * {BK, stages, cta_group}, *t_pred_host.  Synchronises. */
pm_status pm_grouped_autotune(int32_t G, const int32_t* M_host, int32_t N, int32_t K, int32_t dtype,
                              const pm_params* theta_host, int32_t n_sm, int16_t* BM_out_host,
                              int16_t* BN_out_host, int32_t* launch_out_host, float* t_pred_host, void* stream);

/* Every launch-level candidate the grouped autotuner weighs, in its order
 * (BK, stages, cta_group lexicographic; 20 candidates): t_pred_host[20]
 * their predicted makespans (+inf where some group has no valid tile),
 * BM_host/BN_host [20 x G] the per-group tiles each picks, launch_host
 * [20 x 3] {BK, stages, cta_group}.  For measuring the grouped family over
 * the launch space.  Synchronises. */
pm_status pm_grouped_candidates(int32_t G, const int32_t* M_host, int32_t N, int32_t K, int32_t dtype,
                                const pm_params* theta_host, int32_t n_sm, float* t_pred_host, int16_t* BM_host,
                                int16_t* BN_host, int32_t* launch_host, void* stream);

/* Model-pruned measured grouped autotuning (BF16): the grouped autotuner's
 * k best launch-level candidates (k in 1..20, each with its per-group tiles)
 * are timed on the caller's operands (pm_grouped_gemm_run layout; warmup
 * untimed, reps timed launches, CUDA events on `stream`) and the fastest by
 * median is returned in BM_out_host/BN_out_host/launch_out_host; t_pred_host
 * (nullable) receives its predicted makespan, pick_time_out (nullable) its
 * timing.  Overwrites C_dev.  Synchronises. */
pm_status pm_grouped_gemm_autotune(int32_t G, const int32_t* M_host, int32_t N, int32_t K,
                                   const pm_params* theta_host, int32_t n_sm, int32_t k, const void* A_op_dev,
                                   const void* B_op_dev, float* C_dev, int warmup, int reps, void* stream,
                                   int16_t* BM_out_host, int16_t* BN_out_host, int32_t* launch_out_host,
                                   float* t_pred_host, pm_probe_result* pick_time_out);

/* -------------------------------------------------- generic segment model */
/* The paper's generic roofline path for work that the stage model does not
 * cover (Sec. III-E "Generic roofline path" and "Host-device transfer and
 * synchronization"; Eqs. 15 and 16).  A segment is one step of a workload,
 * executed `execs` times; per execution
 *   T = kernels * T_launch
 *     + s_class * max(flops / (n_SM * R_TC[precision] * eta[precision]),
 *                     bytes / B_eff(working_set))            (Eq. 16)
 *     + [h2d_bytes > 0] (h2d_bytes / B_h2d + tau_h2d)           (Eq. 15)
 *     + [d2h_bytes > 0] (d2h_bytes / B_d2h + tau_d2h)
 *     + syncs * tau_sync
 *     + (N_c - 1) tau_c,  tau_c = kappa_launch * kernels * T_launch
 *                                + kappa[class] * (the s_class roofline term)
 * (the roofline and tau_c terms only when kernels >= 1; copies and kernels
 * are summed, not overlapped, as the paper states; the last line is Sec.
 * III-A.6's (N_c - 1) tau_c for a segment run as N_c concurrent copies on N_c
 * streams, with tau_c the part of one copy that cannot overlap the others).
 * T_launch, B_sus, B_peak, w0 and the per-SM rates R_TC come from the stage
 * model's theta. */
typedef enum { PM_SEG_MEMORY = 0, PM_SEG_COMPUTE = 1, PM_SEG_BALANCED = 2, PM_SEG_STENCIL = 3 } pm_segment_class;

typedef struct {
  double flops;          /* FLOPs of the segment's kernels per execution */
  double bytes;          /* DRAM bytes they move per execution */
  double working_set;    /* W of Eq. 16, bytes */
  double h2d_bytes;      /* host-to-device bytes per execution */
  double d2h_bytes;      /* device-to-host bytes per execution */
  int32_t cls;           /* pm_segment_class */
  int32_t precision;     /* pm_dtype of the arithmetic (selects R_TC and eta) */
  int32_t kernels;       /* kernel launches per execution (>= 0) */
  int32_t syncs;         /* host synchronisation points per execution */
  int32_t execs;         /* executions of the segment (>= 1) */
  int32_t streams;       /* concurrent copies N_c on as many streams (0 or 1: one) */
} pm_segment;            /* 64 bytes */

/* Segment parameters psi (SI units): 0-3 class scales s_class (memory,
 * compute, balanced, stencil), 4-6 precision efficiencies eta (FP32, BF16,
 * FP8), 7 B_h2d, 8 tau_h2d, 9 B_d2h, 10 tau_d2h, 11 tau_sync, 12-15 kappa per
 * class, 16 kappa_launch (concurrent-stream interference). */
#define PM_NPSI 17
typedef struct { double v[PM_NPSI]; } pm_segment_params;

/* T (seconds, FP64) of n segments on the GPU.  segs_dev: n pm_segment;
 * t_out_dev: n doubles.  A record with a negative stream count, an unknown class or precision, a
 * negative size or count, or execs < 1 yields NaN.  Async. */
pm_status pm_segment_predict(const pm_segment* segs_dev, int64_t n, const pm_params* theta_host,
                             const pm_segment_params* psi_host, int32_t n_sm, double* t_out_dev, void* stream);

/* ----------------------------------------------------------- diagnostics */
/* Text of the last error on this host thread (valid until the next call). */
const char* pm_last_error(void);

/* Releases what the library holds beyond its static device arrays: its pool
 * of concurrent-probe streams on every device, and the calling thread's
 * host-transfer pipeline (streams, events) and TMA descriptor caches; it also
 * forgets the cached device addresses of the static arrays (the watchdog
 * word, the allocation-free gradient's scratch) and the cached SM counts.
 * Call it before a device reset (cudaDeviceReset reloads the module, so a
 * cached address would go stale).  Work already queued on those streams
 * completes.  Any later call re-creates or looks up what it needs.  Always
 * PM_OK. */
pm_status pm_shutdown(void);

/* Reads (and with clear != 0, clears) the device watchdog word of the current
 * device: PM_OK or PM_ETIMEOUT.  Synchronises the device. */
pm_status pm_device_status(int clear);

/* Watchdog self-test: one kernel waits on an mbarrier that nothing completes,
 * gives up after limit_us microseconds, records PM_ETIMEOUT and returns.
 * Synchronises; returns the status the device recorded (PM_ETIMEOUT). */
pm_status pm_watchdog_selftest(int32_t limit_us, void* stream);

/* Library version (major*10000 + minor*100 + patch). */
int32_t pm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PERFMODEL_H */
