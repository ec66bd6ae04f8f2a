// Batched evaluation of the stage-centric model of arxiv 2605.04178 (Sec. III-A,
// Eqs. 2-8; Eq. 16 for the memory probes), its hand-written adjoint for
// calibration (Sec. III-D), and the model-driven autotuner (Sec. III-B
// adaptive tile selection, Sec. VI autotuning guidance).
//
// One thread per configuration, FP32 arithmetic, integer tile counts.  The
// explicit-configuration kernels stream 24-byte records (HBM-bound at
// 24-28 B per configuration); the autotuner decodes the configuration from
// the thread index and reads nothing per configuration (ALU-bound).
#include <math.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "pm_internal.cuh"

namespace pm {

// Exact unsigned division by a divisor fixed for the whole launch (the number
// of concurrent CTAs), as one multiply-high, a subtract, an add and two shifts
// instead of the generic division sequence (Granlund and Montgomery,
// "Division by Invariant Integers using Multiplication", PLDI 1994, Sec. 4,
// N = 32).  For 1 <= d <= 2^31 and l = ceil(log2 d):
//   m = floor(2^32 (2^l - d) / d) + 1,   t = floor(m x / 2^32),
//   floor(x / d) = (t + ((x - t) >> min(l, 1))) >> max(l - 1, 0)
// for every 0 <= x < 2^32.
struct UDiv {
  uint32_t d, m;
  int s1, s2;
};

inline UDiv make_udiv(uint32_t d) {
  int l = 0;
  while ((1ull << l) < d) ++l;
  UDiv u;
  u.d = d;
  u.m = (uint32_t)((((1ull << l) - d) << 32) / d + 1);
  u.s1 = l < 1 ? l : 1;
  u.s2 = l > 1 ? l - 1 : 0;
  return u;
}

__device__ __forceinline__ uint32_t udiv(uint32_t x, const UDiv& u) {
  const uint32_t t = __umulhi(u.m, x);
  return (t + ((x - t) >> u.s1)) >> u.s2;
}

// Parameters in the arithmetic type F: FP32 for the batched throughput
// paths, FP64 for the calibration objective (pm_model_grad_f64).
// inv[j] = 1 / v[j], rounded once on the host: the per-configuration model
// multiplies where the equations divide by a parameter.  nc[0] / nc[1]
// divide by the concurrent CTAs of one-SM / paired tiles on nc_nsm SMs
// (nc_nsm = 0: not prepared, the generic division is used).  inv_s[s] =
// 1/s and inv_s1[s] = 1/(s - 1) for the ring depths 2..7, inv_nsm = 1/nc_nsm:
// the per-configuration divisions by small integers become multiplications.
constexpr int NP = PM_NPARAMS;     // model parameters
constexpr int NREC = NP + 1;        // loss + gradient per partial record

template <class F>
struct ThetaT {
  F v[NP];
  F inv[NP];
  int reading;       // PM_READING_LITERAL or PM_READING_MEASURED (see pm_model_set_reading)
  int nc_nsm;
  UDiv nc[2];
  F inv_s[8], inv_s1[8], inv_nsm;
};
using Theta = ThetaT<float>;

template <class F>
inline void set_concurrency(ThetaT<F>& t, int n_sm) {
  for (int s = 0; s < 8; ++s) {
    t.inv_s[s] = s >= 1 ? (F)(1.0 / s) : F(0);
    t.inv_s1[s] = s >= 2 ? (F)(1.0 / (s - 1)) : F(0);
  }
  t.inv_nsm = n_sm >= 1 ? (F)(1.0 / n_sm) : F(0);
  t.nc_nsm = 0;
  if (n_sm >= 2) {
    t.nc[0] = make_udiv((uint32_t)n_sm);
    t.nc[1] = make_udiv((uint32_t)(2 * (n_sm / 2)));
    t.nc_nsm = n_sm;
  }
}

__device__ __forceinline__ float pm_exp(float x) { return expf(x); }
__device__ __forceinline__ double pm_exp(double x) { return exp(x); }
__device__ __forceinline__ float pm_log(float x) { return logf(x); }
__device__ __forceinline__ double pm_log(double x) { return log(x); }
__device__ __forceinline__ float pm_max(float a, float b) { return fmaxf(a, b); }
// The FP32 throughput paths take the hardware approximations (relative error
// of a few 1e-7, far inside their 1e-5 tolerance); FP64 stays exact.
__device__ __forceinline__ float pm_exp_fast(float x) { return __expf(x); }
__device__ __forceinline__ double pm_exp_fast(double x) { return exp(x); }
__device__ __forceinline__ float pm_div_fast(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double pm_div_fast(double a, double b) { return a / b; }
// x / s and x / (s - 1) for a ring depth s (tabulated reciprocals for 2..7)
template <class F>
__device__ __forceinline__ F div_stages(F x, int s, const ThetaT<F>& th) {
  return (s >= 1 && s < 8) ? x * th.inv_s[s] : x / (F)s;
}
template <class F>
__device__ __forceinline__ F div_stages_m1(F x, int s, const ThetaT<F>& th) {
  return (s >= 2 && s < 8) ? x * th.inv_s1[s] : x / (F)(s - 1);
}
__device__ __forceinline__ double pm_max(double a, double b) { return fmax(a, b); }

// ceil(a / b) for a >= 0, b > 0: a shift when b is a power of two (every tile
// extent of the search space), else 32-bit unsigned division whenever both fit
// (64-bit division is a long software sequence); exact either way.
__device__ __forceinline__ int64_t cdiv(int64_t a, int64_t b) {
  if (((uint64_t)a | (uint64_t)b) < 0x80000000ull) {
    const uint32_t ua = (uint32_t)a, ub = (uint32_t)b;
    if ((ub & (ub - 1u)) == 0u) return (int64_t)((ua + ub - 1u) >> (__ffs((int)ub) - 1));
    return (int64_t)((ua + ub - 1u) / ub);
  }
  return (a + b - 1) / b;
}

// Non-negative count to the arithmetic type, through a 32-bit conversion
// when it fits (64-bit conversions run on the narrow FP64 pipe).
template <class F>
__device__ __forceinline__ F count_to(int64_t v) {
  return (uint64_t)v < 0x80000000ull ? (F)(int32_t)v : (F)v;
}

// Element bytes, tensor passes per K-step (three-pass TF32 for FP32) and
// operand copies loaded per element (FP32: hi and lo).
__device__ __forceinline__ float dt_bytes(int dt) { return dt == PM_FP32 ? 4.f : (dt == PM_BF16 ? 2.f : 1.f); }
__device__ __forceinline__ float dt_passes(int dt) { return dt == PM_FP32 ? 3.f : 1.f; }
__device__ __forceinline__ float dt_loads(int dt) { return dt == PM_FP32 ? 2.f : 1.f; }
__device__ __forceinline__ int dt_rate(int dt) { return dt == PM_FP32 ? 6 : (dt == PM_BF16 ? 7 : 8); }

__constant__ int16_t kBM[3] = {64, 128, 256};
__constant__ int16_t kBN[3] = {64, 128, 256};
__constant__ int16_t kBK[3][2] = {{32, 64}, {64, 128}, {64, 128}};

// Valid tile space of the autotuners (TMEM strategy A): ring of `s` stages
// within 227 KiB - 2 KiB, FP32 accumulator columns ceil(BM/128)*BN within the
// 512 TMEM columns.
__host__ __device__ inline bool tile_valid(int BM, int BN, int BK, int s, int g, int dt) {
  if (!(BM == 64 || BM == 128 || BM == 256) || !(BN == 64 || BN == 128 || BN == 256)) return false;
  if (dt == PM_FP32) {
    if (BK != 32 && BK != 64) return false;
  } else if (dt == PM_BF16 || dt == PM_FP8E4M3) {
    if (BK != 64 && BK != 128) return false;
  } else {
    return false;
  }
  if (s < 2 || s > 6 || (g != 1 && g != 2)) return false;
  const int e = dt == PM_FP32 ? 4 : (dt == PM_BF16 ? 2 : 1);
  const int l = dt == PM_FP32 ? 2 : 1;
  const int64_t stage = (int64_t)l * e * BK * (BM + BN / g);
  if ((int64_t)s * stage > 232448 - 2048) return false;
  if (((BM + 127) / 128) * BN > 512) return false;
  return true;
}

// Whether the GEMM kernel keeps one accumulator buffer only: it holds two when
// twice the accumulator columns of the tile (ceil(BM/128) BN, or BN/2 for a
// 64-row tile on a CTA pair), plus strategy B's A copy per stage, fit in the
// 512 TMEM columns.
__host__ __device__ inline bool single_buffer(int BM, int BN, int BK, int s, int g, int dt, int tmem_a) {
  const int acc = (BM < 128 && g == 2) ? BN / 2 : ((BM + 127) / 128) * BN;
  const int le = dt == PM_FP32 ? 8 : (dt == PM_BF16 ? 2 : 1);    // load planes x element bytes
  const int a_ring = tmem_a ? s * ((BM + 127) / 128) * (le * BK / 4) : 0;
  return 2 * acc + a_ring > 512;
}

// Intermediate values of one GEMM evaluation, kept for the adjoint.
template <class F>
struct GemmFwdT {
  F T, T_stage, T_rl, A_rl, B_rl;
  F T_c, T_io, T_tma, oma, X, R, S, invR, invS, T_step, T_store;
  F D, DA_r, DA_w, bstep, store_bytes, n_instr;
  F waves, Kt;
  F W, E, rho;          // L2 residency of the TMA loads (measured reading)
  F launch;             // T_launch (+ L_alloc + L_dealloc once per launch, measured reading)
  F T_eq8, T_ring;       // Eq. 8 and the ring bound (measured reading)
  int ri;
  bool oma_free, blend, ring;
  bool drain;           // measured reading, one accumulator buffer: each tile's drain is paid
};
using GemmFwd = GemmFwdT<float>;

// Stage-centric GEMM time:
//   T_TMEM = (D + D_A,r)/BW_rd + n_instr L_mma + (D + D_A,w)/BW_wr   (Eq. 2)
//            D_A = 0 for TMEM strategy A; strategy B writes the A tile
//            into TMEM (D_A,w = l e BM BK) and every pass reads it back
//            (D_A,r = n_p e BM BK); n_instr = 1 (literal reading) or the
//            tensor-pipe instructions of the K-step incl. strategy B's
//            tcgen05.cp copies (measured reading)
//   T_c    = n_p 2 BM' BN BK / (R S) + T_TMEM + T_mgmt/K_tiles    (Eqs. 3, 6)
//            BM' = BM, except 128 for a one-SM 64-row tile (measured
//            reading: M = 64 instructions take the M = 128 time); the
//            measured reading has no T_mgmt/K_tiles (paid once per launch)
//   T_tma  = L_TMA + b_step / (B_TMA rho), b_step = l e BK (BM + BN/g) (Eq. 4,
//            P = 1); rho = 1 (literal reading) or the L2-residency factor
//            1 + (rho_L2 - 1) exp(-W/w0) over the launch's working set W
//            (measured reading)
//   T_io   = (1 - alpha) T_tma + T_sync, T_sync = 2 L_mbar       (Eq. 7; the
//            measured reading drops this T_sync: one barrier per K-step)
//   T_step = max(T_c, T_io) + T_sync                             (Eq. 8; the
//            measured reading adds the bubble of the s-deep ring as O_misc:
//            T_step = max(Eq. 8, (T_tma + T_c + T_sync) / s))
//   T_stage = launch + waves (K_tiles T_step + T_store)
//   T_hat = max(T_stage, launch + max(FLOPs/(n_SM R S), bytes_min/B_peak))
//            launch = T_launch (literal) or T_launch + L_alloc + L_dealloc
//            (measured: the persistent CTAs allocate TMEM once per launch)
//   T_store = L_TMA + 4 BM BN / B_TMA, plus 4 BM BN / B_drain (measured
//            reading) when the kernel keeps one accumulator buffer only, so
//            the next tile waits for the drain (two buffers overlap it)
// W_launch > 0 overrides the working set (a grouped launch passes its own);
// otherwise W = bytes_min of this GEMM (operands once, C once).  single >= 0
// overrides the buffering (a grouped launch passes the launch's); otherwise
// the tile's own.
template <class F>
__device__ __forceinline__ void gemm_forward(const pm_cfg& c, const ThetaT<F>& th, int n_sm, GemmFwdT<F>& f,
                                             F W_launch = F(-1), int single = -1) {
  const bool measured = th.reading == PM_READING_MEASURED;
  const int dt = c.dtype, g = c.cta_group;
  const F e = dt_bytes(dt), np = dt_passes(dt), l = dt_loads(dt);
  const F bytes_min = l * e * ((F)c.M * c.K + (F)c.N * c.K) + F(4) * (F)c.M * (F)c.N;
  f.ri = dt_rate(dt);
  f.R = th.v[f.ri];
  f.invR = th.inv[f.ri];
  const int64_t Kt = cdiv(c.K, c.BK);
  // CTA tiles: ceil(M/BM) ceil(N/BN) (literal); a pair covers 2 BM x BN (measured)
  const int64_t tiles = measured ? (int64_t)g * cdiv(c.M, (int64_t)g * c.BM) * cdiv(c.N, c.BN)
                                 : cdiv(c.M, c.BM) * cdiv(c.N, c.BN);
  // (pairs on fewer than two SMs are rejected by the callers; the guard keeps
  // the division defined)
  const int64_t n_conc = g == 1 ? n_sm : (n_sm >= 2 ? 2 * (n_sm / 2) : 1);
  int64_t waves;
  if (th.nc_nsm == n_sm && (uint64_t)tiles < 0x80000000ull) {
    const UDiv u = g == 1 ? th.nc[0] : th.nc[1];
    waves = (int64_t)udiv((uint32_t)tiles + (u.d - 1u), u);
  } else {
    waves = cdiv(tiles, n_conc);
  }
  f.Kt = count_to<F>(Kt);
  f.waves = count_to<F>(waves);
  // tile products in integers (exact: at most 2^25), one conversion each
  f.D = (F)(4 * (int)c.BM * (int)c.BN);
  // L_mma once per K-step (literal) or once per tcgen05.mma the K-step
  // issues, BK/k_instr per 128-row block per pass (measured)
  const int kin = dt == PM_FP32 ? 8 : (dt == PM_BF16 ? 16 : 32);
  f.n_instr = measured ? np * (F)((c.BK / kin) * ((c.BM + 127) / 128)) : F(1);
  f.DA_w = c.tmem_a ? l * e * c.BM * c.BK : F(0);
  f.DA_r = c.tmem_a ? np * e * c.BM * c.BK : F(0);
  // measured: strategy B's tcgen05.cp per 128-row x 32-byte A slice, each charged L_mma
  if (c.tmem_a && measured) f.n_instr += l * (F)(c.BK * (int)e / 32) * (F)((c.BM + 127) / 128);
  const F T_tmem = (f.D + f.DA_r) * th.inv[10] + f.n_instr * th.v[9] + (f.D + f.DA_w) * th.inv[11];
  const F T_mgmt = measured ? F(0) : th.v[13] / f.Kt;
  f.S = g == 1 ? F(1) : th.v[14];
  f.invS = g == 1 ? F(1) : th.inv[14];
  const int rows = (measured && g == 1 && c.BM < 128) ? 128 : (int)c.BM;
  f.X = (np * (F)(2 * rows * (int)c.BN * (int)c.BK)) * (f.invR * f.invS);
  f.T_c = f.X + T_tmem + T_mgmt;
  // BN / g: exact for the one- and two-SM tiles (power-of-two BN)
  const F bn_g = g == 1 ? (F)c.BN : (g == 2 ? F(0.5) * (F)c.BN : (F)c.BN / (F)g);
  f.bstep = g <= 2 ? l * e * (F)((int)c.BK * ((int)c.BM + ((int)c.BN >> (g - 1))))
                   : l * e * c.BK * ((F)c.BM + bn_g);
  // measured: B_TMA x rho(W), rho = 1 + (rho_L2 - 1) exp(-W/w0) (loads that
  // hit in L2 arrive faster, Sec. III-A.2; Eq. 16's blend shape); w0 <= 0
  // switches the blend off
  f.W = W_launch > F(0) ? W_launch : bytes_min;
  f.blend = measured && th.v[3] > F(0);
  f.E = f.blend ? pm_exp_fast(-f.W * th.inv[3]) : F(0);
  f.rho = f.blend ? F(1) + (th.v[16] - F(1)) * f.E : F(1);
  f.T_tma = th.v[4] + (f.blend ? pm_div_fast(f.bstep * th.inv[5], f.rho) : f.bstep * th.inv[5]);   // rho = 1 unblended
  const F T_sync = F(2) * th.v[12];
  // 1 - alpha = clamp(c_alpha / s, 0, 1) (literal) or clamp(c_alpha / (s - 1),
  // 0, 1) (measured: s - 1 loads in flight while one stage is consumed; a
  // single stage hides nothing)
  const F r = measured ? (c.stages > 1 ? div_stages_m1(th.v[15], c.stages, th) : F(1))
                       : div_stages(th.v[15], c.stages, th);
  f.oma_free = r > F(0) && r < F(1);
  f.oma = r <= F(0) ? F(0) : (r >= F(1) ? F(1) : r);
  f.T_io = measured ? f.oma * f.T_tma : f.oma * f.T_tma + T_sync;
  f.T_eq8 = pm_max(f.T_c, f.T_io) + T_sync;
  // measured: each stage cycles through its load, its MMAs and its full and
  // empty barriers, so s stages finish at most one K-step per cycle / s
  f.T_ring = measured ? div_stages(f.T_tma + f.T_c + T_sync, c.stages, th) : F(0);
  f.ring = measured && f.T_ring > f.T_eq8;
  f.T_step = f.ring ? f.T_ring : f.T_eq8;
  f.store_bytes = f.D;
  f.drain = measured && (single >= 0 ? single != 0
                                     : single_buffer(c.BM, c.BN, c.BK, c.stages, c.cta_group, c.dtype, c.tmem_a));
  f.T_store = th.v[4] + f.store_bytes * th.inv[5] + (f.drain ? f.store_bytes * th.inv[17] : F(0));
  f.launch = measured ? th.v[0] + th.v[13] : th.v[0];
  f.T_stage = f.launch + f.waves * (f.Kt * f.T_step + f.T_store);
  const F flops = np * F(2) * (F)c.M * (F)c.N * (F)c.K;
  f.A_rl = th.nc_nsm == n_sm ? flops * (f.invR * f.invS) * th.inv_nsm : flops * (f.invR * f.invS) / (F)n_sm;
  f.B_rl = bytes_min * th.inv[2];
  f.T_rl = f.launch + (f.A_rl >= f.B_rl ? f.A_rl : f.B_rl);
  f.T = f.T_stage >= f.T_rl ? f.T_stage : f.T_rl;
}

// Adjoint of one tile's K-steps and writeback, tau = K_tiles T_step + T_store
// scaled by the weights g_step (of T_step) and g_store (of T_store):
// d[j] += dtau/dtheta_j; the tensor-rate and S_2SM slopes go to gR and gS
// (the caller adds them to the right entries).  max() passes the gradient
// to its first argument on ties; the clamp stops it outside (0,1).
template <class F>
__device__ __forceinline__ void step_store_adjoint(const pm_cfg& c, const ThetaT<F>& th, const GemmFwdT<F>& f,
                                                   F g_step, F g_store, F (&d)[NP], F& gR, F& gS) {
  const bool measured = th.reading == PM_READING_MEASURED;
  d[4] += g_store;
  d[5] -= g_store * (f.store_bytes * th.inv[5]) * th.inv[5];
  if (f.drain) d[17] -= g_store * (f.store_bytes * th.inv[17]) * th.inv[17];
  // T_step = max(T_eq8, T_ring); ties to Eq. 8
  const F g_eq8 = f.ring ? F(0) : g_step;
  const F g_ring = f.ring ? div_stages(g_step, c.stages, th) : F(0);   // per term of the ring's cycle
  F g_sync = g_eq8 + g_ring;
  F g_c = g_ring, g_io = F(0);
  if (f.T_c >= f.T_io) g_c += g_eq8; else g_io = g_eq8;
  // T_io = oma * T_tma + T_sync
  if (!measured) g_sync += g_io;
  const F g_tma = g_io * f.oma + g_ring;
  if (f.oma_free)
    d[15] += measured ? div_stages_m1(g_io * f.T_tma, c.stages, th) : div_stages(g_io * f.T_tma, c.stages, th);
  d[4] += g_tma;
  const F t_bw = f.blend ? pm_div_fast(f.bstep * th.inv[5], f.rho) : f.bstep * th.inv[5];   // b_step / (B_TMA rho)
  d[5] -= g_tma * t_bw * th.inv[5];
  if (f.blend) {
    // rho = 1 + (rho_L2 - 1) E, E = exp(-W/w0)
    const F g_rho = -pm_div_fast(g_tma * t_bw, f.rho);
    d[16] += g_rho * f.E;
    d[3] += g_rho * (th.v[16] - F(1)) * f.E * (f.W * th.inv[3]) * th.inv[3];
  }
  d[12] += F(2) * g_sync;
  // T_c = X + (D + D_A,r)/BW_rd + n_instr L_mma + (D + D_A,w)/BW_wr + L_mgmt/K_tiles
  gR -= g_c * f.X * f.invR;
  gS -= g_c * f.X * f.invS;
  d[10] -= g_c * ((f.D + f.DA_r) * th.inv[10]) * th.inv[10];
  d[9] += g_c * f.n_instr;
  d[11] -= g_c * ((f.D + f.DA_w) * th.inv[11]) * th.inv[11];
  if (!measured) d[13] += g_c / f.Kt;
}

// Adds the tensor-rate and S_2SM slopes to their entries of d; static
// indices keep d[] in registers.
template <class F>
__device__ __forceinline__ void rate_adjoint(const pm_cfg& c, const GemmFwdT<F>& f, F gR, F gS, F (&d)[NP]) {
  d[6] += f.ri == 6 ? gR : F(0);
  d[7] += f.ri == 7 ? gR : F(0);
  d[8] += f.ri == 8 ? gR : F(0);
  if (c.cta_group == 2) d[14] += gS;
}

// Adjoint of gemm_forward: d[j] += w * dT_hat/dtheta_j.
template <class F>
__device__ __forceinline__ void gemm_adjoint(const pm_cfg& c, const ThetaT<F>& th, const GemmFwdT<F>& f, F w,
                                             F (&d)[NP]) {
  const bool measured = th.reading == PM_READING_MEASURED;
  F g_stage = F(0), g_rl = F(0);
  if (f.T_stage >= f.T_rl) g_stage = w; else g_rl = w;
  F gR = F(0), gS = F(0);
  // the launch term of both branches
  if (measured) d[13] += g_rl + g_stage;
  // roofline branch
  d[0] += g_rl;
  if (g_rl != F(0)) {
    if (f.A_rl >= f.B_rl) {
      gR -= g_rl * f.A_rl * f.invR;
      gS -= g_rl * f.A_rl * f.invS;
    } else {
      d[2] -= g_rl * f.B_rl * th.inv[2];
    }
  }
  // stage branch: launch + waves (K_tiles T_step + T_store)
  d[0] += g_stage;
  step_store_adjoint(c, th, f, g_stage * f.waves * f.Kt, g_stage * f.waves, d, gR, gS);
  rate_adjoint(c, f, gR, gS, d);
}

// Memory probes.  Copy/triad through Eq. 16 with W = beta bytes moved;
// TMA2D: tile latency plus ceil(tiles/SMs) tile round trips (Eq. 4),
// bounded below by the streaming time of Eq. 16.
template <class F>
struct ProbeFwdT {
  F T, T1, T2, Bw, E, W, beta, moved_tiles;
  bool blend;
};
using ProbeFwd = ProbeFwdT<float>;

template <class F>
__device__ __forceinline__ void probe_forward(const pm_cfg& c, const ThetaT<F>& th, int n_sm, ProbeFwdT<F>& f) {
  F W, t2num;
  if (c.kind == PM_KIND_COPY || c.kind == PM_KIND_TRIAD) {
    f.beta = (c.kind == PM_KIND_COPY ? F(8) : F(12)) * (F)c.M;
    W = f.beta;
    t2num = f.beta;
  } else {
    const F t = F(4) * c.BM * c.BN;
    const int64_t nt = cdiv(c.M, c.BM) * cdiv(c.N, c.BN);
    f.moved_tiles = (F)cdiv(nt, n_sm) * F(2) * t;
    f.beta = F(8) * (F)c.M * (F)c.N;
    W = f.beta;
    t2num = f.moved_tiles;
  }
  f.W = W;
  f.blend = th.v[3] > F(0);
  f.E = f.blend ? pm_exp(-W / th.v[3]) : F(0);
  f.Bw = f.blend ? th.v[1] + (th.v[2] - th.v[1]) * f.E : th.v[1];
  if (c.kind == PM_KIND_COPY || c.kind == PM_KIND_TRIAD) {
    f.T1 = th.v[0] + f.beta / f.Bw;
    f.T2 = th.v[0] + f.beta / th.v[2];
  } else {
    f.T1 = th.v[0] + th.v[4] + t2num / th.v[5];
    f.T2 = th.v[0] + f.beta / f.Bw;
  }
  f.T = f.T1 >= f.T2 ? f.T1 : f.T2;
}

template <class F>
__device__ __forceinline__ void bw_adjoint(const ThetaT<F>& th, const ProbeFwdT<F>& f, F gB, F (&d)[NP]) {
  if (f.blend) {
    d[1] += gB * (F(1) - f.E);
    d[2] += gB * f.E;
    const F gE = gB * (th.v[2] - th.v[1]);
    d[3] += gE * f.E * f.W / (th.v[3] * th.v[3]);
  } else {
    d[1] += gB;
  }
}

template <class F>
__device__ __forceinline__ void probe_adjoint(const pm_cfg& c, const ThetaT<F>& th, const ProbeFwdT<F>& f, F w,
                                              F (&d)[NP]) {
  d[0] += w;
  const bool first = f.T1 >= f.T2;
  if (c.kind == PM_KIND_COPY || c.kind == PM_KIND_TRIAD) {
    if (first) bw_adjoint(th, f, -w * f.beta / (f.Bw * f.Bw), d);
    else d[2] -= w * f.beta / (th.v[2] * th.v[2]);
  } else {
    if (first) {
      d[4] += w;
      d[5] -= w * f.moved_tiles / (th.v[5] * th.v[5]);
    } else {
      bw_adjoint(th, f, -w * f.beta / (f.Bw * f.Bw), d);
    }
  }
}

// A record the model can evaluate on n_sm SMs; a CTA pair (cta_group 2)
// needs two SMs (Sec. III-A.4), so on one SM a pair record has no time.
__device__ __forceinline__ bool cfg_sane(const pm_cfg& c, int n_sm) {
  if (c.kind == PM_KIND_GEMM)
    return c.M > 0 && c.N > 0 && c.K > 0 && c.BM > 0 && c.BN > 0 && c.BK > 0 && c.stages > 0 &&
           (c.cta_group == 1 || (c.cta_group == 2 && n_sm >= 2)) && c.dtype >= 0 && c.dtype <= 2 &&
           (c.tmem_a == 0 || c.tmem_a == 1);
  if (c.kind == PM_KIND_COPY || c.kind == PM_KIND_TRIAD) return c.M > 0;
  if (c.kind == PM_KIND_TMA2D) return c.M > 0 && c.N > 0 && c.BM > 0 && c.BN > 0;
  return false;
}

__device__ __forceinline__ pm_cfg load_cfg(const pm_cfg* p) {
  // 24-byte record as three 8-byte loads
  const int2* q = reinterpret_cast<const int2*>(p);
  int2 a = __ldg(q), b = __ldg(q + 1), cc = __ldg(q + 2);
  pm_cfg c;
  int2* o = reinterpret_cast<int2*>(&c);
  o[0] = a; o[1] = b; o[2] = cc;
  return c;
}

// Six blocks per SM (40 registers, no spills): 48 warps hide the latency of
// the dependent FP32 chain better than the 40 of the unbounded 47-register
// build (10-20 % more configurations per second).
__global__ void __launch_bounds__(256, 6) model_predict_kernel(const pm_cfg* __restrict__ cfgs, int64_t n, Theta th,
                                                            int n_sm, float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const pm_cfg c = load_cfg(cfgs + i);
    float t;
    if (!cfg_sane(c, n_sm)) {
      t = __int_as_float(0x7fc00000);
    } else if (c.kind == PM_KIND_GEMM) {
      GemmFwd f;
      gemm_forward(c, th, n_sm, f);
      t = f.T;
    } else {
      ProbeFwd f;
      probe_forward(c, th, n_sm, f);
      t = f.T;
    }
    out[i] = t;
  }
}

// Loss and gradient: per-thread terms and warp sums in F, warp totals
// combined in FP64 into one partial record of NREC values per block; a
// second kernel adds the records in block order (deterministic).
constexpr int kGradThreads = 256;

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) { return warp_sum<double>(v); }

// F = float: per-configuration FP32 terms (throughput path); F = double: the
// whole evaluation in FP64 so the calibration's line searches see a smooth
// objective.  The FP32 kernel is held to four blocks per SM (64 registers,
// 32 warps to hide the dependent-instruction latency; 19 % faster than the
// 78-register build at three); the FP64 one at two (128 registers).
template <class F>
constexpr int grad_min_blocks() { return sizeof(F) == 4 ? 4 : 2; }

template <class F>
__global__ void __launch_bounds__(kGradThreads, grad_min_blocks<F>()) model_grad_kernel(const pm_cfg* __restrict__ cfgs, int64_t n,
                                                                  ThetaT<F> th, int n_sm,
                                                                  const F* __restrict__ t_meas,
                                                                  double* __restrict__ partials) {
  F acc[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) acc[j] = F(0);
  F loss = F(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const pm_cfg c = load_cfg(cfgs + i);
    F d[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) d[j] = F(0);
    F T;
    if (!cfg_sane(c, n_sm)) {
      T = (F)__int_as_float(0x7fc00000);
    } else if (c.kind == PM_KIND_GEMM) {
      GemmFwdT<F> f;
      gemm_forward(c, th, n_sm, f);
      T = f.T;
      gemm_adjoint(c, th, f, F(1), d);
    } else {
      ProbeFwdT<F> f;
      probe_forward(c, th, n_sm, f);
      T = f.T;
      probe_adjoint(c, th, f, F(1), d);
    }
    const F r = pm_log(T) - pm_log(__ldg(t_meas + i));
    loss = fma(r, r, loss);
    const F w = F(2) * r / T;
#pragma unroll
    for (int j = 0; j < NP; ++j) acc[j] = fma(w, d[j], acc[j]);
  }
  // warp sums in F (FP64 arithmetic is scarce on this GPU), warp totals
  // combined in FP64
  __shared__ double red[kGradThreads / 32][NREC];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  F v = warp_sum<F>(loss);
  if (lane == 0) red[warp][0] = (double)v;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    v = warp_sum<F>(acc[j]);
    if (lane == 0) red[warp][j + 1] = (double)v;
  }
  __syncthreads();
  if (threadIdx.x < NREC) {
    double s = 0.0;
    for (int w = 0; w < kGradThreads / 32; ++w) s += red[w][threadIdx.x];
    partials[(int64_t)blockIdx.x * NREC + threadIdx.x] = s;
  }
}

// Warp j sums component j of the block records: lane l adds records l,
// l+32, ... in order, then a fixed butterfly combines the lanes, so the
// result depends only on the number of records (deterministic).
__global__ void __launch_bounds__(NREC * 32) model_grad_finish_kernel(const double* __restrict__ partials,
                                                                    int blocks, int64_t n,
                                                                    double* __restrict__ out) {
  const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double s = 0.0;
#pragma unroll 4
  for (int b = lane; b < blocks; b += 32) s += partials[(int64_t)b * NREC + j];
  s = warp_sum_d(s);
  if (lane == 0) out[j] = s / (double)n;
}

static int grad_blocks(int64_t n) {
  const int64_t want = (n + kGradThreads - 1) / kGradThreads;
  const int cap = std::max(1, sm_count()) * 4;             // one wave: four blocks per SM (launch bound)
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, cap));
}

// Autotuner: one block per shape, thread t evaluates tile configuration t of
// the 180-point space in lexicographic (BM, BN, BK, stages, cta_group) order.
constexpr int kTuneThreads = 192;

__device__ __forceinline__ void decode_tile(int t, int dt, int& BM, int& BN, int& BK, int& s, int& g) {
  BM = kBM[t / 60];
  BN = kBN[(t / 20) % 3];
  BK = kBK[dt][(t / 10) % 2];
  s = 2 + (t / 2) % 5;
  g = 1 + t % 2;
}

__global__ void __launch_bounds__(kTuneThreads) autotune_kernel(const int32_t* __restrict__ MNK, int64_t n, int dt,
                                                                Theta th, int n_sm, pm_cfg* __restrict__ picks,
                                                                float* __restrict__ t_pred) {
  __shared__ float sv[kTuneThreads / 32];
  __shared__ int si[kTuneThreads / 32];
  const int t = threadIdx.x;
  for (int64_t shape = blockIdx.x; shape < n; shape += gridDim.x) {
    pm_cfg c;
    c.M = __ldg(MNK + 3 * shape);
    c.N = __ldg(MNK + 3 * shape + 1);
    c.K = __ldg(MNK + 3 * shape + 2);
    c.dtype = (int8_t)dt;
    c.kind = PM_KIND_GEMM;
    c.tmem_a = 0;
    float v = INFINITY;
    int BM = 0, BN = 0, BK = 0, s = 0, g = 0;
    if (t < 180) {
      decode_tile(t, dt, BM, BN, BK, s, g);
      if (tile_valid(BM, BN, BK, s, g, dt) && (g == 1 || n_sm >= 2) && c.M > 0 && c.N > 0 && c.K > 0) {
        c.BM = (int16_t)BM; c.BN = (int16_t)BN; c.BK = (int16_t)BK;
        c.stages = (int8_t)s; c.cta_group = (int8_t)g;
        GemmFwd f;
        gemm_forward(c, th, n_sm, f);
        v = f.T;
      }
    }
    // argmin, ties to the lower index
    int idx = t;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (ov < v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    if ((t & 31) == 0) { sv[t >> 5] = v; si[t >> 5] = idx; }
    __syncthreads();
    if (t == 0) {
      float bv = sv[0];
      int bi = si[0];
      for (int w = 1; w < kTuneThreads / 32; ++w)
        if (sv[w] < bv || (sv[w] == bv && si[w] < bi)) { bv = sv[w]; bi = si[w]; }
      pm_cfg p = c;
      if (bv < INFINITY) {
        decode_tile(bi, dt, BM, BN, BK, s, g);
        p.BM = (int16_t)BM; p.BN = (int16_t)BN; p.BK = (int16_t)BK;
        p.stages = (int8_t)s; p.cta_group = (int8_t)g;
      } else {
        p.BM = p.BN = p.BK = 0; p.stages = p.cta_group = 0;
      }
      picks[shape] = p;
      t_pred[shape] = bv;
    }
    __syncthreads();
  }
}

// Top-k variant: the k predicted-fastest valid configurations per shape, in
// increasing predicted time (ties to the lower index), by k rounds of block
// argmin over the 180 candidates.
constexpr int kMaxTopK = 16;

__global__ void __launch_bounds__(kTuneThreads) autotune_topk_kernel(const int32_t* __restrict__ MNK, int64_t n,
                                                                     int dt, Theta th, int n_sm, int k,
                                                                     pm_cfg* __restrict__ picks,
                                                                     float* __restrict__ t_pred) {
  __shared__ float sv[kTuneThreads / 32];
  __shared__ int si[kTuneThreads / 32];
  __shared__ int chosen;
  const int t = threadIdx.x;
  for (int64_t shape = blockIdx.x; shape < n; shape += gridDim.x) {
    pm_cfg c;
    c.M = __ldg(MNK + 3 * shape);
    c.N = __ldg(MNK + 3 * shape + 1);
    c.K = __ldg(MNK + 3 * shape + 2);
    c.dtype = (int8_t)dt;
    c.kind = PM_KIND_GEMM;
    c.tmem_a = 0;
    float mine = INFINITY;
    int BM = 0, BN = 0, BK = 0, s = 0, g = 0;
    if (t < 180) {
      decode_tile(t, dt, BM, BN, BK, s, g);
      if (tile_valid(BM, BN, BK, s, g, dt) && (g == 1 || n_sm >= 2) && c.M > 0 && c.N > 0 && c.K > 0) {
        c.BM = (int16_t)BM; c.BN = (int16_t)BN; c.BK = (int16_t)BK;
        c.stages = (int8_t)s; c.cta_group = (int8_t)g;
        GemmFwd f;
        gemm_forward(c, th, n_sm, f);
        mine = f.T;
      }
    }
    for (int r = 0; r < k; ++r) {
      float v = mine;
      int idx = t;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov < v || (ov == v && oi < idx)) { v = ov; idx = oi; }
      }
      if ((t & 31) == 0) { sv[t >> 5] = v; si[t >> 5] = idx; }
      __syncthreads();
      if (t == 0) {
        float bv = sv[0];
        int bi = si[0];
        for (int w = 1; w < kTuneThreads / 32; ++w)
          if (sv[w] < bv || (sv[w] == bv && si[w] < bi)) { bv = sv[w]; bi = si[w]; }
        pm_cfg p = c;
        if (bv < INFINITY) {
          decode_tile(bi, dt, BM, BN, BK, s, g);
          p.BM = (int16_t)BM; p.BN = (int16_t)BN; p.BK = (int16_t)BK;
          p.stages = (int8_t)s; p.cta_group = (int8_t)g;
        } else {
          p.BM = p.BN = p.BK = 0; p.stages = p.cta_group = 0;
        }
        picks[shape * k + r] = p;
        t_pred[shape * k + r] = bv;
        chosen = bv < INFINITY ? bi : -1;
      }
      __syncthreads();
      if (t == chosen) mine = INFINITY;
      __syncthreads();
    }
  }
}

// Grouped launches.  The kernel's static schedule (pm_grouped_gemm_run):
// with several groups the launch lists them largest tile (BM x BN) first,
// ties in the caller's order, and deals the listed tiles to the n_conc
// workers round by round, reversing the worker order on odd rounds; one
// group is dealt plainly round by round.  A group-q tile costs
//   tau_q = K_tiles T_step_q + T_store_q
// with that group's (BM, BN) and the launch's (BK, stages, cta_group), and
// the launch ends with its busiest worker:
//   T_hat = launch + max_w sum_q n_{w,q} tau_q.
constexpr int kGroupThreads = 256;
constexpr int kMaxGroups = 1024;

__device__ __forceinline__ int64_t count_congruent(int64_t X, int64_t w, int64_t n) {
  // number of t in [0, X] with t = w (mod n), for X >= -1
  return X < w ? 0 : (X - w) / n + 1;
}

// How many of the listed positions [a, b) are dealt to worker w of n.
// Reversing odd rounds gives position i to worker w exactly when
// i mod 2n is w or 2n - 1 - w.
__device__ __forceinline__ int64_t dealt(int64_t a, int64_t b, int64_t w, int64_t n, bool reverse_odd) {
  if (!reverse_odd) return count_congruent(b - 1, w, n) - count_congruent(a - 1, w, n);
  const int64_t p = 2 * n, w2 = p - 1 - w;
  return count_congruent(b - 1, w, p) - count_congruent(a - 1, w, p) + count_congruent(b - 1, w2, p) -
         count_congruent(a - 1, w2, p);
}

// Working set of a grouped launch (every group's A rows, its B and its C),
// for the L2 residency of the TMA loads; called by all threads of a block.
template <class F>
__device__ F grouped_working_set(const int32_t* Mg, int G, int N, int K, int dt) {
  __shared__ unsigned long long sum_m;
  if (threadIdx.x == 0) sum_m = 0ull;
  __syncthreads();
  unsigned long long mine = 0ull;
  for (int q = threadIdx.x; q < G; q += blockDim.x) mine += (unsigned long long)Mg[q];
  atomicAdd(&sum_m, mine);
  __syncthreads();
  const F sm = (F)sum_m;
  __syncthreads();
  return (F)dt_loads(dt) * (F)dt_bytes(dt) * (sm * (F)K + (F)G * (F)N * (F)K) + F(4) * sm * (F)N;
}

// The launch's list of groups: list[i] = the group at position i, off[i] =
// its first tile; tiles[q] = group q's tiles.  Largest tile area first
// (area / 4096 = 2^class, class 0..4; a group without a valid tile, area 0,
// last), ties in the caller's order.  Called by all threads.
__device__ void grouped_list(const int16_t* bm, const int16_t* bn, const int64_t* tiles, int G, int16_t* list,
                             int64_t* off) {
  if (threadIdx.x == 0) {
    int k = 0;
    if (G > 1) {
      for (int cls = 4; cls >= -1; --cls)
        for (int q = 0; q < G; ++q)
          if (__ffs(((int)bm[q] * (int)bn[q]) >> 12) - 1 == cls) list[k++] = (int16_t)q;
    } else {
      list[0] = 0;
    }
    off[0] = 0;
    for (int i = 0; i < G; ++i) off[i + 1] = off[i] + tiles[list[i]];
  }
  __syncthreads();
}

// Busiest worker's time and (in *w_star) the first worker that has it;
// busy_w adds n_{w,q} tau_q over the list in order.  Called by all threads;
// the result is valid in every thread.
template <class F>
__device__ F grouped_makespan(const F* tau, const int16_t* list, const int64_t* off, int G, int64_t n_conc,
                              int* w_star) {
  __shared__ F red_v[kGroupThreads / 32];
  __shared__ int red_i[kGroupThreads / 32];
  const bool rev = G > 1;
  F mx = F(-1);
  int mi = 0x7fffffff;
  for (int64_t w = threadIdx.x; w < n_conc; w += blockDim.x) {
    F busy = F(0);
    for (int i = 0; i < G; ++i) {
      const int64_t cnt = dealt(off[i], off[i + 1], w, n_conc, rev);
      if (cnt) busy += (F)cnt * tau[list[i]];
    }
    if (busy > mx) { mx = busy; mi = (int)w; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const F ov = __shfl_xor_sync(0xffffffffu, mx, o);
    const int oi = __shfl_xor_sync(0xffffffffu, mi, o);
    if (ov > mx || (ov == mx && oi < mi)) { mx = ov; mi = oi; }
  }
  if ((threadIdx.x & 31) == 0) { red_v[threadIdx.x >> 5] = mx; red_i[threadIdx.x >> 5] = mi; }
  __syncthreads();
  F m = red_v[0];
  int i0 = red_i[0];
  for (int w = 1; w < (int)(blockDim.x / 32); ++w)
    if (red_v[w] > m || (red_v[w] == m && red_i[w] < i0)) { m = red_v[w]; i0 = red_i[w]; }
  __syncthreads();
  if (w_star) *w_star = i0;
  return m;
}

template <class F>
__device__ __forceinline__ int64_t launch_tiles(const ThetaT<F>& th, int M, int N, int BM, int BN, int g) {
  return th.reading == PM_READING_MEASURED ? (int64_t)g * cdiv(M, (int64_t)g * BM) * cdiv(N, BN)
                                           : cdiv(M, BM) * cdiv(N, BN);
}

template <class F>
__device__ __forceinline__ F launch_time(const ThetaT<F>& th) {
  return th.reading == PM_READING_MEASURED ? th.v[0] + th.v[13] : th.v[0];
}

// Grouped autotuner: block b handles launch-level combination b =
// (BK index, stages, cta_group) in lexicographic order; threads pick each
// group's (BM, BN) minimising tiles x tau, then the makespan of the launch's
// schedule is evaluated.
__global__ void __launch_bounds__(kGroupThreads) grouped_tune_kernel(const int32_t* __restrict__ Mg, int G, int N,
                                                                     int K, int dt, Theta th, int n_sm,
                                                                     float* __restrict__ out_t,
                                                                     int16_t* __restrict__ out_bm,
                                                                     int16_t* __restrict__ out_bn) {
  __shared__ float tau[kMaxGroups];
  __shared__ int64_t tiles[kMaxGroups];
  __shared__ int64_t off[kMaxGroups + 1];
  __shared__ int16_t bm_s[kMaxGroups], bn_s[kMaxGroups], list[kMaxGroups];
  const int combo = blockIdx.x;                 // 0..19
  const int BK = kBK[dt][combo / 10];
  const int s = 2 + (combo / 2) % 5;
  const int g = 1 + combo % 2;
  const float W = grouped_working_set<float>(Mg, G, N, K, dt);
  bool any_invalid = false;
  for (int q = threadIdx.x; q < G; q += blockDim.x) {
    float best = INFINITY;
    int bm = 0, bn = 0;
    float btau = 0.f;
    int64_t btiles = 0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const int BM = kBM[a], BN = kBN[b];
        if (!tile_valid(BM, BN, BK, s, g, dt)) continue;
        pm_cfg c;
        c.M = Mg[q]; c.N = N; c.K = K; c.BM = (int16_t)BM; c.BN = (int16_t)BN; c.BK = (int16_t)BK;
        c.stages = (int8_t)s; c.cta_group = (int8_t)g; c.dtype = (int8_t)dt; c.kind = 0; c.tmem_a = 0;
        GemmFwd f;
        gemm_forward(c, th, n_sm, f, W);
        const float tq = f.Kt * f.T_step + f.T_store;   // one tile of this group
        const int64_t nt = launch_tiles(th, c.M, N, BM, BN, g);
        const float cost = (float)nt * tq;
        if (cost < best) { best = cost; bm = BM; bn = BN; btau = tq; btiles = nt; }
      }
    if (best == INFINITY) any_invalid = true;
    // each group's own tile decides its buffering here; the launch's rule is
    // applied below
    tau[q] = btau;
    tiles[q] = btiles;
    bm_s[q] = (int16_t)bm;
    bn_s[q] = (int16_t)bn;
    out_bm[combo * G + q] = (int16_t)bm;
    out_bn[combo * G + q] = (int16_t)bn;
  }
  any_invalid = __syncthreads_or(any_invalid);
  // the launch keeps one accumulator buffer if any group's tile needs it
  // (measured reading): every other group's tile then pays its drain too
  bool single = false;
  for (int q = threadIdx.x; q < G; q += blockDim.x)
    single = single || (bm_s[q] > 0 && single_buffer(bm_s[q], bn_s[q], BK, s, g, dt, 0));
  single = __syncthreads_or(single);
  if (single && th.reading == PM_READING_MEASURED)
    for (int q = threadIdx.x; q < G; q += blockDim.x)
      if (bm_s[q] > 0 && !single_buffer(bm_s[q], bn_s[q], BK, s, g, dt, 0))
        tau[q] += 4.0f * (float)bm_s[q] * (float)bn_s[q] * th.inv[17];
  __syncthreads();
  grouped_list(bm_s, bn_s, tiles, G, list, off);
  const float t = grouped_makespan<float>(tau, list, off, G, g == 1 ? n_sm : 2 * (n_sm / 2), nullptr);
  if (threadIdx.x == 0)
    out_t[combo] = (any_invalid || (g != 1 && n_sm < 2)) ? INFINITY : launch_time(th) + t;
}

// Stage-model makespan of one grouped launch with given per-group tiles (the
// schedule of pm_grouped_gemm_run; same terms as the grouped autotuner), in
// F; with grad != nullptr also its gradient in theta (out: T_hat, then NP
// slopes): the busiest worker's tiles through the tile adjoint.
template <class F>
__global__ void __launch_bounds__(kGroupThreads) grouped_predict_kernel(const int32_t* __restrict__ Mg,
                                                                        const int16_t* __restrict__ BMg,
                                                                        const int16_t* __restrict__ BNg, int G, int N,
                                                                        int K, int BK, int s, int g, int dt,
                                                                        ThetaT<F> th, int n_sm, bool grad,
                                                                        F* __restrict__ out) {
  __shared__ F tau[kMaxGroups];
  __shared__ int64_t tiles[kMaxGroups];
  __shared__ int64_t off[kMaxGroups + 1];
  __shared__ int16_t list[kMaxGroups], pos[kMaxGroups];
  __shared__ F red_d[kGroupThreads / 32][NP];
  const F W = grouped_working_set<F>(Mg, G, N, K, dt);
  const int64_t n_conc = g == 1 ? n_sm : 2 * (n_sm / 2);
  // one accumulator buffer for the whole launch if any group's tile needs it
  bool single = false;
  for (int q = threadIdx.x; q < G; q += blockDim.x) single = single || single_buffer(BMg[q], BNg[q], BK, s, g, dt, 0);
  const int sb = __syncthreads_or(single) ? 1 : 0;
  for (int q = threadIdx.x; q < G; q += blockDim.x) {
    pm_cfg c;
    c.M = Mg[q]; c.N = N; c.K = K; c.BM = BMg[q]; c.BN = BNg[q]; c.BK = (int16_t)BK;
    c.stages = (int8_t)s; c.cta_group = (int8_t)g; c.dtype = (int8_t)dt; c.kind = 0; c.tmem_a = 0;
    GemmFwdT<F> f;
    gemm_forward(c, th, n_sm, f, W, sb);
    tau[q] = f.Kt * f.T_step + f.T_store;
    tiles[q] = launch_tiles(th, c.M, N, c.BM, c.BN, g);
  }
  __syncthreads();
  grouped_list(BMg, BNg, tiles, G, list, off);
  int w_star = 0;
  const F t = grouped_makespan<F>(tau, list, off, G, n_conc, &w_star);
  const bool none = g != 1 && n_sm < 2;
  if (threadIdx.x == 0) out[0] = none ? (F)__int_as_float(0x7fc00000) : launch_time(th) + t;
  if (!grad) return;
  for (int i = threadIdx.x; i < G; i += blockDim.x) pos[list[i]] = (int16_t)i;
  __syncthreads();
  // d T_hat = d launch + sum_q n_{w*,q} d tau_q
  F d[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) d[j] = F(0);
  for (int q = threadIdx.x; q < G; q += blockDim.x) {
    const int64_t cnt = dealt(off[pos[q]], off[pos[q] + 1], w_star, n_conc, G > 1);
    if (!cnt) continue;
    pm_cfg c;
    c.M = Mg[q]; c.N = N; c.K = K; c.BM = BMg[q]; c.BN = BNg[q]; c.BK = (int16_t)BK;
    c.stages = (int8_t)s; c.cta_group = (int8_t)g; c.dtype = (int8_t)dt; c.kind = 0; c.tmem_a = 0;
    GemmFwdT<F> f;
    gemm_forward(c, th, n_sm, f, W, sb);
    F gR = F(0), gS = F(0);
    step_store_adjoint(c, th, f, (F)cnt * f.Kt, (F)cnt, d, gR, gS);
    rate_adjoint(c, f, gR, gS, d);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const F v = warp_sum<F>(d[j]);
    if (lane == 0) red_d[warp][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < NP) {
    F v = F(0);
    for (int w = 0; w < kGroupThreads / 32; ++w) v += red_d[w][threadIdx.x];
    if (threadIdx.x == 0) v += F(1);                                           // T_launch
    if (threadIdx.x == 13 && th.reading == PM_READING_MEASURED) v += F(1);     // L_alloc + L_dealloc
    out[1 + threadIdx.x] = none ? (F)__int_as_float(0x7fc00000) : v;
  }
}

static std::atomic<int> g_reading{PM_READING_MEASURED};

static Theta to_theta(const pm_params* p, int n_sm) {
  Theta t;
  for (int j = 0; j < NP; ++j) {
    t.v[j] = p->v[j];
    t.inv[j] = (float)(1.0 / (double)p->v[j]);
  }
  t.reading = g_reading.load();
  set_concurrency(t, n_sm);
  return t;
}

}  // namespace pm

using namespace pm;

extern "C" pm_status pm_model_predict(const pm_cfg* cfgs_dev, int64_t n, const pm_params* theta_host, int32_t n_sm,
                                      float* t_out_dev, void* stream) {
  PM_REQUIRE(n >= 0, PM_EINVAL, "n < 0");
  if (n == 0) return PM_OK;
  PM_REQUIRE(cfgs_dev && theta_host && t_out_dev && n_sm > 0, PM_EINVAL, "null pointer or n_sm <= 0");
  PM_REQUIRE(((uintptr_t)cfgs_dev & 7) == 0, PM_EINVAL, "cfgs_dev must be 8-byte aligned");
  const int64_t want = (n + 255) / 256;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)std::max(1, sm_count()) * 16));
  model_predict_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(cfgs_dev, n, to_theta(theta_host, n_sm),
                                                                            n_sm, t_out_dev);
  return launch_status("model_predict_kernel");
}

extern "C" pm_status pm_model_grad_workspace(int64_t n, size_t* bytes) {
  PM_REQUIRE(bytes != nullptr && n >= 0, PM_EINVAL, "bad arguments");
  *bytes = (size_t)grad_blocks(std::max<int64_t>(n, 1)) * NREC * sizeof(double);
  return PM_OK;
}

extern "C" pm_status pm_model_grad(const pm_cfg* cfgs_dev, int64_t n, const pm_params* theta_host, int32_t n_sm,
                                   const float* t_meas_dev, void* workspace_dev, size_t workspace_bytes,
                                   double* out_dev, void* stream) {
  PM_REQUIRE(n > 0, PM_EINVAL, "n must be positive");
  PM_REQUIRE(cfgs_dev && theta_host && t_meas_dev && workspace_dev && out_dev && n_sm > 0, PM_EINVAL,
             "null pointer or n_sm <= 0");
  PM_REQUIRE(((uintptr_t)cfgs_dev & 7) == 0 && ((uintptr_t)workspace_dev & 7) == 0, PM_EINVAL,
             "cfgs_dev and workspace_dev must be 8-byte aligned");
  const int blocks = grad_blocks(n);
  PM_REQUIRE(workspace_bytes >= (size_t)blocks * NREC * sizeof(double), PM_ENOMEM,
             "workspace of %zu bytes is smaller than the %zu needed", workspace_bytes,
             (size_t)blocks * NREC * sizeof(double));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  model_grad_kernel<float><<<blocks, kGradThreads, 0, s>>>(cfgs_dev, n, to_theta(theta_host, n_sm), n_sm, t_meas_dev,
                                                           static_cast<double*>(workspace_dev));
  pm_status st = launch_status("model_grad_kernel");
  if (st != PM_OK) return st;
  model_grad_finish_kernel<<<1, NREC * 32, 0, s>>>(static_cast<const double*>(workspace_dev), blocks, n, out_dev);
  return launch_status("model_grad_finish_kernel");
}

extern "C" pm_status pm_model_grad_f64(const pm_cfg* cfgs_dev, int64_t n, const double* theta_host, int32_t n_sm,
                                       const double* t_meas_dev, void* workspace_dev, size_t workspace_bytes,
                                       double* out_dev, void* stream) {
  PM_REQUIRE(n > 0, PM_EINVAL, "n must be positive");
  PM_REQUIRE(cfgs_dev && theta_host && t_meas_dev && workspace_dev && out_dev && n_sm > 0, PM_EINVAL,
             "null pointer or n_sm <= 0");
  PM_REQUIRE(((uintptr_t)cfgs_dev & 7) == 0 && ((uintptr_t)workspace_dev & 7) == 0 && ((uintptr_t)t_meas_dev & 7) == 0,
             PM_EINVAL, "cfgs_dev, t_meas_dev and workspace_dev must be 8-byte aligned");
  const int blocks = grad_blocks(n);
  PM_REQUIRE(workspace_bytes >= (size_t)blocks * NREC * sizeof(double), PM_ENOMEM,
             "workspace of %zu bytes is smaller than the %zu needed", workspace_bytes,
             (size_t)blocks * NREC * sizeof(double));
  ThetaT<double> th;
  for (int j = 0; j < NP; ++j) {
    th.v[j] = theta_host[j];
    th.inv[j] = 1.0 / theta_host[j];
  }
  th.reading = g_reading.load();
  set_concurrency(th, n_sm);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  model_grad_kernel<double><<<blocks, kGradThreads, 0, s>>>(cfgs_dev, n, th, n_sm, t_meas_dev,
                                                            static_cast<double*>(workspace_dev));
  pm_status st = launch_status("model_grad_kernel");
  if (st != PM_OK) return st;
  model_grad_finish_kernel<<<1, NREC * 32, 0, s>>>(static_cast<const double*>(workspace_dev), blocks, n, out_dev);
  return launch_status("model_grad_finish_kernel");
}

extern "C" pm_status pm_model_set_reading(int32_t reading) {
  PM_REQUIRE(reading == PM_READING_LITERAL || reading == PM_READING_MEASURED, PM_EINVAL,
             "reading %d is not a pm_reading", reading);
  g_reading.store(reading);
  return PM_OK;
}

extern "C" int32_t pm_model_reading(void) { return g_reading.load(); }

extern "C" pm_status pm_autotune_pick(const int32_t* MNK_dev, int64_t n, int32_t dtype, const pm_params* theta_host,
                                      int32_t n_sm, pm_cfg* picks_dev, float* t_pred_dev, void* stream) {
  PM_REQUIRE(n >= 0, PM_EINVAL, "n < 0");
  if (n == 0) return PM_OK;
  PM_REQUIRE(MNK_dev && theta_host && picks_dev && t_pred_dev && n_sm > 0, PM_EINVAL, "null pointer or n_sm <= 0");
  PM_REQUIRE(dtype >= 0 && dtype <= 2, PM_EINVAL, "dtype %d is not a pm_dtype", dtype);
  const int grid = (int)std::min<int64_t>(n, (int64_t)std::max(1, sm_count()) * 16);
  autotune_kernel<<<grid, kTuneThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      MNK_dev, n, dtype, to_theta(theta_host, n_sm), n_sm, picks_dev, t_pred_dev);
  return launch_status("autotune_kernel");
}

extern "C" pm_status pm_autotune_topk(const int32_t* MNK_dev, int64_t n, int32_t dtype, const pm_params* theta_host,
                                      int32_t n_sm, int32_t k, pm_cfg* picks_dev, float* t_pred_dev, void* stream) {
  PM_REQUIRE(n >= 0, PM_EINVAL, "n < 0");
  if (n == 0) return PM_OK;
  PM_REQUIRE(MNK_dev && theta_host && picks_dev && t_pred_dev && n_sm > 0, PM_EINVAL, "null pointer or n_sm <= 0");
  PM_REQUIRE(dtype >= 0 && dtype <= 2, PM_EINVAL, "dtype %d is not a pm_dtype", dtype);
  PM_REQUIRE(k >= 1 && k <= kMaxTopK, PM_EINVAL, "k must be in [1, %d]", kMaxTopK);
  const int grid = (int)std::min<int64_t>(n, (int64_t)std::max(1, sm_count()) * 16);
  autotune_topk_kernel<<<grid, kTuneThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      MNK_dev, n, dtype, to_theta(theta_host, n_sm), n_sm, k, picks_dev, t_pred_dev);
  return launch_status("autotune_topk_kernel");
}

namespace pm {

// All 20 launch-level candidates (BK, stages, cta_group) of the grouped
// autotuner: predicted makespan ht[i] and per-group tiles hbm/hbn[i * G + q].
static pm_status grouped_candidates(int32_t G, const int32_t* M_host, int32_t N, int32_t K, int32_t dtype,
                                    const pm_params* theta_host, int32_t n_sm, cudaStream_t s, float* ht,
                                    std::vector<int16_t>& hbm, std::vector<int16_t>& hbn) {
  PM_REQUIRE(G > 0 && G <= kMaxGroups, PM_EINVAL, "G must be in [1, %d]", kMaxGroups);
  PM_REQUIRE(M_host && theta_host && n_sm > 0, PM_EINVAL, "null pointer or n_sm <= 0");
  PM_REQUIRE(N > 0 && K > 0 && dtype >= 0 && dtype <= 2, PM_EINVAL, "bad N, K or dtype");
  for (int q = 0; q < G; ++q) PM_REQUIRE(M_host[q] > 0, PM_EINVAL, "M[%d] <= 0", q);
  // device scratch: M (G int32), t (20 floats), bm/bn (20 x G int16 each)
  const size_t bytes = 256 + G * 4 + 20 * 4 + 2 * 20 * (size_t)G * 2 + 16;
  char* buf = nullptr;
  PM_CUDA(cudaMallocAsync((void**)&buf, bytes, s));
  int32_t* dM = (int32_t*)buf;
  float* dt = (float*)(buf + ((G * 4 + 15) & ~15));
  int16_t* dbm = (int16_t*)((char*)dt + 96);
  int16_t* dbn = dbm + 20 * G;
  hbm.assign(20 * (size_t)G, 0);
  hbn.assign(20 * (size_t)G, 0);
  pm_status st = PM_OK;
  cudaError_t e = cudaMemcpyAsync(dM, M_host, G * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    grouped_tune_kernel<<<20, kGroupThreads, 0, s>>>(dM, G, N, K, dtype, to_theta(theta_host, n_sm), n_sm, dt, dbm, dbn);
    st = launch_status("grouped_tune_kernel");
    if (st == PM_OK) e = cudaMemcpyAsync(ht, dt, 20 * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (st == PM_OK && e == cudaSuccess)
      e = cudaMemcpyAsync(hbm.data(), dbm, hbm.size() * 2, cudaMemcpyDeviceToHost, s);
    if (st == PM_OK && e == cudaSuccess)
      e = cudaMemcpyAsync(hbn.data(), dbn, hbn.size() * 2, cudaMemcpyDeviceToHost, s);
  }
  cudaFreeAsync(buf, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (st != PM_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "grouped autotune copies");
  return PM_OK;
}

// Launch-level parameters of candidate i: {BK, stages, cta_group}.
static void grouped_launch_of(int i, int dtype, int32_t* launch) {
  launch[0] = (int32_t)(dtype == PM_FP32 ? (i / 10 ? 64 : 32) : (i / 10 ? 128 : 64));
  launch[1] = 2 + (i / 2) % 5;
  launch[2] = 1 + i % 2;
}

}  // namespace pm

namespace pm {

// One grouped launch's makespan on the GPU (one block), in F; with grad also
// its gradient.  out_host: 1 value, or 1 + NP with grad.
template <class F>
static pm_status grouped_eval(int32_t G, const int32_t* M_host, int32_t N, int32_t K, const int16_t* BM_host,
                              const int16_t* BN_host, int32_t BK, int32_t stages, int32_t cta_group, int32_t dtype,
                              const ThetaT<F>& th, int32_t n_sm, bool grad, F* out_host, cudaStream_t s) {
  PM_REQUIRE(G > 0 && G <= kMaxGroups, PM_EINVAL, "G must be in [1, %d]", kMaxGroups);
  PM_REQUIRE(M_host && BM_host && BN_host && out_host && n_sm > 0, PM_EINVAL, "null pointer or n_sm <= 0");
  PM_REQUIRE(N > 0 && K > 0 && dtype >= 0 && dtype <= 2, PM_EINVAL, "bad N, K or dtype");
  for (int q = 0; q < G; ++q) {
    PM_REQUIRE(M_host[q] > 0, PM_EINVAL, "M[%d] <= 0", q);
    PM_REQUIRE(tile_valid(BM_host[q], BN_host[q], BK, stages, cta_group, dtype), PM_EUNSUPPORTED,
               "group %d: tile %dx%dx%d stages=%d cta_group=%d outside the valid space", q, BM_host[q], BN_host[q],
               BK, stages, cta_group);
  }
  const int n_out = grad ? 1 + NP : 1;
  char* buf = nullptr;
  const size_t bytes = 256 + (size_t)G * 8 + 16 + (size_t)n_out * sizeof(F);
  PM_CUDA(cudaMallocAsync((void**)&buf, bytes, s));
  int32_t* dM = (int32_t*)buf;
  int16_t* dbm = (int16_t*)(buf + ((G * 4 + 15) & ~15));
  int16_t* dbn = dbm + ((G + 7) & ~7);
  F* dt = (F*)(dbn + ((G + 7) & ~7));
  pm_status st = PM_OK;
  cudaError_t e = cudaMemcpyAsync(dM, M_host, G * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dbm, BM_host, G * 2, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dbn, BN_host, G * 2, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    grouped_predict_kernel<F><<<1, kGroupThreads, 0, s>>>(dM, dbm, dbn, G, N, K, BK, stages, cta_group, dtype, th,
                                                           n_sm, grad, dt);
    st = launch_status("grouped_predict_kernel");
    if (st == PM_OK) e = cudaMemcpyAsync(out_host, dt, n_out * sizeof(F), cudaMemcpyDeviceToHost, s);
  }
  cudaFreeAsync(buf, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (st != PM_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "grouped predict copies");
  return PM_OK;
}

}  // namespace pm

extern "C" pm_status pm_grouped_predict(int32_t G, const int32_t* M_host, int32_t N, int32_t K,
                                        const int16_t* BM_host, const int16_t* BN_host, int32_t BK, int32_t stages,
                                        int32_t cta_group, int32_t dtype, const pm_params* theta_host, int32_t n_sm,
                                        float* t_pred_host, void* stream) {
  PM_REQUIRE(theta_host && t_pred_host && n_sm > 0, PM_EINVAL, "null pointer or n_sm <= 0");
  return grouped_eval<float>(G, M_host, N, K, BM_host, BN_host, BK, stages, cta_group, dtype,
                             to_theta(theta_host, n_sm), n_sm, false, t_pred_host, static_cast<cudaStream_t>(stream));
}

extern "C" pm_status pm_grouped_grad(int32_t G, const int32_t* M_host, int32_t N, int32_t K, const int16_t* BM_host,
                                     const int16_t* BN_host, int32_t BK, int32_t stages, int32_t cta_group,
                                     int32_t dtype, const double* theta_host, int32_t n_sm, double* out_host,
                                     void* stream) {
  PM_REQUIRE(theta_host && out_host && n_sm > 0, PM_EINVAL, "null pointer or n_sm <= 0");
  ThetaT<double> th;
  for (int j = 0; j < NP; ++j) {
    th.v[j] = theta_host[j];
    th.inv[j] = 1.0 / theta_host[j];
  }
  th.reading = g_reading.load();
  set_concurrency(th, n_sm);
  return grouped_eval<double>(G, M_host, N, K, BM_host, BN_host, BK, stages, cta_group, dtype, th, n_sm, true,
                              out_host, static_cast<cudaStream_t>(stream));
}

extern "C" pm_status pm_grouped_candidates(int32_t G, const int32_t* M_host, int32_t N, int32_t K, int32_t dtype,
                                           const pm_params* theta_host, int32_t n_sm, float* t_pred_host,
                                           int16_t* BM_host, int16_t* BN_host, int32_t* launch_host, void* stream) {
  PM_REQUIRE(t_pred_host && BM_host && BN_host && launch_host, PM_EINVAL, "null output pointer");
  std::vector<int16_t> hbm, hbn;
  pm_status st = grouped_candidates(G, M_host, N, K, dtype, theta_host, n_sm, static_cast<cudaStream_t>(stream),
                                    t_pred_host, hbm, hbn);
  if (st != PM_OK) return st;
  std::copy(hbm.begin(), hbm.end(), BM_host);
  std::copy(hbn.begin(), hbn.end(), BN_host);
  for (int i = 0; i < 20; ++i) grouped_launch_of(i, dtype, launch_host + 3 * i);
  return PM_OK;
}

extern "C" pm_status pm_grouped_autotune(int32_t G, const int32_t* M_host, int32_t N, int32_t K, int32_t dtype,
                                         const pm_params* theta_host, int32_t n_sm, int16_t* BM_out_host,
                                         int16_t* BN_out_host, int32_t* launch_out_host, float* t_pred_host,
                                         void* stream) {
  PM_REQUIRE(BM_out_host && BN_out_host && launch_out_host && t_pred_host, PM_EINVAL, "null output pointer");
  float ht[20];
  std::vector<int16_t> hbm, hbn;
  pm_status st = grouped_candidates(G, M_host, N, K, dtype, theta_host, n_sm, static_cast<cudaStream_t>(stream), ht,
                                    hbm, hbn);
  if (st != PM_OK) return st;
  int best = 0;                                   // first minimum, as the GPU's pick kernel scans
  for (int i = 1; i < 20; ++i)
    if (ht[i] < ht[best]) best = i;
  PM_REQUIRE(ht[best] < INFINITY, PM_EUNSUPPORTED, "no valid grouped configuration");
  for (int q = 0; q < G; ++q) {
    BM_out_host[q] = hbm[(size_t)best * G + q];
    BN_out_host[q] = hbn[(size_t)best * G + q];
  }
  grouped_launch_of(best, dtype, launch_out_host);
  *t_pred_host = ht[best];
  return PM_OK;
}

extern "C" pm_status pm_grouped_gemm_autotune(int32_t G, const int32_t* M_host, int32_t N, int32_t K,
                                              const pm_params* theta_host, int32_t n_sm, int32_t k,
                                              const void* A_op_dev, const void* B_op_dev, float* C_dev, int warmup,
                                              int reps, void* stream, int16_t* BM_out_host, int16_t* BN_out_host,
                                              int32_t* launch_out_host, float* t_pred_host,
                                              pm_probe_result* pick_time_out) {
  PM_REQUIRE(BM_out_host && BN_out_host && launch_out_host, PM_EINVAL, "null output pointer");
  PM_REQUIRE(k >= 1 && k <= 20, PM_EINVAL, "k must be in [1, 20]");
  PM_REQUIRE(warmup >= 0 && reps >= 1 && reps <= 100000, PM_EINVAL, "warmup >= 0 and 1 <= reps <= 1e5 required");
  PM_REQUIRE(A_op_dev && B_op_dev && C_dev, PM_EINVAL, "null operand or output pointer");
  NvtxRange nvtx("pm_grouped_gemm_autotune");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float ht[20];
  std::vector<int16_t> hbm, hbn;
  pm_status st = grouped_candidates(G, M_host, N, K, PM_BF16, theta_host, n_sm, s, ht, hbm, hbn);
  if (st != PM_OK) return st;
  // the model's k best launches (stable order), each timed; the fastest wins
  int order[20];
  for (int i = 0; i < 20; ++i) order[i] = i;
  std::stable_sort(order, order + 20, [&](int a, int b) { return ht[a] < ht[b]; });
  cudaEvent_t e0, e1;
  PM_CUDA(cudaEventCreate(&e0));
  PM_CUDA(cudaEventCreate(&e1));
  double best_t = 1e300;
  int best = -1;
  pm_probe_result best_r = {};
  pm_clock c0, c1;
  read_clock(&c0);
  for (int j = 0; j < k && st == PM_OK; ++j) {
    const int i = order[j];
    if (!(ht[i] < INFINITY)) break;
    int32_t L[3];
    grouped_launch_of(i, PM_BF16, L);
    const int16_t* bm = hbm.data() + (size_t)i * G;
    const int16_t* bn = hbn.data() + (size_t)i * G;
    for (int w = 0; w < warmup && st == PM_OK; ++w)
      st = pm_grouped_gemm_run(G, M_host, N, K, bm, bn, L[0], L[1], L[2], A_op_dev, B_op_dev, C_dev, stream);
    std::vector<double> t;
    for (int r = 0; r < reps && st == PM_OK; ++r) {
      cudaEventRecord(e0, s);
      st = pm_grouped_gemm_run(G, M_host, N, K, bm, bn, L[0], L[1], L[2], A_op_dev, B_op_dev, C_dev, stream);
      cudaEventRecord(e1, s);
      cudaError_t ce = cudaEventSynchronize(e1);
      if (ce != cudaSuccess) { st = cuda_fail(ce, "cudaEventSynchronize"); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      t.push_back(ms * 1e-3);
    }
    if (st != PM_OK) break;
    std::sort(t.begin(), t.end());
    const double med = t.size() % 2 ? t[t.size() / 2] : 0.5 * (t[t.size() / 2 - 1] + t[t.size() / 2]);
    if (med < best_t) {
      best_t = med;
      best = i;
      best_r.median_s = med;
      best_r.p25_s = t[t.size() / 4];
      best_r.p75_s = t[(3 * t.size()) / 4];
      best_r.min_s = t.front();
      best_r.bytes = 0.0;
      best_r.final_index = 0;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  read_clock(&c1);
  clock_record(&best_r, c0, c1);
  if (st != PM_OK) return st;
  PM_REQUIRE(best >= 0, PM_EUNSUPPORTED, "no valid grouped configuration");
  for (int q = 0; q < G; ++q) {
    BM_out_host[q] = hbm[(size_t)best * G + q];
    BN_out_host[q] = hbn[(size_t)best * G + q];
  }
  grouped_launch_of(best, PM_BF16, launch_out_host);
  if (t_pred_host) *t_pred_host = ht[best];
  if (pick_time_out) *pick_time_out = best_r;
  return PM_OK;
}

// ----------------------------------------------------------------------------
// Allocation-free variant of pm_model_grad.
//
// Some callers cannot allocate device memory at the point where they need the
// calibration gradient: a host program that links only this library and owns
// no CUDA allocator, a runtime working inside a fixed device-memory budget, or
// code that must not trigger allocator traffic in its hot loop.  For them the
// per-block partial sums live in a fixed array compiled into this library,
// resident on every GPU that loads it for the life of the process.
//
// Capacity: the call launches the same grid as pm_model_grad (grad_blocks(n):
// at most four blocks per SM, one partial record of NREC doubles each), so its
// partial sums are added in the same order and its output is bit-identical to
// pm_model_grad's.  The array holds kGradStaticRecords records (622,592
// bytes), enough for GPUs of up to 1024 SMs; batches are limited to
// kGradStaticRecords * kGradThreads = 1,048,576 configurations per call.
// Every record a call reads is first written by that call, so nothing has to
// be cleared between calls; two calls whose kernels overlap on a GPU share the
// array and race.
namespace pm {

constexpr int kGradStaticRecords = 4096;
static __device__ __align__(256) double g_grad_scratch[kGradStaticRecords * NREC];

static double* g_grad_scratch_ptr[64];
static std::mutex g_grad_scratch_mu;

// Device address of g_grad_scratch for the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device with that device current.
// Forgets the cached addresses (pm_shutdown; a device reset reloads the module).
void clear_grad_scratch_cache() {
  std::lock_guard<std::mutex> lk(g_grad_scratch_mu);
  for (auto& p : g_grad_scratch_ptr) p = nullptr;
}

static pm_status grad_scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  PM_REQUIRE(dev >= 0 && dev < 64, PM_EINVAL, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_grad_scratch_mu);
  if (g_grad_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_grad_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_grad_scratch)");
    g_grad_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_grad_scratch_ptr[dev];
  return PM_OK;
}

}  // namespace pm

extern "C" pm_status pm_model_grad_noalloc(const pm_cfg* cfgs_dev, int64_t n, const pm_params* theta_host,
                                           int32_t n_sm, const float* t_meas_dev, double* out_dev, void* stream) {
  PM_REQUIRE(n > 0, PM_EINVAL, "n must be positive");
  PM_REQUIRE(n <= (int64_t)kGradStaticRecords * kGradThreads, PM_ENOMEM,
             "pm_model_grad_noalloc takes at most %lld configurations per call (got %lld); split the batch or "
             "use pm_model_grad with a workspace",
             (long long)kGradStaticRecords * kGradThreads, (long long)n);
  PM_REQUIRE(cfgs_dev && theta_host && t_meas_dev && out_dev && n_sm > 0, PM_EINVAL, "null pointer or n_sm <= 0");
  PM_REQUIRE(((uintptr_t)cfgs_dev & 7) == 0, PM_EINVAL, "cfgs_dev must be 8-byte aligned");
  double* scratch = nullptr;
  pm_status st = grad_scratch_address(&scratch);
  if (st != PM_OK) return st;
  const int blocks = grad_blocks(n);
  PM_REQUIRE(blocks <= kGradStaticRecords, PM_ENOMEM, "%d partial records exceed the %d the array holds", blocks,
             kGradStaticRecords);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  model_grad_kernel<float><<<blocks, kGradThreads, 0, s>>>(cfgs_dev, n, to_theta(theta_host, n_sm), n_sm, t_meas_dev, scratch);
  st = launch_status("model_grad_kernel");
  if (st != PM_OK) return st;
  model_grad_finish_kernel<<<1, NREC * 32, 0, s>>>(scratch, blocks, n, out_dev);
  return launch_status("model_grad_finish_kernel");
}
