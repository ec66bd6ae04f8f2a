// CPU FP64 oracle for the GB300 performance-model hot path.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
// calls this file; only the tests, the package's smoke check and the bench's
// CPU-baseline arm do.  It shares no source with the CUDA library.
//
// Contents (each function cites the passage of arxiv 2605.04178 it follows):
//   * plain FP64 GEMM (the definition C = A.B, used for every precision);
//   * reference conversions to bf16, tf32 (hi/lo split) and FP8 e4m3, written
//     from the formats' definitions;
//   * probe references (triad with one rounding, pointer-chase walk);
//   * the Blackwell stage-centric model (Sec. III-A, Eqs. 1-8) with the
//     readings listed at model_gemm(), the working-set bandwidth of Eq. 16 for
//     the memory probes, and the grouped-launch makespan;
//   * its gradient, by forward-mode dual numbers carried through the same
//     code (no hand-derived adjoint here);
//   * brute-force autotuning (argmin of the model over the tile space).
//
// Build: g++ -O2 -std=c++17 -fopenmp -ffp-contract=off -shared -fPIC.
// FP contraction is off so x86 and Arm hosts give identical FP64 results.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>

typedef int64_t i64;

static inline i64 ceil_div(i64 a, i64 b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------------
// Plain GEMM.  C[i][j] = sum_k A[i][k] * B[k][j] in FP64, k ascending.
// The paper validates GEMM kernels against measured time only (Sec. V-B);
// the numerical reference is the textbook definition.
// ---------------------------------------------------------------------------
extern "C" void orc_gemm_f64(const float* A, const float* B, i64 M, i64 N, i64 K, double* C) {
#pragma omp parallel for schedule(static)
  for (i64 i = 0; i < M; ++i) {
    double* c = C + i * N;
    for (i64 j = 0; j < N; ++j) c[j] = 0.0;
    for (i64 k = 0; k < K; ++k) {
      const double a = (double)A[i * K + k];
      const float* b = B + k * N;
      for (i64 j = 0; j < N; ++j) c[j] += a * (double)b[j];
    }
  }
}

// Same product with FP64 operands (used for the dequantised-operand reference).
extern "C" void orc_gemm_f64_f64(const double* A, const double* B, i64 M, i64 N, i64 K, double* C) {
#pragma omp parallel for schedule(static)
  for (i64 i = 0; i < M; ++i) {
    double* c = C + i * N;
    for (i64 j = 0; j < N; ++j) c[j] = 0.0;
    for (i64 k = 0; k < K; ++k) {
      const double a = A[i * K + k];
      const double* b = B + k * N;
      for (i64 j = 0; j < N; ++j) c[j] += a * b[j];
    }
  }
}

// ---------------------------------------------------------------------------
// Number formats (Sec. II: the tensor cores take FP32/TF32, BF16, FP8 inputs).
// Each conversion rounds to nearest, ties to even, from the format definition.
// ---------------------------------------------------------------------------

// Round |x| (finite, FP64-exact FP32 value) to a multiple of 2^q, ties to even.
static double round_to_quantum(double ax, int q) {
  const double scaled = std::ldexp(ax, -q);  // exact: power-of-two scaling
  double f = std::floor(scaled);
  const double rem = scaled - f;             // exact
  if (rem > 0.5 || (rem == 0.5 && std::fmod(f, 2.0) != 0.0)) f += 1.0;
  return std::ldexp(f, q);
}

// bf16: 8 exponent bits, 7 explicit mantissa bits (same exponent range as FP32).
extern "C" void orc_to_bf16(const float* x, i64 n, float* y) {
  for (i64 i = 0; i < n; ++i) {
    const double v = x[i];
    if (!std::isfinite(v) || v == 0.0) { y[i] = x[i]; continue; }
    int ex; std::frexp(std::fabs(v), &ex);          // |v| in [2^(ex-1), 2^ex)
    int q = (ex - 1) - 7;
    if (q < -133) q = -133;                         // FP32 subnormal spacing 2^-149, bf16 keeps 7 bits: 2^-133
    double r = round_to_quantum(std::fabs(v), q);
    y[i] = (float)std::copysign(r, v);
  }
}

// tf32: FP32 exponent, 10 explicit mantissa bits.  The split used for
// three-pass TF32 products: hi = tf32(x), lo = tf32(x - hi).
static float to_tf32(float xf) {
  const double v = xf;
  if (!std::isfinite(v) || v == 0.0) return xf;
  int ex; std::frexp(std::fabs(v), &ex);
  int q = (ex - 1) - 10;
  if (q < -136) q = -136;
  double r = round_to_quantum(std::fabs(v), q);
  return (float)std::copysign(r, v);
}
extern "C" void orc_tf32_split(const float* x, i64 n, float* hi, float* lo) {
  for (i64 i = 0; i < n; ++i) {
    const float h = to_tf32(x[i]);
    const float r = x[i] - h;                       // exact in FP32
    hi[i] = h;
    lo[i] = to_tf32(r);
  }
}

// FP8 e4m3 (OCP "E4M3FN"): bias 7, 3 mantissa bits, no infinities, largest
// finite 448, smallest normal 2^-6, subnormal spacing 2^-9.  Saturating: any
// finite value whose rounding exceeds 448 becomes +-448.
extern "C" void orc_to_e4m3(const float* x, i64 n, uint8_t* code) {
  for (i64 i = 0; i < n; ++i) {
    const double v = x[i];
    if (std::isnan(v)) { code[i] = 0x7F; continue; }
    const uint8_t sign = std::signbit(v) ? 0x80 : 0x00;
    double a = std::fabs(v);
    if (std::isinf(a)) a = 448.0;
    int q;
    if (a < std::ldexp(1.0, -6)) {
      q = -9;
    } else {
      int ex; std::frexp(a, &ex);
      q = (ex - 1) - 3;
    }
    double r = round_to_quantum(a, q);
    if (r > 448.0) r = 448.0;
    uint8_t mag;
    if (r == 0.0) {
      mag = 0;
    } else if (r < std::ldexp(1.0, -6)) {           // subnormal: m * 2^-9
      mag = (uint8_t)std::ldexp(r, 9);
    } else {
      int ex; double fr = std::frexp(r, &ex);       // r = fr * 2^ex, fr in [0.5, 1)
      const int E = (ex - 1) + 7;
      const int m = (int)std::ldexp(fr * 2.0 - 1.0, 3);
      mag = (uint8_t)((E << 3) | m);
    }
    code[i] = sign | mag;
  }
}
extern "C" void orc_from_e4m3(const uint8_t* code, i64 n, float* y) {
  for (i64 i = 0; i < n; ++i) {
    const int c = code[i];
    const int E = (c >> 3) & 0xF, m = c & 7;
    double v;
    if (E == 0xF && m == 7) v = NAN;
    else if (E == 0) v = std::ldexp((double)m, -9);
    else v = std::ldexp(1.0 + m / 8.0, E - 7);
    y[i] = (float)((c & 0x80) ? -v : v);
  }
}

// ---------------------------------------------------------------------------
// Probe references (Sec. V-A microbenchmarks, re-targeted: STREAM-style copy
// and triad for the memory-bound class, pointer chase after Mei & Chu).
// ---------------------------------------------------------------------------
// Triad a[i] = s*c[i] + b[i] with a single rounding (fused multiply-add).
extern "C" void orc_triad_f32(const float* b, const float* c, float s, i64 n, float* a) {
  for (i64 i = 0; i < n; ++i) a[i] = std::fmaf(s, c[i], b[i]);
}

// Follow next pointers: node i holds its successor index at word i*stride_words.
extern "C" uint32_t orc_pchase(const uint32_t* buf, i64 stride_words, uint32_t start, i64 hops) {
  uint32_t j = start;
  for (i64 h = 0; h < hops; ++h) j = buf[(i64)j * stride_words];
  return j;
}

// ---------------------------------------------------------------------------
// Dual numbers: value plus the NP partial derivatives with respect to the
// model parameters theta.  Arithmetic follows the usual differentiation rules.
// ---------------------------------------------------------------------------
enum { NP = 18 };
struct Dual {
  double v;
  double d[NP];
};
static inline Dual dconst(double v) { Dual r; r.v = v; for (int j = 0; j < NP; ++j) r.d[j] = 0.0; return r; }
static inline Dual dvar(double v, int j) { Dual r = dconst(v); r.d[j] = 1.0; return r; }
static inline Dual operator+(const Dual& a, const Dual& b) { Dual r; r.v = a.v + b.v; for (int j = 0; j < NP; ++j) r.d[j] = a.d[j] + b.d[j]; return r; }
static inline Dual operator-(const Dual& a, const Dual& b) { Dual r; r.v = a.v - b.v; for (int j = 0; j < NP; ++j) r.d[j] = a.d[j] - b.d[j]; return r; }
static inline Dual operator*(const Dual& a, const Dual& b) { Dual r; r.v = a.v * b.v; for (int j = 0; j < NP; ++j) r.d[j] = a.d[j] * b.v + a.v * b.d[j]; return r; }
static inline Dual operator/(const Dual& a, const Dual& b) {
  Dual r; r.v = a.v / b.v;
  for (int j = 0; j < NP; ++j) r.d[j] = (a.d[j] * b.v - a.v * b.d[j]) / (b.v * b.v);
  return r;
}
static inline Dual operator*(double s, const Dual& a) { Dual r; r.v = s * a.v; for (int j = 0; j < NP; ++j) r.d[j] = s * a.d[j]; return r; }
static inline Dual operator+(double s, const Dual& a) { Dual r = a; r.v += s; return r; }
static inline Dual operator-(double s, const Dual& a) { Dual r; r.v = s - a.v; for (int j = 0; j < NP; ++j) r.d[j] = -a.d[j]; return r; }
static inline Dual operator/(double s, const Dual& b) { return dconst(s) / b; }
static inline Dual dexp(const Dual& a) { Dual r; r.v = std::exp(a.v); for (int j = 0; j < NP; ++j) r.d[j] = r.v * a.d[j]; return r; }
// max() takes the first argument on a tie; its derivative is the chosen branch's.
static inline Dual dmax(const Dual& a, const Dual& b) { return (a.v >= b.v) ? a : b; }
static inline Dual dclamp01(const Dual& a) {
  if (a.v <= 0.0) return dconst(0.0);
  if (a.v >= 1.0) return dconst(1.0);
  return a;
}

// Plain-double versions of the same operations, so one template serves both.
static inline double dexp(double a) { return std::exp(a); }
static inline double dmax(double a, double b) { return (a >= b) ? a : b; }
static inline double dclamp01(double a) { return a <= 0.0 ? 0.0 : (a >= 1.0 ? 1.0 : a); }
template <class T> static inline T lift(double v) { return T(v); }
template <> inline Dual lift<Dual>(double v) { return dconst(v); }
// The value of either type, for comparisons that choose a branch.
static inline double value_of(double a) { return a; }
static inline double value_of(const Dual& a) { return a.v; }

// ---------------------------------------------------------------------------
// Model parameters theta (SI units: seconds, bytes/s, FLOP/s, bytes):
//  0 T_launch      kernel launch overhead                   (Sec. III-C, P_launch)
//  1 B_sus         sustained HBM bandwidth                   (Eq. 16)
//  2 B_peak        peak HBM bandwidth                        (Eq. 16)
//  3 w0            working-set scale of the bandwidth blend  (Eq. 16)
//  4 L_TMA         TMA copy latency                          (Eq. 4)
//  5 B_TMA         TMA bandwidth per SM                      (Eq. 4)
//  6 R_TC tf32     tensor throughput per SM, TF32            (Eq. 3)
//  7 R_TC bf16     tensor throughput per SM, BF16            (Eq. 3)
//  8 R_TC fp8      tensor throughput per SM, FP8             (Eq. 3)
//  9 L_mma         tcgen05.mma latency                       (Eq. 2)
// 10 BW_TMEM_read  TMEM read bandwidth per SM                (Eq. 2)
// 11 BW_TMEM_write TMEM write bandwidth per SM               (Eq. 2)
// 12 L_mbar        mbarrier latency                          (T_sync)
// 13 L_alloc+L_dealloc  TMEM management                      (T_TMEM_mgmt)
// 14 S_2SM         2-SM cooperative speedup                  (Eq. 6)
// 15 c_alpha       overlap law alpha(s) = clamp(1 - c_alpha/s, 0, 1) (reading 1: s - 1)
// 16 rho_L2        TMA load speed-up of an L2-resident working set over a
//                  streaming one (reading 1; Sec. III-A.2: L2 hit rates
//                  strongly affect B_TMA); unused by reading 0
// 17 B_drain       per-SM rate at which a single-buffered accumulator is
//                  drained before the next tile may start (reading 1;
//                  Sec. III-A.5: T_store, overlapped only when the kernel
//                  double-buffers TMEM); unused by reading 0
// ---------------------------------------------------------------------------

enum { K_GEMM = 0, K_COPY = 1, K_TRIAD = 2, K_TMA2D = 3 };
enum { DT_FP32 = 0, DT_BF16 = 1, DT_FP8 = 2 };

struct Cfg {
  i64 M, N, K;
  int BM, BN, BK, s, g, dtype, kind;
  int tmem_a = 0;   // TMEM strategy of Sec. III-A.1: 0 = A, 1 = B (A operand also in TMEM)
};

static double elem_bytes(int dt) { return dt == DT_FP32 ? 4.0 : (dt == DT_BF16 ? 2.0 : 1.0); }
// Tensor passes per K-step: three-pass TF32 (hi.hi + hi.lo + lo.hi) for FP32.
static double mma_passes(int dt) { return dt == DT_FP32 ? 3.0 : 1.0; }
// Operand copies loaded per element: FP32 loads the hi and lo halves.
static double load_mult(int dt) { return dt == DT_FP32 ? 2.0 : 1.0; }
static int rate_index(int dt) { return dt == DT_FP32 ? 6 : (dt == DT_BF16 ? 7 : 8); }
// K depth of one tcgen05.mma instruction: 32 bytes of each operand row.
static int instr_k(int dt) { return dt == DT_FP32 ? 8 : (dt == DT_BF16 ? 16 : 32); }

// Tile-space validity (shared-memory ring and TMEM capacity, Sec. III-A.1:
// accumulators beyond 256 KB of TMEM per SM would spill).
static const i64 SMEM_OPTIN = 232448;     // 227 KiB per block
static const i64 SMEM_RESERVE = 2048;     // barriers, TMEM slot, alignment
extern "C" int orc_cfg_valid(int BM, int BN, int BK, int s, int g, int dtype, int tmem_a) {
  const bool bm_ok = BM == 64 || BM == 128 || BM == 256;
  const bool bn_ok = BN == 64 || BN == 128 || BN == 256;
  bool bk_ok;
  if (dtype == DT_FP32) bk_ok = BK == 32 || BK == 64;
  else if (dtype == DT_BF16 || dtype == DT_FP8) bk_ok = BK == 64 || BK == 128;
  else return 0;
  if (!bm_ok || !bn_ok || !bk_ok || s < 2 || s > 6 || (g != 1 && g != 2)) return 0;
  const i64 stage = (i64)(load_mult(dtype) * elem_bytes(dtype)) * BK * (BM + BN / g);
  if (s * stage > SMEM_OPTIN - SMEM_RESERVE) return 0;
  const i64 acc_cols = ceil_div(BM, 128) * BN;   // FP32 accumulator columns of one tile
  if (acc_cols > 512) return 0;
  if (tmem_a == 0) return 1;
  if (tmem_a != 1) return 0;
  // Strategy B: the A tile of every stage also lives in TMEM, 128 rows per
  // block in the lanes and l*BK*e bytes of K in 32-bit columns; built for
  // single-SM tiles of whole 128-row blocks.
  if (g != 1 || BM < 128) return 0;
  const i64 a_cols = (i64)s * ceil_div(BM, 128) * (i64)(load_mult(dtype) * elem_bytes(dtype)) * BK / 4;
  return acc_cols + a_cols <= 512 ? 1 : 0;
}

static inline bool operator<=(const Dual& a, const Dual& b) { return a.v <= b.v; }

// Eq. 16 working-set bandwidth; w0 <= 0 disables the blend.
template <class T>
static T b_eff(const T* th, double W) {
  if (th[3] <= lift<T>(0.0) ) return th[1];
  return th[1] + (th[2] - th[1]) * dexp(lift<T>(-W) / th[3]);
}

// Two sets of readings of the points the paper leaves open:
//   0 the literal equations: L_mma once per K-step (Eq. 2),
//     alpha(s) = clamp(1 - c_alpha/s, 0, 1), T_sync in both Eq. 7 and Eq. 8,
//     TMEM management amortised per K-step;
//   1 (default) readings measured on this GPU's kernels: L_mma once per tensor-pipe
//     instruction the K-step issues (BK/k_instr per 128-row block per pass,
//     plus strategy B's copies), alpha(s) = clamp(1 - c_alpha/(s-1), 0, 1)
//     (an s-stage ring keeps s-1 loads in flight), T_sync once per K-step
//     (Eq. 8; the barrier of Eq. 7 is the same one), O_misc of Eq. 8 = the
//     bubble of the s-deep ring (T_step >= (T_tma + T_c + T_sync)/s), B_TMA
//     scaled by an L2-residency factor rho(W) = 1 + (rho_L2 - 1) exp(-W/w0)
//     over the launch's working set W (Eq. 16's blend shape), the TMEM
//     management of Sec. III-A.5 paid once per launch (a persistent CTA
//     allocates its tensor memory once, not once per tile), a single-SM
//     tile of 64 rows taking the tensor time of 128 rows (an M = 64
//     tcgen05.mma on one SM runs at half the per-SM rate), and a launch
//     whose accumulator cannot be double-buffered in the 512 TMEM columns
//     paying each tile's drain before the next tile starts (T_store plus
//     4 BM BN / B_drain; a double-buffered launch overlaps it).
static int g_reading = 1;   // the measured readings by default
extern "C" void orc_set_reading(int r) { g_reading = r == 0 ? 0 : 1; }
extern "C" int orc_reading() { return g_reading; }

// Output tiles a launch runs on its CTAs: ceil(M/BM) ceil(N/BN) in the literal
// reading; in the measured reading a CTA pair covers 2 BM x BN, so a pair
// launch runs 2 ceil(M / 2BM) ceil(N/BN) CTA tiles (the last pair-row may be
// half idle).
static i64 cta_tiles(i64 M, i64 N, int BM, int BN, int g) {
  if (g_reading == 1) return (i64)g * ceil_div(M, (i64)g * BM) * ceil_div(N, (i64)BN);
  return ceil_div(M, (i64)BM) * ceil_div(N, (i64)BN);
}

// Whether a launch keeps one accumulator buffer only: the kernel holds two
// when twice the accumulator columns of its largest tile (ceil(BM/128) BN,
// or BN/2 for a 64-row tile on a CTA pair), plus strategy B's A copy per
// stage, fit in the 512 TMEM columns.
static bool single_buffer(int BM, int BN, int BK, int s, int g, int dtype, int tmem_a) {
  const i64 acc = (BM < 128 && g == 2) ? (i64)BN / 2 : ceil_div(BM, 128) * (i64)BN;
  const i64 a_ring = tmem_a ? (i64)s * ceil_div(BM, 128) * (i64)(load_mult(dtype) * elem_bytes(dtype)) * BK / 4 : 0;
  return 2 * acc + a_ring > 512;
}

// One K-step and one tile of the stage model (Eqs. 2-8).  Returns T_step and
// T_store through the out-arguments; shared by the GEMM and grouped models.
// W is the launch's working set in bytes (operands and C), used by the
// measured reading's L2 residency of the TMA loads; single_buf says whether
// the launch has one accumulator buffer only (measured reading: its drain is
// not overlapped).
template <class T>
static void stage_terms(const Cfg& c, i64 Kt, const T* th, double W, bool single_buf, T& Tstep, T& Tstore) {
  const bool measured = g_reading == 1;
  const double e = elem_bytes(c.dtype), np = mma_passes(c.dtype), l = load_mult(c.dtype);
  const T& R = th[rate_index(c.dtype)];
  // Eq. 2: per K-step TMEM cost, D_accum = FP32 accumulator bytes of the tile,
  // L_mma once per K-step (reading 0) or once per tensor-pipe instruction
  // (reading 1: BK / k_instr K-slices per 128-row block, per TF32 pass).
  const double D = 4.0 * c.BM * c.BN;
  double n_instr = measured ? np * (double)(c.BK / instr_k(c.dtype)) * (double)ceil_div(c.BM, 128) : 1.0;
  // Strategy B ("A and accumulators in TMEM", Sec. III-A.1) adds the A tile's
  // TMEM traffic: written once per K-step by the copy into TMEM (l planes),
  // read by every tensor pass.  Under reading 1 its copies (one per 128-row x
  // 32-byte slice of each plane) are tensor-pipe instructions charged L_mma.
  const double DA_w = c.tmem_a ? l * e * c.BM * c.BK : 0.0;
  const double DA_r = c.tmem_a ? np * e * c.BM * c.BK : 0.0;
  if (c.tmem_a && measured) n_instr += l * (c.BK * e / 32.0) * (double)ceil_div(c.BM, 128);
  const T T_tmem = (D + DA_r) / th[10] + n_instr * th[9] + (D + DA_w) / th[11];
  // T_TMEM_mgmt amortised over the K-steps (Sec. III-A.5); the measured
  // reading charges it once per launch instead (model_gemm).
  const T T_mgmt = measured ? lift<T>(0.0) : th[13] / lift<T>((double)Kt);
  // Eqs. 3 and 6: S_mode = 1 for one SM, S_2SM for a CTA pair.  Measured
  // reading: a one-SM tile of 64 rows issues M = 64 instructions, which take
  // as long as M = 128 ones, so its tensor time is that of 128 rows.
  const T S = (c.g == 1) ? lift<T>(1.0) : th[14];
  const double rows = (measured && c.g == 1 && c.BM < 128) ? 128.0 : (double)c.BM;
  const T T_c = lift<T>(np * 2.0 * rows * c.BN * c.BK) / (R * S) + T_tmem + T_mgmt;
  // Eq. 4 with P = 1 (no multicast); the CTA pair loads 2 M_A + M_B per
  // K-step, i.e. each CTA its own A rows and half of B (Sec. III-A.4).
  const double b_step = l * e * c.BK * (c.BM + (double)c.BN / c.g);
  // B_TMA depends on how many of the loads hit in L2 (Sec. III-A.2).  The
  // measured reading gives it the working-set shape of Eq. 16: B_TMA is
  // scaled by rho(W) = 1 + (rho_L2 - 1) exp(-W / w0), which falls from
  // rho_L2 for a launch whose operands stay in L2 to 1 for one streaming
  // from HBM (w0 <= 0 switches it off).  The literal reading keeps B_TMA
  // constant.
  T rho = lift<T>(1.0);
  if (measured && !(th[3] <= lift<T>(0.0))) rho = 1.0 + (th[16] - lift<T>(1.0)) * dexp(lift<T>(-W) / th[3]);
  const T B_tma = th[5] * rho;
  const T T_tma = th[4] + b_step / B_tma;
  // T_sync = N_bar * L_mbar with N_bar = 2 (full and empty barrier per stage).
  const T T_sync = 2.0 * th[12];
  // Eq. 7 with T_decomp = 0 and alpha from the pipeline depth: reading 0
  // alpha = 1 - c_alpha/s; reading 1 alpha = 1 - c_alpha/(s-1) (one stage
  // overlaps nothing) and the sync is counted once, in Eq. 8.
  T alpha = lift<T>(0.0);
  if (measured) alpha = c.s <= 1 ? lift<T>(0.0) : dclamp01(1.0 - th[15] / lift<T>((double)(c.s - 1)));
  else alpha = dclamp01(1.0 - th[15] / lift<T>((double)c.s));
  const T T_io = measured ? (1.0 - alpha) * T_tma : (1.0 - alpha) * T_tma + T_sync;
  // Eq. 8.  Literal reading: O_misc = 0.  Measured reading: O_misc is the
  // pipeline bubble of the s-deep ring (Sec. III-A.5 counts pipeline bubbles
  // in O_misc): every stage cycles through its load, its MMAs and its full
  // and empty barriers, so s stages complete at most one K-step per
  // (T_tma + T_c + T_sync) / s, and T_step is the larger of that and Eq. 8.
  Tstep = dmax(T_c, T_io) + T_sync;
  if (measured) Tstep = dmax(Tstep, (T_tma + T_c + T_sync) / lift<T>((double)c.s));
  // Writeback of the FP32 tile: L_store_setup + bytes(C_tile)/B (Sec. III-A.5).
  // Measured reading: with one accumulator buffer the next tile's MMAs wait
  // until the epilogue has read the whole accumulator out, so the launch
  // also pays 4 BM BN / B_drain per tile; two buffers hide that behind the
  // next tile's main loop.
  Tstore = th[4] + (4.0 * c.BM * c.BN) / th[5];
  if (measured && single_buf) Tstore = Tstore + (4.0 * c.BM * c.BN) / th[17];
}

// Stage-centric GEMM time (Sec. III-A; total of Sec. III-C's unified summary):
//   T_hat = max(T_stage, T_roofline)
//   T_stage = T_launch + waves * (K_tiles * T_step + T_store)
// Readings: persistent CTAs, one per SM (pairs for cta_group 2), so the
// tiles run in discrete waves; T_sync stays in both Eq. 7 and Eq. 8 as
// printed; the naive roofline of Sec. II-A (with S_mode) bounds from below.
template <class T>
static T model_gemm(const Cfg& c, const T* th, int n_sm) {
  // A CTA pair (cta_group::2, Sec. III-A.4) runs on two SMs: with fewer than
  // two there is no pair to run it, so the configuration has no time (NaN,
  // like any record the model cannot evaluate); the autotuners skip it.
  if (c.g != 1 && n_sm < 2) return lift<T>(NAN);
  const i64 Kt = ceil_div(c.K, c.BK);
  const i64 tiles = cta_tiles(c.M, c.N, c.BM, c.BN, c.g);
  const i64 n_conc = (c.g == 1) ? n_sm : 2 * (n_sm / 2);
  const i64 waves = ceil_div(tiles, n_conc);
  const double e = elem_bytes(c.dtype), np = mma_passes(c.dtype), l = load_mult(c.dtype);
  // bytes the launch must move at least: both operands once, C written once;
  // also its working set
  const double bytes_min = l * e * ((double)c.M * c.K + (double)c.N * c.K) + 4.0 * (double)c.M * c.N;
  T Tstep, Tstore;
  stage_terms<T>(c, Kt, th, bytes_min, single_buffer(c.BM, c.BN, c.BK, c.s, c.g, c.dtype, c.tmem_a), Tstep, Tstore);
  // the launch: T_launch, plus under the measured reading the TMEM
  // management the persistent kernel pays once
  const T launch = g_reading == 1 ? th[0] + th[13] : th[0];
  const T T_stage = launch + lift<T>((double)waves) * (lift<T>((double)Kt) * Tstep + Tstore);
  const T& R = th[rate_index(c.dtype)];
  const T S = (c.g == 1) ? lift<T>(1.0) : th[14];
  const double flops = np * 2.0 * (double)c.M * (double)c.N * (double)c.K;
  const T T_rl = launch + dmax(lift<T>(flops) / (lift<T>((double)n_sm) * R * S), lift<T>(bytes_min) / th[2]);
  return dmax(T_stage, T_rl);
}

// Memory probes through Eq. 16: beta bytes moved, working set W = beta.
template <class T>
static T model_probe(const Cfg& c, const T* th, int n_sm) {
  if (c.kind == K_COPY || c.kind == K_TRIAD) {
    const double beta = (c.kind == K_COPY ? 8.0 : 12.0) * (double)c.M;
    const T B = b_eff<T>(th, beta);
    return dmax(th[0] + lift<T>(beta) / B, th[0] + lift<T>(beta) / th[2]);
  }
  // TMA 2D copy of an M x N FP32 matrix in r x c tiles, one persistent CTA per
  // SM: tile latency once, then ceil(tiles / SMs) tile round trips (Eq. 4),
  // bounded below by the streaming time of Eq. 16.
  const double t = 4.0 * c.BM * c.BN;
  const i64 nt = ceil_div(c.M, c.BM) * ceil_div(c.N, c.BN);
  const double moved = 2.0 * 4.0 * (double)c.M * (double)c.N;
  const T B = b_eff<T>(th, moved);
  return dmax(th[0] + th[4] + lift<T>((double)ceil_div(nt, n_sm) * 2.0 * t) / th[5], th[0] + lift<T>(moved) / B);
}

template <class T>
static T model_any(const Cfg& c, const T* th, int n_sm) {
  return c.kind == K_GEMM ? model_gemm<T>(c, th, n_sm) : model_probe<T>(c, th, n_sm);
}

static Cfg make_cfg(i64 i, const int32_t* M, const int32_t* N, const int32_t* K, const int32_t* BM,
                    const int32_t* BN, const int32_t* BK, const int32_t* s, const int32_t* g,
                    const int32_t* dt, const int32_t* kind, const int32_t* ta) {
  Cfg c;
  c.M = M[i]; c.N = N[i]; c.K = K[i]; c.BM = BM[i]; c.BN = BN[i]; c.BK = BK[i];
  c.s = s[i]; c.g = g[i]; c.dtype = dt[i]; c.kind = kind[i]; c.tmem_a = ta[i];
  return c;
}

// Batched prediction; grad (n x 16, nullable) receives dT_hat/dtheta.
extern "C" void orc_model_batch(i64 n, const int32_t* M, const int32_t* N, const int32_t* K,
                                const int32_t* BM, const int32_t* BN, const int32_t* BK,
                                const int32_t* s, const int32_t* g, const int32_t* dt,
                                const int32_t* kind, const int32_t* tmem_a, const double* theta, int n_sm,
                                double* t_out, double* grad) {
#pragma omp parallel for schedule(static)
  for (i64 i = 0; i < n; ++i) {
    const Cfg c = make_cfg(i, M, N, K, BM, BN, BK, s, g, dt, kind, tmem_a);
    if (grad) {
      Dual th[NP];
      for (int j = 0; j < NP; ++j) th[j] = dvar(theta[j], j);
      const Dual t = model_any<Dual>(c, th, n_sm);
      t_out[i] = t.v;
      for (int j = 0; j < NP; ++j) grad[i * NP + j] = t.d[j];
    } else {
      t_out[i] = model_any<double>(c, theta, n_sm);
    }
  }
}

// Calibration loss (Sec. III-D: parameters fitted to measured times):
//   L = (1/n) sum_i (ln T_hat_i - ln T_i)^2,
//   dL/dtheta_j = (2/n) sum_i r_i * (dT_hat_i/dtheta_j) / T_hat_i.
extern "C" void orc_model_loss_grad(i64 n, const int32_t* M, const int32_t* N, const int32_t* K,
                                    const int32_t* BM, const int32_t* BN, const int32_t* BK,
                                    const int32_t* s, const int32_t* g, const int32_t* dt,
                                    const int32_t* kind, const int32_t* tmem_a, const double* theta, int n_sm,
                                    const double* t_meas, double* loss, double* grad) {
  std::vector<double> t(n), gr((size_t)n * NP);
  orc_model_batch(n, M, N, K, BM, BN, BK, s, g, dt, kind, tmem_a, theta, n_sm, t.data(), gr.data());
  double L = 0.0;
  double G[NP] = {0};
  for (i64 i = 0; i < n; ++i) {
    const double r = std::log(t[i]) - std::log(t_meas[i]);
    L += r * r;
    for (int j = 0; j < NP; ++j) G[j] += 2.0 * r * gr[(size_t)i * NP + j] / t[i];
  }
  *loss = L / (double)n;
  for (int j = 0; j < NP; ++j) grad[j] = G[j] / (double)n;
}

// ---------------------------------------------------------------------------
// Autotuning (Sec. III-B "adaptive tile selection", Sec. VI "autotuning
// guidance"): the predicted-fastest valid configuration; the first minimum
// in lexicographic (BM, BN, BK, stages, cta_group) order wins.
// ---------------------------------------------------------------------------
static const int BMS[3] = {64, 128, 256};
static const int BNS[3] = {64, 128, 256};
static const int BKS[3][2] = {{32, 64}, {64, 128}, {64, 128}};

extern "C" void orc_autotune(i64 n, const int32_t* MNK, int dtype, const double* theta, int n_sm,
                             int32_t* pick /* n x 5 */, double* t_pick) {
#pragma omp parallel for schedule(dynamic, 16)
  for (i64 i = 0; i < n; ++i) {
    double best = INFINITY;
    int bt[5] = {0, 0, 0, 0, 0};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        for (int k = 0; k < 2; ++k)
          for (int s = 2; s <= 6; ++s)
            for (int g = 1; g <= 2; ++g) {
              if (!orc_cfg_valid(BMS[a], BNS[b], BKS[dtype][k], s, g, dtype, 0)) continue;
              Cfg c;
              c.M = MNK[3 * i]; c.N = MNK[3 * i + 1]; c.K = MNK[3 * i + 2];
              c.BM = BMS[a]; c.BN = BNS[b]; c.BK = BKS[dtype][k]; c.s = s; c.g = g;
              c.dtype = dtype; c.kind = K_GEMM;
              const double t = model_gemm<double>(c, theta, n_sm);
              if (t < best) { best = t; bt[0] = c.BM; bt[1] = c.BN; bt[2] = c.BK; bt[3] = s; bt[4] = g; }
            }
    for (int j = 0; j < 5; ++j) pick[5 * i + j] = bt[j];
    t_pick[i] = best;
  }
}

// ---------------------------------------------------------------------------
// Grouped launch (one persistent kernel over G problems with shared N, K).
// The paper has no grouped model; this extends Eq. 8 to the kernel's static
// schedule.  With several groups the launch lists them largest tile first
// (BM x BN; ties keep the caller's order) and its tiles are dealt to the
// n_conc workers (CTAs) round by round, reversing the worker order on odd
// rounds; one group is dealt plainly round by round.  A group-g tile costs
// tau_g = K_tiles * T_step_g + T_store_g, and the launch ends with its
// busiest worker:
//   T_hat = launch + max_w sum_g n_{w,g} tau_g,
// n_{w,g} = the number of group-g tiles worker w is dealt.
// ---------------------------------------------------------------------------
// Working set of a grouped launch: every group's A rows, its own B and its C.
static double grouped_working_set(int G, const int32_t* Mg, int32_t N, int32_t K, int dtype) {
  const double le = load_mult(dtype) * elem_bytes(dtype);
  double W = 0.0;
  for (int q = 0; q < G; ++q) W += le * ((double)Mg[q] * K + (double)N * K) + 4.0 * (double)Mg[q] * N;
  return W;
}

// The order in which a launch lists its groups.
static std::vector<int> group_order(int G, const int32_t* BMg, const int32_t* BNg) {
  std::vector<int> order(G);
  for (int q = 0; q < G; ++q) order[q] = q;
  if (G > 1)
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return (i64)BMg[a] * BNg[a] > (i64)BMg[b] * BNg[b]; });
  return order;
}

// The worker that runs the tile at position i of the launch's list.
static i64 worker_of(i64 i, i64 n_conc, bool reverse_odd_rounds) {
  const i64 round = i / n_conc, j = i % n_conc;
  return (reverse_odd_rounds && round % 2 == 1) ? n_conc - 1 - j : j;
}

template <class T>
static T grouped_time(int G, const int32_t* Mg, int32_t N, int32_t K, const int32_t* BMg, const int32_t* BNg,
                      int BK, int s, int g, int dtype, const T* th, int n_sm) {
  if (g != 1 && n_sm < 2) return lift<T>(NAN);   // no SM pair for a cta_group::2 launch
  const i64 n_conc = (g == 1) ? n_sm : 2 * (n_sm / 2);
  const double W = grouped_working_set(G, Mg, N, K, dtype);
  const std::vector<int> order = group_order(G, BMg, BNg);
  // one accumulator buffer for the whole launch if its largest tile needs it
  bool single = false;
  for (int q = 0; q < G; ++q) single = single || single_buffer(BMg[q], BNg[q], BK, s, g, dtype, 0);
  std::vector<T> busy(n_conc, lift<T>(0.0));
  std::vector<i64> count(n_conc);
  i64 t = 0;
  for (int q : order) {
    Cfg c;
    c.M = Mg[q]; c.N = N; c.K = K; c.BM = BMg[q]; c.BN = BNg[q]; c.BK = BK; c.s = s; c.g = g;
    c.dtype = dtype; c.kind = K_GEMM;
    const i64 Kt = ceil_div(K, BK);
    T Tstep, Tstore;
    stage_terms<T>(c, Kt, th, W, single, Tstep, Tstore);
    const T tau = lift<T>((double)Kt) * Tstep + Tstore;
    // With cta_group 2 a pair of consecutive tiles runs on a worker pair;
    // each CTA of the pair is one worker.
    const i64 tiles = cta_tiles(c.M, N, c.BM, c.BN, g);
    std::fill(count.begin(), count.end(), (i64)0);
    for (i64 j = 0; j < tiles; ++j, ++t) ++count[worker_of(t, n_conc, G > 1)];
    for (i64 w = 0; w < n_conc; ++w)
      if (count[w]) busy[w] = busy[w] + lift<T>((double)count[w]) * tau;
  }
  T mx = busy[0];                                  // the first busiest worker
  for (i64 w = 1; w < n_conc; ++w)
    if (value_of(busy[w]) > value_of(mx)) mx = busy[w];
  const T launch = g_reading == 1 ? th[0] + th[13] : th[0];
  return launch + mx;
}

extern "C" double orc_grouped_predict(int G, const int32_t* Mg, int32_t N, int32_t K,
                                      const int32_t* BMg, const int32_t* BNg, int BK, int s, int g,
                                      int dtype, const double* theta, int n_sm) {
  return grouped_time<double>(G, Mg, N, K, BMg, BNg, BK, s, g, dtype, theta, n_sm);
}

// The same makespan with its gradient in theta (grad: NP doubles).
extern "C" double orc_grouped_predict_grad(int G, const int32_t* Mg, int32_t N, int32_t K,
                                           const int32_t* BMg, const int32_t* BNg, int BK, int s, int g,
                                           int dtype, const double* theta, int n_sm, double* grad) {
  Dual th[NP];
  for (int j = 0; j < NP; ++j) th[j] = dvar(theta[j], j);
  const Dual t = grouped_time<Dual>(G, Mg, N, K, BMg, BNg, BK, s, g, dtype, th, n_sm);
  for (int j = 0; j < NP; ++j) grad[j] = t.d[j];
  return t.v;
}

// Grouped autotune: for each launch-level (BK, stages, cta_group) in
// lexicographic order, each group takes the (BM, BN) minimising
// tiles_g * tau_g (first minimum); the launch with the smallest makespan wins.
extern "C" double orc_grouped_autotune(int G, const int32_t* Mg, int32_t N, int32_t K, int dtype,
                                       const double* theta, int n_sm, int32_t* BMg, int32_t* BNg,
                                       int32_t* launch /* BK, s, g */) {
  double best = INFINITY;
  std::vector<int32_t> bm(G), bn(G);
  const double W = grouped_working_set(G, Mg, N, K, dtype);
  for (int k = 0; k < 2; ++k)
    for (int s = 2; s <= 6; ++s)
      for (int g = 1; g <= 2; ++g) {
        const int BK = BKS[dtype][k];
        bool ok = true;
        for (int q = 0; q < G && ok; ++q) {
          double bq = INFINITY;
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
              if (!orc_cfg_valid(BMS[a], BNS[b], BK, s, g, dtype, 0)) continue;
              Cfg c;
              c.M = Mg[q]; c.N = N; c.K = K; c.BM = BMS[a]; c.BN = BNS[b]; c.BK = BK; c.s = s;
              c.g = g; c.dtype = dtype; c.kind = K_GEMM;
              const i64 Kt = ceil_div(K, BK);
              double Tstep, Tstore;
              // the group's tile alone decides its buffering here; the
              // launch's makespan below applies the launch-wide rule
              stage_terms<double>(c, Kt, theta, W, single_buffer(c.BM, c.BN, BK, s, g, dtype, 0), Tstep, Tstore);
              const double tiles = (double)cta_tiles(c.M, N, c.BM, c.BN, g);
              const double cost = tiles * ((double)Kt * Tstep + Tstore);
              if (cost < bq) { bq = cost; bm[q] = c.BM; bn[q] = c.BN; }
            }
          if (bq == INFINITY) ok = false;
        }
        if (!ok) continue;
        const double t = orc_grouped_predict(G, Mg, N, K, bm.data(), bn.data(), BK, s, g, dtype, theta, n_sm);
        if (t < best) {
          best = t;
          for (int q = 0; q < G; ++q) { BMg[q] = bm[q]; BNg[q] = bn[q]; }
          launch[0] = BK; launch[1] = s; launch[2] = g;
        }
      }
  return best;
}

// ---------------------------------------------------------------------------
// Generic roofline path (Sec. III-E "Generic roofline path: scaling, working
// set, and launches" and "Host-device transfer and synchronization"): a
// workload segment outside the stage model takes, per execution, its kernel
// launches, a class-scaled roofline whose bandwidth follows Eq. 16, the host
// transfers of Eq. 15 and its synchronisation points; the total multiplies by
// the number of executions.  Copies and kernels are summed (no overlap).
// Concurrent streams (Sec. III-A.6): a segment run as N_c copies on N_c
// streams adds (N_c - 1) tau_c to its single-stream time, with tau_c the part
// of one copy that cannot overlap the others: a fraction kappa_launch of its
// launches and a fraction kappa_class of its class-scaled roofline time.
//   psi: 0-3 class scales (memory, compute, balanced, stencil),
//        4-6 precision efficiencies (FP32, BF16, FP8),
//        7 B_h2d, 8 tau_h2d, 9 B_d2h, 10 tau_d2h, 11 tau_sync,
//        12-15 kappa per class, 16 kappa_launch.
// ---------------------------------------------------------------------------
enum { NPSI = 17 };
extern "C" void orc_segment_predict(i64 n, const double* flops, const double* bytes, const double* wset,
                                    const double* h2d, const double* d2h, const int32_t* cls,
                                    const int32_t* prec, const int32_t* kernels, const int32_t* syncs,
                                    const int32_t* execs, const int32_t* streams, const double* theta,
                                    const double* psi, int n_sm, double* t_out) {
  for (i64 i = 0; i < n; ++i) {
    const bool ok = cls[i] >= 0 && cls[i] <= 3 && prec[i] >= 0 && prec[i] <= 2 && kernels[i] >= 0 &&
                    syncs[i] >= 0 && execs[i] >= 1 && streams[i] >= 0 && flops[i] >= 0 && bytes[i] >= 0 &&
                    wset[i] >= 0 && h2d[i] >= 0 && d2h[i] >= 0;
    if (!ok) {
      t_out[i] = NAN;
      continue;
    }
    double t = 0.0;
    if (kernels[i] > 0) {
      // the extra launches of a multi-kernel segment, then one roofline
      const double launches = kernels[i] * theta[0];
      const double bandwidth = b_eff<double>(theta, wset[i]);               // Eq. 16
      const double peak = n_sm * theta[rate_index(prec[i])] * psi[4 + prec[i]];
      const double memory_time = bytes[i] / bandwidth;
      const double compute_time = flops[i] / peak;
      const double roof = psi[cls[i]] * (compute_time > memory_time ? compute_time : memory_time);
      t += launches + roof;
      // N_c concurrent copies: (N_c - 1) tau_c more (0 or 1 stream: none)
      if (streams[i] > 1) t += (streams[i] - 1) * (psi[16] * launches + psi[12 + cls[i]] * roof);
    }
    if (h2d[i] > 0) t += h2d[i] / psi[7] + psi[8];                          // Eq. 15
    if (d2h[i] > 0) t += d2h[i] / psi[9] + psi[10];
    t += syncs[i] * psi[11];
    t_out[i] = execs[i] * t;
  }
}

// Five-point stencil of the generic path's stencil class: interior points
// 0.5 x + 0.125 ((up + down) + (left + right)) in FP32 with every operation
// rounded on its own (the file is compiled without contraction); border
// points copied.
extern "C" void orc_stencil5_f32(const float* in, i64 rows, i64 cols, float* out) {
#pragma omp parallel for schedule(static)
  for (i64 i = 0; i < rows; ++i)
    for (i64 j = 0; j < cols; ++j) {
      const i64 k = i * cols + j;
      if (i == 0 || j == 0 || i == rows - 1 || j == cols - 1) {
        out[k] = in[k];
        continue;
      }
      const float vert = in[k - cols] + in[k + cols];
      const float horz = in[k - 1] + in[k + 1];
      const float half = 0.5f * in[k];
      const float eighth = 0.125f * (vert + horz);
      out[k] = half + eighth;
    }
}
