// The GEMM family the stage-centric model of arxiv 2605.04178 predicts
// (Sec. III-A, Fig. "cta-exec-model"): per K-step a TMA load of the A and B
// tiles into a shared-memory ring (Eq. 4), tcgen05.mma into an FP32 TMEM
// accumulator (Eqs. 2-3; Eq. 6 for CTA pairs), mbarrier hand-offs (T_sync),
// and an epilogue that drains TMEM to global memory (T_store).
//
// Kernel shape (sm_103a): one persistent CTA per SM (CTA pair per two SMs for
// cta_group 2), 6 warps:
//   warp 0      TMA producer (one thread): waits empty[s], loads stage s;
//   warp 1      TMEM allocator and MMA issuer (one thread): waits full[s],
//               issues BK/k_instr MMAs per row block, commits to empty[s];
//               after the last K-step commits to acc_full[buffer];
//   warps 2..5  epilogue: wait acc_full, tcgen05.ld 32-column chunks, scale,
//               store FP32 C (masked at the M/N edges), release the buffer.
// Two TMEM accumulator buffers when they fit, so the epilogue of tile i
// overlaps the main loop of tile i+1.  Each CTA of a pair loads its own A
// rows and half of B (traffic 2 M_A + M_B per pair, no multicast); the pair
// leader issues the cta_group::2 MMAs.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdlib.h>

#include <algorithm>
#include <mutex>

#include "pm_internal.cuh"

namespace pm {

constexpr int kGemmThreads = 192;
constexpr int kMaxStages = 6;
constexpr int kRasterGroup = 8;

struct GemmParams {
  int M, N, K;
  int BM, BN, BK, stages;
  int tiles_m, tiles_n, n_tiles;   // tiles_m counts pair rows (2*BM) for cta_group 2
  int Kt;
  int sw;                          // swizzle span in bytes (64 or 128)
  int n_atoms;                     // swizzle atoms along K per stage
  int n_mblk;                      // 128-row MMA blocks per CTA tile
  int acc_cols, nbuf, alloc_cols;
  uint32_t stage_bytes, a_part_bytes, b_part_bytes, tx_bytes;
  uint32_t idesc;
  int lo_row_a, lo_row_b;          // row offset of the lo half (three-pass TF32)
  // TMEM layout of the accumulator: 0 = one row per lane (128-row blocks),
  // 1 = 64 rows in lanes 0-15 of each 32-lane quarter (M = 64, one SM),
  // 2 = 64 rows in lanes 0-63 for columns [0, N/2) and again in lanes
  //     64-127 for columns [N/2, N) (M = 128 split over a CTA pair).
  int layout;
  float* C;
  const float* scales;             // FP8: {s_A, s_B}
  Watchdog wd;
};

__device__ __forceinline__ void tile_coords(int t, const GemmParams& p, int& tm, int& tn) {
  const int per_group = kRasterGroup * p.tiles_n;
  const int gid = t / per_group;
  const int first = gid * kRasterGroup;
  const int gsz = min(p.tiles_m - first, kRasterGroup);
  const int r = t % per_group;
  tm = first + r % gsz;
  tn = r / gsz;
}

template <int CG, int KIND>
__global__ void __launch_bounds__(kGemmThreads, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const GemmParams p) {
  extern __shared__ __align__(1024) uint8_t dsmem[];
  __shared__ __align__(8) uint64_t full_bar[kMaxStages];
  __shared__ __align__(8) uint64_t empty_bar[kMaxStages];
  __shared__ __align__(8) uint64_t accf_bar[2];
  __shared__ __align__(8) uint64_t acce_bar[2];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  constexpr int L = (KIND == 1) ? 2 : 1;              // operand halves (hi, lo) for three-pass TF32
  constexpr int E = (KIND == 0) ? 2 : (KIND == 1 ? 4 : 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = (CG == 2) ? cluster_ctarank() : 0u;
  const int cta = (CG == 2) ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int n_ctas = (CG == 2) ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  const uint32_t base = (smem_u32(dsmem) + 1023u) & ~1023u;
  const uint32_t swcode = p.sw == 128 ? 2u : 4u;
  volatile int* abort_p = &abort_flag;

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(smem_u32(&full_bar[s]), CG);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&accf_bar[b]), 1);
      mbar_init(smem_u32(&acce_bar[b]), 4 * CG);
    }
    mbar_init(smem_u32(&done_bar), 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmB);
  }
  if (warp == 1) {
    tmem_alloc<CG>(smem_u32(&tmem_slot), (uint32_t)p.alloc_cols);
    tmem_relinquish<CG>();
  }
  tc_fence_before();
  if constexpr (CG == 2) cluster_sync(); else __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int t = cta; t < p.n_tiles && ok; t += n_ctas) {
        int tm, tn;
        tile_coords(t, p, tm, tn);
        const int arow = (CG == 1) ? tm * p.BM : tm * 2 * p.BM + (int)rank * p.BM;
        const int brow = tn * p.BN + (CG == 2 ? (int)rank * (p.BN / 2) : 0);
        for (int kt = 0; kt < p.Kt; ++kt) {
          if (!mbar_wait(smem_u32(&empty_bar[stage]), phase ^ 1u, p.wd, abort_p, SITE_GEMM_PRODUCER)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&full_bar[stage]);
          uint32_t fbc = fb;
          if constexpr (CG == 1) {
            mbar_arrive_expect_tx(fb, p.tx_bytes);
          } else {
            fbc = mapa_shared(fb, 0);
            mbar_arrive_expect_tx_cluster(fbc, p.tx_bytes);
          }
          const uint32_t sbase = base + (uint32_t)stage * p.stage_bytes;
          const uint32_t bbase = sbase + (uint32_t)(L * p.n_atoms) * p.a_part_bytes;
#pragma unroll
          for (int h = 0; h < L; ++h) {
            for (int a = 0; a < p.n_atoms; ++a) {
              const int x = kt * p.BK + a * (p.sw / E);
              const uint32_t da = sbase + (uint32_t)(h * p.n_atoms + a) * p.a_part_bytes;
              const uint32_t db = bbase + (uint32_t)(h * p.n_atoms + a) * p.b_part_bytes;
              if constexpr (CG == 1) {
                tma_load_2d(da, &tmA, fb, x, arow + h * p.lo_row_a);
                tma_load_2d(db, &tmB, fb, x, brow + h * p.lo_row_b);
              } else {
                tma_load_2d_pair(da, &tmA, fbc, x, arow + h * p.lo_row_a);
                tma_load_2d_pair(db, &tmB, fbc, x, brow + h * p.lo_row_b);
              }
            }
          }
          if (++stage == p.stages) { stage = 0; phase ^= 1u; }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------- MMA issuer
    if (lane == 0 && rank == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      const uint32_t sbo = 8u * (uint32_t)p.sw;
      int it = 0;
      for (int t = cta; t < p.n_tiles && ok; t += n_ctas, ++it) {
        const int buf = it % p.nbuf;
        const uint32_t use = (uint32_t)(it / p.nbuf);
        if (!mbar_wait(smem_u32(&acce_bar[buf]), (use & 1u) ^ 1u, p.wd, abort_p, SITE_GEMM_MMA)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d0 = tmem_base + (uint32_t)(buf * p.acc_cols);
        for (int kt = 0; kt < p.Kt; ++kt) {
          if (!mbar_wait(smem_u32(&full_bar[stage]), phase, p.wd, abort_p, SITE_GEMM_MMA)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sbase = base + (uint32_t)stage * p.stage_bytes;
          const uint32_t bbase = sbase + (uint32_t)(L * p.n_atoms) * p.a_part_bytes;
          constexpr int PASSES = (KIND == 1) ? 3 : 1;
#pragma unroll
          for (int pass = 0; pass < PASSES; ++pass) {
            const int ha = (pass == 2) ? 1 : 0;   // hi.hi, hi.lo, lo.hi
            const int hb = (pass == 1) ? 1 : 0;
            for (int a = 0; a < p.n_atoms; ++a) {
              const uint32_t pa = sbase + (uint32_t)(ha * p.n_atoms + a) * p.a_part_bytes;
              const uint32_t pb = bbase + (uint32_t)(hb * p.n_atoms + a) * p.b_part_bytes;
              for (int kk = 0; kk < p.sw / 32; ++kk) {
                const uint64_t bdesc = smem_desc(pb + 32u * kk, sbo, swcode);
                const uint32_t acc = (kt | pass | a | kk) != 0 ? 1u : 0u;
                for (int m = 0; m < p.n_mblk; ++m) {
                  const uint64_t adesc = smem_desc(pa + (uint32_t)(m * 128 * p.sw) + 32u * kk, sbo, swcode);
                  umma<CG, KIND>(d0 + (uint32_t)(m * p.BN), adesc, bdesc, p.idesc, acc);
                }
              }
            }
          }
          if constexpr (CG == 1) umma_commit(smem_u32(&empty_bar[stage]));
          else umma_commit_pair(smem_u32(&empty_bar[stage]), (uint16_t)3);
          if (++stage == p.stages) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        if constexpr (CG == 1) umma_commit(smem_u32(&accf_bar[buf]));
        else umma_commit_pair(smem_u32(&accf_bar[buf]), (uint16_t)3);
      }
      // all MMAs of this thread complete before the teardown frees TMEM
      if constexpr (CG == 1) umma_commit(smem_u32(&done_bar));
      else umma_commit_pair(smem_u32(&done_bar), (uint16_t)1);
      mbar_wait(smem_u32(&done_bar), 0u, p.wd, nullptr, SITE_GEMM_TEARDOWN);
    }
  } else {
    // --------------------------------------------------------------- epilogue
    const int q = warp & 3;                               // TMEM lane quarter of this warp
    float scale = 1.f;
    if constexpr (KIND == 2) scale = 1.f / (__ldg(p.scales) * __ldg(p.scales + 1));
    const bool vec = (p.N & 3) == 0;
    // rows and columns this warp's TMEM lane quarter holds
    int lrow, qcol0, qcols;
    bool lvalid;
    if (p.layout == 1) {
      lrow = 16 * q + lane; lvalid = lane < 16; qcol0 = 0; qcols = p.BN;
    } else if (p.layout == 2) {
      lrow = 32 * (q & 1) + lane; lvalid = true; qcol0 = (q >> 1) * (p.BN / 2); qcols = p.BN / 2;
    } else {
      lrow = 32 * q + lane; lvalid = true; qcol0 = 0; qcols = p.BN;
    }
    int it = 0;
    for (int t = cta; t < p.n_tiles; t += n_ctas, ++it) {
      const int buf = it % p.nbuf;
      const uint32_t use = (uint32_t)(it / p.nbuf);
      if (!mbar_wait(smem_u32(&accf_bar[buf]), use & 1u, p.wd, abort_p, SITE_GEMM_EPILOGUE)) break;
      tc_fence_after();
      int tm, tn;
      tile_coords(t, p, tm, tn);
      const int crow0 = (CG == 1) ? tm * p.BM : tm * 2 * p.BM + (int)rank * p.BM;
      const int ccol0 = tn * p.BN + qcol0;
      for (int m = 0; m < p.n_mblk; ++m) {
        const int row = crow0 + m * 128 + lrow;
        const bool rvalid = lvalid && row < p.M;
        float* crow = p.C + (size_t)row * p.N;
        for (int j = 0; j < qcols / 32; ++j) {
          uint32_t r[32];
          const uint32_t taddr =
              tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * p.acc_cols + m * p.BN + 32 * j);
          tmem_ld_32x32b_x32(taddr, r);
          tmem_ld_wait();
          const int col0 = ccol0 + 32 * j;
          if (rvalid) {
            if (vec && col0 + 32 <= p.N) {
#pragma unroll
              for (int v = 0; v < 8; ++v) {
                float4 o;
                o.x = __uint_as_float(r[4 * v + 0]) * scale;
                o.y = __uint_as_float(r[4 * v + 1]) * scale;
                o.z = __uint_as_float(r[4 * v + 2]) * scale;
                o.w = __uint_as_float(r[4 * v + 3]) * scale;
                *reinterpret_cast<float4*>(crow + col0 + 4 * v) = o;
              }
            } else {
              for (int v = 0; v < 32; ++v)
                if (col0 + v < p.N) crow[col0 + v] = __uint_as_float(r[v]) * scale;
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        const uint32_t eb = smem_u32(&acce_bar[buf]);
        if constexpr (CG == 1) mbar_arrive(eb);
        else mbar_arrive_cluster(mapa_shared(eb, 0));
      }
    }
  }

  // ---------------------------------------------------------------- teardown
  tc_fence_before();
  __syncthreads();
  if constexpr (CG == 2) cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc<CG>(tmem_base, (uint32_t)p.alloc_cols);
  }
}

// --------------------------------------------------------------- operand prep
// Row-major FP32 inputs to the tensor-core operand formats.  HBM-bound
// pre-passes outside the GEMM proper.
__device__ __forceinline__ float tf32_rn(float x) {
  // round to nearest even at mantissa bit 13 (finite inputs)
  uint32_t b = __float_as_uint(x);
  if ((b & 0x7f800000u) == 0x7f800000u) return x;
  b = (b + 0xfffu + ((b >> 13) & 1u)) & 0xffffe000u;
  return __uint_as_float(b);
}

__global__ void amax_kernel(const float* __restrict__ x, int64_t n, unsigned int* __restrict__ amax_bits) {
  float m = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(__ldg(x + i)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax_bits, __float_as_uint(m));
}

__device__ __forceinline__ float fp8_scale_of(unsigned int amax_bits) {
  const float amax = __uint_as_float(amax_bits);
  return amax > 0.f ? 448.f / amax : 1.f;
}

// Row-major [R, C] FP32 -> same layout in the operand format (A side).
__global__ void convert_rows_kernel(const float* __restrict__ x, int64_t n, int mode, void* __restrict__ y,
                                    float* __restrict__ y_lo, const unsigned int* __restrict__ amax_bits,
                                    float* __restrict__ scale_out) {
  float s = 1.f;
  if (mode == PM_FP8E4M3) {
    s = fp8_scale_of(*amax_bits);
    if (blockIdx.x == 0 && threadIdx.x == 0 && scale_out) *scale_out = s;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = __ldg(x + i);
    if (mode == PM_BF16) {
      static_cast<__nv_bfloat16*>(y)[i] = __float2bfloat16_rn(v);
    } else if (mode == PM_FP8E4M3) {
      static_cast<__nv_fp8_storage_t*>(y)[i] = __nv_cvt_float_to_fp8(v * s, __NV_SATFINITE, __NV_E4M3);
    } else {
      const float hi = tf32_rn(v);
      static_cast<float*>(y)[i] = hi;
      y_lo[i] = tf32_rn(v - hi);
    }
  }
}

// Row-major [K, N] FP32 -> K-major [N, K] operand (B side), 32x32 tiles.
__global__ void transpose_convert_kernel(const float* __restrict__ x, int K, int N, int mode, void* __restrict__ y,
                                         float* __restrict__ y_lo, const unsigned int* __restrict__ amax_bits,
                                         float* __restrict__ scale_out) {
  __shared__ float tile[32][33];
  float s = 1.f;
  if (mode == PM_FP8E4M3) {
    s = fp8_scale_of(*amax_bits);
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0 && scale_out) *scale_out = s;
  }
  const int n0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, nn = n0 + threadIdx.x;
    tile[r][threadIdx.x] = (k < K && nn < N) ? __ldg(x + (size_t)k * N + nn) : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int nn = n0 + r, k = k0 + threadIdx.x;
    if (nn < N && k < K) {
      const float v = tile[threadIdx.x][r];
      const size_t o = (size_t)nn * K + k;
      if (mode == PM_BF16) {
        static_cast<__nv_bfloat16*>(y)[o] = __float2bfloat16_rn(v);
      } else if (mode == PM_FP8E4M3) {
        static_cast<__nv_fp8_storage_t*>(y)[o] = __nv_cvt_float_to_fp8(v * s, __NV_SATFINITE, __NV_E4M3);
      } else {
        const float hi = tf32_rn(v);
        static_cast<float*>(y)[o] = hi;
        y_lo[o] = tf32_rn(v - hi);
      }
    }
  }
}

// ------------------------------------------------------------------ host side
static inline int dt_elem(int dt) { return dt == PM_FP32 ? 4 : (dt == PM_BF16 ? 2 : 1); }
static inline int dt_halves(int dt) { return dt == PM_FP32 ? 2 : 1; }

bool gemm_tile_valid(int BM, int BN, int BK, int s, int g, int dt) {
  if (!(BM == 64 || BM == 128 || BM == 256) || !(BN == 64 || BN == 128 || BN == 256)) return false;
  if (dt == PM_FP32) {
    if (BK != 32 && BK != 64) return false;
  } else if (dt == PM_BF16 || dt == PM_FP8E4M3) {
    if (BK != 64 && BK != 128) return false;
  } else {
    return false;
  }
  if (s < 2 || s > kMaxStages || (g != 1 && g != 2)) return false;
  const int64_t stage = (int64_t)dt_halves(dt) * dt_elem(dt) * BK * (BM + BN / g);
  if ((int64_t)s * stage > 232448 - 2048) return false;
  if (((BM + 127) / 128) * BN > 512) return false;
  return true;
}

struct TmapKey {
  const void* ptr;
  uint64_t rows, cols;
  uint32_t box_rows, box_cols;
  int dt, sw;
  bool operator==(const TmapKey& o) const {
    return ptr == o.ptr && rows == o.rows && cols == o.cols && box_rows == o.box_rows && box_cols == o.box_cols &&
           dt == o.dt && sw == o.sw;
  }
};
struct TmapEntry {
  TmapKey key;
  CUtensorMap map;
  bool used = false;
};
static thread_local TmapEntry g_tmaps[16];
static thread_local int g_tmap_next = 0;

pm_status cached_tmap(CUtensorMap* out, const void* ptr, int dtcode, uint64_t rows, uint64_t cols, uint32_t box_rows,
                      uint32_t box_cols, int sw) {
  TmapKey k{ptr, rows, cols, box_rows, box_cols, dtcode, sw};
  for (auto& e : g_tmaps)
    if (e.used && e.key == k) {
      *out = e.map;
      return PM_OK;
    }
  TmapEntry& e = g_tmaps[g_tmap_next];
  g_tmap_next = (g_tmap_next + 1) % 16;
  pm_status st = make_tmap_2d(&e.map, ptr, dtcode, rows, cols, box_rows, box_cols, sw);
  if (st != PM_OK) {
    e.used = false;
    return st;
  }
  e.key = k;
  e.used = true;
  *out = e.map;
  return PM_OK;
}

template <int CG, int KIND>
static pm_status launch_gemm(const CUtensorMap& ta, const CUtensorMap& tb, const GemmParams& p, int grid,
                             size_t smem, cudaStream_t s) {
  auto kern = gemm_kernel<CG, KIND>;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [&] {
    attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448 - 1024);
  });
  if (attr_err != cudaSuccess) return cuda_fail(attr_err, "cudaFuncSetAttribute(gemm_kernel)");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(kGemmThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (CG == 2) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, ta, tb, p);
  if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchKernelEx(gemm_kernel)");
  return PM_OK;
}

pm_status gemm_plan(const pm_cfg& c, GemmParams& p, size_t& smem) {
  const int dt = c.dtype, g = c.cta_group;
  PM_REQUIRE(c.kind == PM_KIND_GEMM, PM_EINVAL, "cfg.kind must be PM_KIND_GEMM");
  PM_REQUIRE(c.M > 0 && c.N > 0 && c.K > 0, PM_EINVAL, "M, N, K must be positive");
  PM_REQUIRE(gemm_tile_valid(c.BM, c.BN, c.BK, c.stages, g, dt), PM_EUNSUPPORTED,
             "tile configuration BM=%d BN=%d BK=%d stages=%d cta_group=%d dtype=%d is outside the valid space",
             c.BM, c.BN, c.BK, c.stages, g, dt);
  const int e = dt_elem(dt), L = dt_halves(dt);
  PM_REQUIRE(((int64_t)c.K * e) % 16 == 0, PM_EINVAL, "K*%d bytes must be a multiple of 16", e);
  p.M = c.M; p.N = c.N; p.K = c.K;
  p.BM = c.BM; p.BN = c.BN; p.BK = c.BK; p.stages = c.stages;
  p.tiles_m = (c.M + g * c.BM - 1) / (g * c.BM);
  p.tiles_n = (c.N + c.BN - 1) / c.BN;
  p.n_tiles = p.tiles_m * p.tiles_n;
  p.Kt = (c.K + c.BK - 1) / c.BK;
  p.sw = std::min(128, c.BK * e);
  p.n_atoms = c.BK * e / p.sw;
  p.n_mblk = (c.BM + 127) / 128;
  p.layout = c.BM >= 128 ? 0 : (g == 1 ? 1 : 2);
  p.acc_cols = p.layout == 2 ? c.BN / 2 : p.n_mblk * c.BN;
  p.nbuf = (2 * p.acc_cols <= 512) ? 2 : 1;
  int need = p.nbuf * p.acc_cols, cols = 32;
  while (cols < need) cols <<= 1;
  p.alloc_cols = cols;
  p.a_part_bytes = (uint32_t)c.BM * p.sw;
  p.b_part_bytes = (uint32_t)(c.BN / g) * p.sw;
  p.stage_bytes = (uint32_t)(L * p.n_atoms) * (p.a_part_bytes + p.b_part_bytes);
  p.tx_bytes = p.stage_bytes;
  const int bm = c.BM;
  const int mma_m = (g == 1) ? std::min(bm, 128) : 2 * std::min(bm, 128);
  const uint32_t fmt = dt == PM_BF16 ? 1u : (dt == PM_FP32 ? 2u : 0u);
  p.idesc = instr_desc(fmt, (uint32_t)mma_m, (uint32_t)c.BN);
  p.lo_row_a = (L == 2) ? c.M : 0;
  p.lo_row_b = (L == 2) ? c.N : 0;
  smem = (size_t)c.stages * p.stage_bytes + 1024;
  return PM_OK;
}

pm_status gemm_launch(const pm_cfg& c, const void* A_op, const void* B_op, float* C, const float* scales,
                      cudaStream_t s) {
  GemmParams p;
  size_t smem = 0;
  pm_status st = gemm_plan(c, p, smem);
  if (st != PM_OK) return st;
  PM_REQUIRE(A_op && B_op && C, PM_EINVAL, "null operand or output pointer");
  PM_REQUIRE(c.dtype != PM_FP8E4M3 || scales, PM_EINVAL, "FP8 GEMM needs scales_dev");
  const int dt = c.dtype, g = c.cta_group;
  const int e = dt_elem(dt), L = dt_halves(dt);
  const int dtcode = dt == PM_BF16 ? TMAP_BF16 : (dt == PM_FP32 ? TMAP_F32 : TMAP_U8);
  CUtensorMap ta, tb;
  st = cached_tmap(&ta, A_op, dtcode, (uint64_t)L * c.M, (uint64_t)c.K, (uint32_t)c.BM, (uint32_t)(p.sw / e), p.sw);
  if (st != PM_OK) return st;
  st = cached_tmap(&tb, B_op, dtcode, (uint64_t)L * c.N, (uint64_t)c.K, (uint32_t)(c.BN / g), (uint32_t)(p.sw / e),
                   p.sw);
  if (st != PM_OK) return st;
  unsigned int* w = watchdog_word();
  PM_REQUIRE(w != nullptr, PM_ECUDA, "watchdog word unavailable");
  p.wd = Watchdog{w, watchdog_limit_ns()};
  p.C = C;
  p.scales = scales;
  const int sms = sm_count();
  int grid;
  if (g == 1) grid = std::min(p.n_tiles, sms);
  else grid = 2 * std::min(p.n_tiles, sms / 2);
  if (g == 1) {
    if (dt == PM_BF16) return launch_gemm<1, 0>(ta, tb, p, grid, smem, s);
    if (dt == PM_FP32) return launch_gemm<1, 1>(ta, tb, p, grid, smem, s);
    return launch_gemm<1, 2>(ta, tb, p, grid, smem, s);
  }
  if (dt == PM_BF16) return launch_gemm<2, 0>(ta, tb, p, grid, smem, s);
  if (dt == PM_FP32) return launch_gemm<2, 1>(ta, tb, p, grid, smem, s);
  return launch_gemm<2, 2>(ta, tb, p, grid, smem, s);
}

}  // namespace pm

using namespace pm;

extern "C" pm_status pm_gemm_operand_bytes(int32_t dtype, int32_t M, int32_t N, int32_t K, size_t* a_bytes,
                                           size_t* b_bytes) {
  PM_REQUIRE(a_bytes && b_bytes, PM_EINVAL, "null output pointer");
  PM_REQUIRE(dtype >= 0 && dtype <= 2 && M > 0 && N > 0 && K > 0, PM_EINVAL, "bad dtype or shape");
  *a_bytes = (size_t)dt_halves(dtype) * dt_elem(dtype) * (size_t)M * K;
  *b_bytes = (size_t)dt_halves(dtype) * dt_elem(dtype) * (size_t)N * K;
  return PM_OK;
}

extern "C" pm_status pm_gemm_prepare(int32_t dtype, const float* A_dev, const float* B_dev, int32_t M, int32_t N,
                                     int32_t K, void* A_op_dev, void* B_op_dev, float* scales_dev, void* stream) {
  PM_REQUIRE(dtype >= 0 && dtype <= 2 && M > 0 && N > 0 && K > 0, PM_EINVAL, "bad dtype or shape");
  PM_REQUIRE(A_dev && B_dev && A_op_dev && B_op_dev, PM_EINVAL, "null pointer");
  PM_REQUIRE(dtype != PM_FP8E4M3 || scales_dev, PM_EINVAL, "FP8 needs scales_dev (4 floats)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int sms = std::max(1, sm_count());
  const int64_t nA = (int64_t)M * K, nB = (int64_t)K * N;
  unsigned int* amax = nullptr;
  if (dtype == PM_FP8E4M3) {
    amax = reinterpret_cast<unsigned int*>(scales_dev + 2);
    PM_CUDA(cudaMemsetAsync(amax, 0, 2 * sizeof(unsigned int), s));
    amax_kernel<<<sms * 4, 256, 0, s>>>(A_dev, nA, amax);
    amax_kernel<<<sms * 4, 256, 0, s>>>(B_dev, nB, amax + 1);
    pm_status st = launch_status("amax_kernel");
    if (st != PM_OK) return st;
  }
  float* a_lo = dtype == PM_FP32 ? static_cast<float*>(A_op_dev) + nA : nullptr;
  float* b_lo = dtype == PM_FP32 ? static_cast<float*>(B_op_dev) + (int64_t)N * K : nullptr;
  convert_rows_kernel<<<sms * 8, 256, 0, s>>>(A_dev, nA, dtype, A_op_dev, a_lo, amax,
                                              dtype == PM_FP8E4M3 ? scales_dev : nullptr);
  pm_status st = launch_status("convert_rows_kernel");
  if (st != PM_OK) return st;
  dim3 grid((N + 31) / 32, (K + 31) / 32);
  PM_REQUIRE(grid.y <= 65535, PM_EINVAL, "K too large for the transpose grid");
  transpose_convert_kernel<<<grid, dim3(32, 8), 0, s>>>(B_dev, K, N, dtype, B_op_dev, b_lo,
                                                          amax ? amax + 1 : nullptr,
                                                          dtype == PM_FP8E4M3 ? scales_dev + 1 : nullptr);
  return launch_status("transpose_convert_kernel");
}

extern "C" pm_status pm_gemm_run(const pm_cfg* cfg, const void* A_op_dev, const void* B_op_dev, float* C_dev,
                                 const float* scales_dev, void* stream) {
  PM_REQUIRE(cfg != nullptr, PM_EINVAL, "cfg is NULL");
  return gemm_launch(*cfg, A_op_dev, B_op_dev, C_dev, scales_dev, static_cast<cudaStream_t>(stream));
}

extern "C" pm_status pm_grouped_gemm_run(int32_t G, const int32_t* M_host, int32_t N, int32_t K,
                                         const int16_t* BM_host, const int16_t* BN_host, int32_t BK,
                                         int32_t stages, int32_t cta_group, const void* A_op_dev,
                                         const void* B_op_dev, float* C_dev, void* stream) {
  (void)G; (void)M_host; (void)N; (void)K; (void)BM_host; (void)BN_host; (void)BK; (void)stages;
  (void)cta_group; (void)A_op_dev; (void)B_op_dev; (void)C_dev; (void)stream;
  pm::set_error("grouped GEMM is not built yet");
  return PM_EUNSUPPORTED;
}
