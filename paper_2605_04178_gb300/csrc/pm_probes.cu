// Calibration probes (arxiv 2605.04178, Sec. V-A microbenchmarks, re-targeted
// to GB300): STREAM-style copy and triad for the memory-bound class (Eq. 16),
// a TMA 2D tile copy for L_TMA / B_TMA (Eq. 4), and a pointer chase for the
// latency of each memory level (Sec. III-B cites Mei & Chu's p-chase).
#include <algorithm>
#include <mutex>
#include <vector>

#include "pm_internal.cuh"

namespace pm {

// TMEM address of lane 32*warp, column 0 (a warp may only touch its quarter).
__device__ __forceinline__ uint32_t tmem_base_row(uint32_t base, int warp) {
  return base + ((uint32_t)(32 * (warp & 3)) << 16);
}

// ------------------------------------------------------------------- copy/triad
// 128-bit loads and stores, four independent vectors in flight per thread,
// grid sized to a multiple of the SM count (HBM-bound: 8 B/elem copy,
// 12 B/elem triad).
constexpr int kStreamThreads = 256;
constexpr int kStreamUnroll = 4;

__global__ void __launch_bounds__(kStreamThreads) copy_kernel(const float4* __restrict__ src,
                                                              float4* __restrict__ dst, int64_t n4,
                                                              const float* __restrict__ src_tail,
                                                              float* __restrict__ dst_tail, int tail) {
  const int64_t stride = (int64_t)gridDim.x * kStreamThreads;
  int64_t i = (int64_t)blockIdx.x * kStreamThreads + threadIdx.x;
  for (; i + (kStreamUnroll - 1) * stride < n4; i += kStreamUnroll * stride) {
    float4 v[kStreamUnroll];
#pragma unroll
    for (int u = 0; u < kStreamUnroll; ++u) v[u] = __ldcs(src + i + u * stride);
#pragma unroll
    for (int u = 0; u < kStreamUnroll; ++u) __stcs(dst + i + u * stride, v[u]);
  }
  for (; i < n4; i += stride) __stcs(dst + i, __ldcs(src + i));
  if (blockIdx.x == 0 && threadIdx.x < tail) dst_tail[threadIdx.x] = src_tail[threadIdx.x];
}

__global__ void __launch_bounds__(kStreamThreads) triad_kernel(float4* __restrict__ a, const float4* __restrict__ b,
                                                               const float4* __restrict__ c, float s, int64_t n4,
                                                               float* __restrict__ a_tail,
                                                               const float* __restrict__ b_tail,
                                                               const float* __restrict__ c_tail, int tail) {
  const int64_t stride = (int64_t)gridDim.x * kStreamThreads;
  int64_t i = (int64_t)blockIdx.x * kStreamThreads + threadIdx.x;
  for (; i + (kStreamUnroll - 1) * stride < n4; i += kStreamUnroll * stride) {
    float4 vb[kStreamUnroll], vc[kStreamUnroll];
#pragma unroll
    for (int u = 0; u < kStreamUnroll; ++u) {
      vb[u] = __ldcs(b + i + u * stride);
      vc[u] = __ldcs(c + i + u * stride);
    }
#pragma unroll
    for (int u = 0; u < kStreamUnroll; ++u) {
      float4 r;
      r.x = __fmaf_rn(s, vc[u].x, vb[u].x);
      r.y = __fmaf_rn(s, vc[u].y, vb[u].y);
      r.z = __fmaf_rn(s, vc[u].z, vb[u].z);
      r.w = __fmaf_rn(s, vc[u].w, vb[u].w);
      __stcs(a + i + u * stride, r);
    }
  }
  for (; i < n4; i += stride) {
    const float4 vb = __ldcs(b + i), vc = __ldcs(c + i);
    float4 r;
    r.x = __fmaf_rn(s, vc.x, vb.x);
    r.y = __fmaf_rn(s, vc.y, vb.y);
    r.z = __fmaf_rn(s, vc.z, vb.z);
    r.w = __fmaf_rn(s, vc.w, vb.w);
    __stcs(a + i, r);
  }
  if (blockIdx.x == 0 && threadIdx.x < tail) a_tail[threadIdx.x] = __fmaf_rn(s, c_tail[threadIdx.x], b_tail[threadIdx.x]);
}

// ---------------------------------------------------------------- pointer chase
// One thread follows the cycle; node j's successor is the word at j*16.
// start == kContinue resumes from the node the previous launch ended on, so
// repeated launches keep walking new nodes instead of re-walking cached ones.
constexpr uint32_t kContinue = 0xFFFFFFFFu;

__global__ void pchase_kernel(const uint32_t* __restrict__ buf, uint32_t start, int64_t hops,
                              uint32_t* __restrict__ out) {
  uint32_t j = start == kContinue ? *out : start;
  for (int64_t h = 0; h < hops; ++h) j = buf[(size_t)j * 16];
  *out = j;
}

// ----------------------------------------------------------------- TMA 2D copy
// One persistent CTA per SM; one thread drives a ring of `depth` tile slots:
// TMA load (completion on full[s]) -> TMA store of the same slot; a slot is
// refilled once the store that reads it has finished reading shared memory.
constexpr int kTmaMaxDepth = 4;

__global__ void __launch_bounds__(32) tma2d_copy_kernel(const __grid_constant__ CUtensorMap src,
                                                        const __grid_constant__ CUtensorMap dst, int tiles_r,
                                                        int tiles_c, int tile_r, int tile_c, int depth,
                                                        uint32_t slot_bytes, Watchdog wd) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[kTmaMaxDepth];
  if (threadIdx.x != 0) return;
  const uint32_t base = (smem_u32(smem) + 127u) & ~127u;
  const uint32_t tile_bytes = (uint32_t)tile_r * tile_c * 4u;
  for (int s = 0; s < depth; ++s) mbar_init(smem_u32(&full[s]), 1);
  fence_mbar_init();
  prefetch_tmap(&src);
  prefetch_tmap(&dst);
  const int nt = tiles_r * tiles_c;
  const int mine = (nt - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;  // tiles of this CTA
  auto tile_of = [&](int i, int& x, int& y) {
    const int t = (int)blockIdx.x + i * (int)gridDim.x;
    y = (t / tiles_c) * tile_r;
    x = (t % tiles_c) * tile_c;
  };
  int issued = 0;
  for (; issued < depth && issued < mine; ++issued) {
    int x, y;
    tile_of(issued, x, y);
    const uint32_t b = smem_u32(&full[issued]);
    mbar_arrive_expect_tx(b, tile_bytes);
    tma_load_2d(base + issued * slot_bytes, &src, b, x, y);
  }
  bool ok = true;
  int i = 0;
  for (; i < mine; ++i) {
    const int s = i % depth;
    if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((i / depth) & 1), wd, nullptr, SITE_TMA_PROBE)) {
      ok = false;
      break;
    }
    int x, y;
    tile_of(i, x, y);
    tma_store_2d(&dst, base + s * slot_bytes, x, y);
    bulk_commit();
    if (issued < mine) {
      bulk_wait_read<0>();  // the slot's store has read shared memory
      int x2, y2;
      tile_of(issued, x2, y2);
      const uint32_t b = smem_u32(&full[s]);
      mbar_arrive_expect_tx(b, tile_bytes);
      tma_load_2d(base + s * slot_bytes, &src, b, x2, y2);
      ++issued;
    }
  }
  if (!ok) {
    // Give the loads already issued a bounded chance to land before exiting.
    Watchdog wd2 = wd;
    for (int j = i; j < issued; ++j)
      mbar_wait(smem_u32(&full[j % depth]), (uint32_t)((j / depth) & 1), wd2, nullptr, SITE_TMA_PROBE);
  }
  bulk_wait_all();
}

// ------------------------------------------------ Blackwell instruction probes
// (Sec. V-A (iii)-(iv): tcgen05.mma throughput by shape and precision, mbarrier
// wait latency, TMEM load/store bandwidth.)  Each computes a checkable value.

// One CTA (pair) per SM issues `iters` back-to-back MMAs of one shape from
// operands of 1.0 into one accumulator, so D = iters * k_instr exactly.
template <int CG, int KIND>
__global__ void __launch_bounds__(128, 1) mma_probe_kernel(int64_t iters, int M, int N, uint32_t* __restrict__ out,
                                                           Watchdog wd) {
  extern __shared__ __align__(1024) uint8_t smp[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = CG == 2 ? cluster_ctarank() : 0u;
  const uint32_t base = (smem_u32(smp) + 1023u) & ~1023u;
  uint32_t* p = reinterpret_cast<uint32_t*>(smp + (base - smem_u32(smp)));
  const uint32_t one = KIND == 0 ? 0x3F803F80u : (KIND == 1 ? 0x3F800000u : 0x38383838u);
  for (int i = threadIdx.x; i < 48 * 1024 / 4; i += blockDim.x) p[i] = one;   // A 16 KB, B 32 KB
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc<CG>(smem_u32(&slot), 256);
    tmem_relinquish<CG>();
  }
  tc_fence_before();
  if constexpr (CG == 2) cluster_sync(); else __syncthreads();
  tc_fence_after();
  const uint32_t tm = slot;
  if (warp == 1 && lane == 0 && rank == 0) {
    const uint32_t fmt = KIND == 0 ? 1u : (KIND == 1 ? 2u : 0u);
    const uint32_t idesc = instr_desc(fmt, (uint32_t)M, (uint32_t)N);
    const uint64_t ad = smem_desc(base, 1024, 2), bd = smem_desc(base + 16384, 1024, 2);
    for (int64_t i = 0; i < iters; ++i) umma<CG, KIND>(tm, ad, bd, idesc, i > 0 ? 1u : 0u);
    if constexpr (CG == 1) umma_commit(smem_u32(&bar));
    else umma_commit_pair(smem_u32(&bar), (uint16_t)3);
  }
  if (warp == 0 && lane == 0) mbar_wait(smem_u32(&bar), 0u, wd, nullptr, SITE_MMA_PROBE);
  __syncthreads();
  tc_fence_after();
  if (warp == 0) {
    uint32_t r[32];
    tmem_ld_32x32b_x32(tm, r);
    tmem_ld_wait();
    if (lane == 0) out[blockIdx.x] = r[0];
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (CG == 2) cluster_sync();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc<CG>(tm, 256);
  }
}

// Two threads of different warps pass a token through two mbarriers `iters`
// times; out[0] = completed round trips.
__global__ void __launch_bounds__(64) mbar_probe_kernel(int64_t iters, uint32_t* __restrict__ out, Watchdog wd) {
  __shared__ __align__(8) uint64_t bar[2];
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar[0]), 1);
    mbar_init(smem_u32(&bar[1]), 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t done = 0;
    for (int64_t i = 0; i < iters; ++i) {
      mbar_arrive(smem_u32(&bar[0]));
      if (!mbar_wait(smem_u32(&bar[1]), (uint32_t)(i & 1), wd, nullptr, SITE_MBAR_PROBE)) break;
      ++done;
    }
    out[0] = (uint32_t)done;
  } else if (threadIdx.x == 32) {
    for (int64_t i = 0; i < iters; ++i) {
      if (!mbar_wait(smem_u32(&bar[0]), (uint32_t)(i & 1), wd, nullptr, SITE_MBAR_PROBE)) break;
      mbar_arrive(smem_u32(&bar[1]));
    }
  }
}

// TMEM bandwidth: every SM fills its 128 lanes x 512 columns with
// lane*512 + column; 8 warps (two per 32-lane quarter, one per column half)
// then make `iters` passes of tcgen05.ld, four 32-column loads in flight per
// wait, summing what they read (store = 0), or of tcgen05.st writing
// value + pass (store = 1) followed by one summing read pass.
// out[cta*256 + thread] = the thread's sum (mod 2^32) over its 256 columns.
__global__ void __launch_bounds__(256, 1) tmem_probe_kernel(int64_t iters, int store, uint32_t* __restrict__ out) {
  __shared__ uint32_t slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    tmem_alloc<1>(smem_u32(&slot), 512);
    tmem_relinquish<1>();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t row = tmem_base_row(slot, warp) + (uint32_t)(256 * (warp >> 2));
  const uint32_t lg = (uint32_t)(32 * (warp & 3) + lane);
  const uint32_t c0 = (uint32_t)(256 * (warp >> 2));
  uint32_t r[32];
  for (int c = 0; c < 8; ++c) {
#pragma unroll
    for (int v = 0; v < 32; ++v) r[v] = lg * 512u + c0 + (uint32_t)(32 * c + v);
    tmem_st_32x32b_x32(row + 32u * c, r);
  }
  tmem_st_wait();
  uint32_t acc = 0;
  if (!store) {
    for (int64_t it = 0; it < iters; ++it)
      for (int c = 0; c < 8; c += 4) {
        uint32_t r1[32], r2[32], r3[32];
        tmem_ld_32x32b_x32(row + 32u * c, r);
        tmem_ld_32x32b_x32(row + 32u * (c + 1), r1);
        tmem_ld_32x32b_x32(row + 32u * (c + 2), r2);
        tmem_ld_32x32b_x32(row + 32u * (c + 3), r3);
        tmem_ld_wait();
#pragma unroll
        for (int v = 0; v < 32; ++v) acc += (r[v] + r1[v]) + (r2[v] + r3[v]);
      }
  } else {
    for (int64_t it = 0; it < iters; ++it) {
      for (int c = 0; c < 8; ++c) {
#pragma unroll
        for (int v = 0; v < 32; ++v) r[v] = lg * 512u + c0 + (uint32_t)(32 * c + v) + (uint32_t)it;
        tmem_st_32x32b_x32(row + 32u * c, r);
      }
      tmem_st_wait();
    }
    for (int c = 0; c < 8; ++c) {
      tmem_ld_32x32b_x32(row + 32u * c, r);
      tmem_ld_wait();
#pragma unroll
      for (int v = 0; v < 32; ++v) acc += r[v];
    }
  }
  out[(size_t)blockIdx.x * 256 + threadIdx.x] = acc;
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc<1>(slot, 512);
  }
}

// Five-point stencil over a rows x cols FP32 grid (the stencil class of the
// generic roofline path): interior points take
//   out = 0.5 x + 0.125 ((up + down) + (left + right)),
// each operation rounded on its own (no contraction), border points are
// copied.  One thread per output point, 32 x 8 blocks.
__global__ void __launch_bounds__(256) stencil5_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                       int64_t rows, int64_t cols) {
  const int64_t j = (int64_t)blockIdx.x * 32 + threadIdx.x;
  const int64_t i = (int64_t)blockIdx.y * 8 + threadIdx.y;
  if (i >= rows || j >= cols) return;
  const int64_t k = i * cols + j;
  const float x = __ldg(in + k);
  if (i == 0 || j == 0 || i == rows - 1 || j == cols - 1) {
    out[k] = x;
    return;
  }
  const float vert = __fadd_rn(__ldg(in + k - cols), __ldg(in + k + cols));
  const float horz = __fadd_rn(__ldg(in + k - 1), __ldg(in + k + 1));
  out[k] = __fadd_rn(__fmul_rn(0.5f, x), __fmul_rn(0.125f, __fadd_rn(vert, horz)));
}

// The same stencil with four consecutive points per thread (cols % 4 == 0,
// 16-byte aligned rows): 128-bit loads of the point's row and the rows above
// and below; the left and right neighbours come from the adjacent lanes'
// vectors by shuffle (one scalar load at each warp edge).  Same arithmetic
// per point as stencil5_kernel, so the results are identical.
__device__ __forceinline__ float stencil_point(float x, float up, float down, float left, float right) {
  const float vert = __fadd_rn(up, down);
  const float horz = __fadd_rn(left, right);
  return __fadd_rn(__fmul_rn(0.5f, x), __fmul_rn(0.125f, __fadd_rn(vert, horz)));
}

__global__ void __launch_bounds__(256) stencil5_vec4_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                            int64_t rows, int64_t cols) {
  const int64_t c4 = cols / 4;                         // float4 columns
  const int64_t j4 = (int64_t)blockIdx.x * 32 + threadIdx.x;
  const int64_t i = (int64_t)blockIdx.y * 8 + threadIdx.y;
  const bool live = i < rows && j4 < c4;
  const float4* in4 = reinterpret_cast<const float4*>(in);
  float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
  if (live) x = __ldg(in4 + i * c4 + j4);
  // neighbours across the vector boundary: lane - 1's .w and lane + 1's .x
  float left = __shfl_up_sync(0xffffffffu, x.w, 1);
  float right = __shfl_down_sync(0xffffffffu, x.x, 1);
  if (!live) return;
  const int64_t k = i * cols + 4 * j4;
  if (threadIdx.x == 0 && j4 > 0) left = __ldg(in + k - 1);
  if ((threadIdx.x == 31 || j4 == c4 - 1) && j4 + 1 < c4) right = __ldg(in + k + 4);
  float4 y = x;
  if (i > 0 && i < rows - 1) {
    const float4 u = __ldg(in4 + (i - 1) * c4 + j4);
    const float4 d = __ldg(in4 + (i + 1) * c4 + j4);
    const bool first = j4 == 0, last = j4 == c4 - 1;
    if (!first) y.x = stencil_point(x.x, u.x, d.x, left, x.y);
    y.y = stencil_point(x.y, u.y, d.y, x.x, x.z);
    y.z = stencil_point(x.z, u.z, d.z, x.y, x.w);
    if (!last) y.w = stencil_point(x.w, u.w, d.w, x.z, right);
  }
  reinterpret_cast<float4*>(out)[i * c4 + j4] = y;
}

// Device address of page-locked host memory registered with CUDA (the
// allocation must be CUDA pinned memory; anything else is refused).
static pm_status mapped_host_pointer(void* host, void** out) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, host);
  if (e != cudaSuccess) return cuda_fail(e, "cudaPointerGetAttributes");
  PM_REQUIRE(at.type == cudaMemoryTypeHost && at.devicePointer != nullptr, PM_EINVAL,
             "buffer is not CUDA page-locked host memory mapped into the device address space");
  *out = at.devicePointer;
  return PM_OK;
}

static int stream_grid(int64_t n4) {
  const int sms = std::max(1, sm_count());
  const int64_t need = (n4 + (int64_t)kStreamThreads * kStreamUnroll - 1) / ((int64_t)kStreamThreads * kStreamUnroll);
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * 8));
}

static int tma_depth(uint32_t slot_bytes) {
  const uint32_t budget = 200u * 1024u;
  return std::max(1, std::min<int>(kTmaMaxDepth, (int)(budget / slot_bytes)));
}

struct TmaProbeCache {
  const void* src = nullptr;
  const void* dst = nullptr;
  int64_t rows = 0, cols = 0;
  int tr = 0, tc = 0;
  CUtensorMap ms, md;
};
static thread_local TmaProbeCache g_tma_cache;
void clear_probe_tmap_cache_this_thread() { g_tma_cache = TmaProbeCache(); }

static pm_status probe_launch(const pm_probe_args* a, void* buf0, void* buf1, void* buf2, cudaStream_t s) {
  switch (a->kind) {
    case PM_PROBE_COPY: {
      PM_REQUIRE(buf0 && buf1 && a->n > 0, PM_EINVAL, "copy probe: null buffer or n <= 0");
      PM_REQUIRE(((uintptr_t)buf0 & 15) == 0 && ((uintptr_t)buf1 & 15) == 0, PM_EINVAL,
                 "copy probe: buffers must be 16-byte aligned");
      const int64_t n4 = a->n / 4;
      const int tail = (int)(a->n - n4 * 4);
      copy_kernel<<<stream_grid(n4), kStreamThreads, 0, s>>>(
          (const float4*)buf0, (float4*)buf1, n4, (const float*)buf0 + n4 * 4, (float*)buf1 + n4 * 4, tail);
      return launch_status("copy_kernel");
    }
    case PM_PROBE_TRIAD: {
      PM_REQUIRE(buf0 && buf1 && buf2 && a->n > 0, PM_EINVAL, "triad probe: null buffer or n <= 0");
      PM_REQUIRE((((uintptr_t)buf0 | (uintptr_t)buf1 | (uintptr_t)buf2) & 15) == 0, PM_EINVAL,
                 "triad probe: buffers must be 16-byte aligned");
      const int64_t n4 = a->n / 4;
      const int tail = (int)(a->n - n4 * 4);
      triad_kernel<<<stream_grid(n4), kStreamThreads, 0, s>>>(
          (float4*)buf0, (const float4*)buf1, (const float4*)buf2, a->scalar, n4, (float*)buf0 + n4 * 4,
          (const float*)buf1 + n4 * 4, (const float*)buf2 + n4 * 4, tail);
      return launch_status("triad_kernel");
    }
    case PM_PROBE_PCHASE: {
      PM_REQUIRE(buf0 && buf1 && a->n > 0 && a->hops >= 0, PM_EINVAL, "pchase probe: bad arguments");
      PM_REQUIRE(a->start < (uint64_t)a->n || a->start == kContinue, PM_EINVAL,
                 "pchase probe: start outside the node range");
      pchase_kernel<<<1, 1, 0, s>>>((const uint32_t*)buf0, a->start, a->hops, (uint32_t*)buf1);
      return launch_status("pchase_kernel");
    }
    case PM_PROBE_TMA2D: {
      PM_REQUIRE(buf0 && buf1 && a->rows > 0 && a->cols > 0, PM_EINVAL, "tma2d probe: bad arguments");
      PM_REQUIRE(a->tile_r >= 8 && a->tile_r <= 256 && a->tile_c >= 4 && a->tile_c <= 256 && a->tile_c % 4 == 0,
                 PM_EINVAL, "tma2d probe: tile %dx%d outside [8,256]x[4,256] (cols multiple of 4)", a->tile_r,
                 a->tile_c);
      PM_REQUIRE(a->rows < (1ll << 31) && a->cols < (1ll << 31), PM_EINVAL, "tma2d probe: matrix too large");
      TmaProbeCache& c = g_tma_cache;
      if (c.src != buf0 || c.dst != buf1 || c.rows != a->rows || c.cols != a->cols || c.tr != a->tile_r ||
          c.tc != a->tile_c) {
        pm_status st = make_tmap_2d(&c.ms, buf0, TMAP_F32, a->rows, a->cols, a->tile_r, a->tile_c, 0);
        if (st != PM_OK) return st;
        st = make_tmap_2d(&c.md, buf1, TMAP_F32, a->rows, a->cols, a->tile_r, a->tile_c, 0);
        if (st != PM_OK) return st;
        c.src = buf0; c.dst = buf1; c.rows = a->rows; c.cols = a->cols; c.tr = a->tile_r; c.tc = a->tile_c;
      }
      const uint32_t slot = ((uint32_t)a->tile_r * a->tile_c * 4u + 127u) & ~127u;
      const int depth = tma_depth(slot);
      const int smem = depth * (int)slot + 128;
      PM_CUDA(cudaFuncSetAttribute(tma2d_copy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      const int tiles_r = (int)((a->rows + a->tile_r - 1) / a->tile_r);
      const int tiles_c = (int)((a->cols + a->tile_c - 1) / a->tile_c);
      const int grid = std::max(1, std::min(sm_count(), tiles_r * tiles_c));
      unsigned int* w = watchdog_word();
      PM_REQUIRE(w != nullptr, PM_ECUDA, "watchdog word unavailable");
      tma2d_copy_kernel<<<grid, 32, smem, s>>>(c.ms, c.md, tiles_r, tiles_c, a->tile_r, a->tile_c, depth, slot,
                                               Watchdog{w, watchdog_limit_ns()});
      return launch_status("tma2d_copy_kernel");
    }
    case PM_PROBE_H2D:
    case PM_PROBE_D2H: {
      PM_REQUIRE(buf0 && buf1 && a->n > 0, PM_EINVAL, "copy-engine probe: null buffer or n <= 0");
      PM_CUDA(cudaMemcpyAsync(buf1, buf0, (size_t)a->n,
                              a->kind == PM_PROBE_H2D ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost, s));
      return PM_OK;
    }
    case PM_PROBE_HOST_READ:
    case PM_PROBE_HOST_WRITE: {
      // SMs stream the host buffer through its device mapping (no copy engine)
      PM_REQUIRE(buf0 && buf1 && a->n > 0, PM_EINVAL, "host-link probe: null buffer or n <= 0");
      void* host = a->kind == PM_PROBE_HOST_READ ? buf0 : buf1;
      void* mapped = nullptr;
      pm_status st = mapped_host_pointer(host, &mapped);
      if (st != PM_OK) return st;
      const void* src = a->kind == PM_PROBE_HOST_READ ? mapped : buf0;
      void* dst = a->kind == PM_PROBE_HOST_READ ? buf1 : mapped;
      PM_REQUIRE((((uintptr_t)src | (uintptr_t)dst) & 15) == 0, PM_EINVAL,
                 "host-link probe: buffers must be 16-byte aligned");
      const int64_t n4 = a->n / 4;
      const int tail = (int)(a->n - n4 * 4);
      copy_kernel<<<stream_grid(n4), kStreamThreads, 0, s>>>((const float4*)src, (float4*)dst, n4,
                                                             (const float*)src + n4 * 4, (float*)dst + n4 * 4, tail);
      return launch_status("copy_kernel");
    }
    case PM_PROBE_STENCIL: {
      PM_REQUIRE(buf0 && buf1 && buf0 != buf1 && a->rows > 0 && a->cols > 0, PM_EINVAL,
                 "stencil probe: need distinct buffers and a positive grid");
      PM_REQUIRE((a->rows + 7) / 8 < 65536 && (a->cols + 31) / 32 < (1ll << 31), PM_EINVAL,
                 "stencil probe: grid too large");
      if (a->cols % 4 == 0 && a->cols >= 8 && (((uintptr_t)buf0 | (uintptr_t)buf1) & 15) == 0) {
        const dim3 grid((unsigned)((a->cols / 4 + 31) / 32), (unsigned)((a->rows + 7) / 8));
        stencil5_vec4_kernel<<<grid, dim3(32, 8), 0, s>>>((const float*)buf0, (float*)buf1, a->rows, a->cols);
        return launch_status("stencil5_vec4_kernel");
      }
      const dim3 grid((unsigned)((a->cols + 31) / 32), (unsigned)((a->rows + 7) / 8));
      stencil5_kernel<<<grid, dim3(32, 8), 0, s>>>((const float*)buf0, (float*)buf1, a->rows, a->cols);
      return launch_status("stencil5_kernel");
    }
    case PM_PROBE_MMA: {
      const int cg = (int)a->rows, dt = (int)a->cols, M = a->tile_c, N = a->tile_r;
      PM_REQUIRE(buf0 && a->n >= 1 && a->n <= (1 << 19), PM_EINVAL, "mma probe: need buf0 and 1 <= n <= 2^19");
      PM_REQUIRE(cg == 1 || cg == 2, PM_EINVAL, "mma probe: rows (cta_group) must be 1 or 2");
      PM_REQUIRE(dt >= 0 && dt <= 2, PM_EINVAL, "mma probe: cols (dtype) must be a pm_dtype");
      PM_REQUIRE(cg == 1 ? (M == 64 || M == 128) : (M == 128 || M == 256), PM_EINVAL,
                 "mma probe: M %d not an instruction height for cta_group %d", M, cg);
      PM_REQUIRE(N >= 16 && N <= 256 && N % 16 == 0, PM_EINVAL, "mma probe: N must be a multiple of 16 in [16,256]");
      int grid = a->start ? (int)a->start : sm_count();
      if (cg == 2) grid &= ~1;
      PM_REQUIRE(grid >= cg, PM_EINVAL, "mma probe: grid too small");
      unsigned int* w = watchdog_word();
      PM_REQUIRE(w != nullptr, PM_ECUDA, "watchdog word unavailable");
      Watchdog wd{w, watchdog_limit_ns()};
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(grid);
      cfg.blockDim = dim3(128);
      cfg.dynamicSmemBytes = 49 * 1024;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 2;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      if (cg == 2) { cfg.attrs = attr; cfg.numAttrs = 1; }
      uint32_t* out = static_cast<uint32_t*>(buf0);
      cudaError_t e;
#define PM_MMA_PROBE(CG, KIND)                                                                           \
  do {                                                                                                   \
    cudaFuncSetAttribute(mma_probe_kernel<CG, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, 49 * 1024); \
    e = cudaLaunchKernelEx(&cfg, mma_probe_kernel<CG, KIND>, a->n, M, N, out, wd);                     \
  } while (0)
      if (cg == 1) {
        if (dt == PM_BF16) PM_MMA_PROBE(1, 0); else if (dt == PM_FP32) PM_MMA_PROBE(1, 1); else PM_MMA_PROBE(1, 2);
      } else {
        if (dt == PM_BF16) PM_MMA_PROBE(2, 0); else if (dt == PM_FP32) PM_MMA_PROBE(2, 1); else PM_MMA_PROBE(2, 2);
      }
#undef PM_MMA_PROBE
      if (e != cudaSuccess) return cuda_fail(e, "mma_probe_kernel");
      return PM_OK;
    }
    case PM_PROBE_MBAR: {
      PM_REQUIRE(buf0 && a->n >= 1, PM_EINVAL, "mbarrier probe: need buf0 and n >= 1");
      unsigned int* w = watchdog_word();
      PM_REQUIRE(w != nullptr, PM_ECUDA, "watchdog word unavailable");
      mbar_probe_kernel<<<1, 64, 0, s>>>(a->n, static_cast<uint32_t*>(buf0), Watchdog{w, watchdog_limit_ns()});
      return launch_status("mbar_probe_kernel");
    }
    case PM_PROBE_TMEM_LD:
    case PM_PROBE_TMEM_ST: {
      PM_REQUIRE(buf0 && a->n >= 1, PM_EINVAL, "tmem probe: need buf0 and n >= 1");
      tmem_probe_kernel<<<sm_count(), 256, 0, s>>>(a->n, a->kind == PM_PROBE_TMEM_ST ? 1 : 0,
                                                    static_cast<uint32_t*>(buf0));
      return launch_status("tmem_probe_kernel");
    }
    default:
      set_error("unknown probe kind %d", a->kind);
      return PM_EINVAL;
  }
}

static double probe_bytes(const pm_probe_args* a) {
  switch (a->kind) {
    case PM_PROBE_COPY: return 8.0 * (double)a->n;
    case PM_PROBE_TRIAD: return 12.0 * (double)a->n;
    case PM_PROBE_TMA2D: return 8.0 * (double)a->rows * (double)a->cols;
    case PM_PROBE_PCHASE: return 4.0 * (double)a->hops;
    case PM_PROBE_H2D:
    case PM_PROBE_D2H: return (double)a->n;
    case PM_PROBE_HOST_READ:
    case PM_PROBE_HOST_WRITE: return 4.0 * (double)a->n;
    case PM_PROBE_STENCIL: return 8.0 * (double)a->rows * (double)a->cols;
    case PM_PROBE_MMA: {
      // FLOPs of the launch: issuing CTAs x n x 2 M N k_instr
      const int cg = (int)a->rows, dt = (int)a->cols;
      int grid = a->start ? (int)a->start : sm_count();
      if (cg == 2) grid &= ~1;
      const double kin = dt == PM_FP32 ? 8.0 : (dt == PM_BF16 ? 16.0 : 32.0);
      return (double)(grid / cg) * (double)a->n * 2.0 * a->tile_c * a->tile_r * kin;
    }
    case PM_PROBE_MBAR: return 0.0;
    case PM_PROBE_TMEM_LD:
    case PM_PROBE_TMEM_ST: return (double)sm_count() * 128.0 * 512.0 * 4.0 * (double)a->n;
    default: return 0.0;
  }
}

}  // namespace pm

using namespace pm;

extern "C" pm_status pm_probe_launch(const pm_probe_args* args, void* buf0, void* buf1, void* buf2, void* stream) {
  PM_REQUIRE(args != nullptr, PM_EINVAL, "args is NULL");
  return probe_launch(args, buf0, buf1, buf2, static_cast<cudaStream_t>(stream));
}

extern "C" pm_status pm_probe_run(const pm_probe_args* args, void* buf0, void* buf1, void* buf2, int warmup,
                                  int reps, void* stream, pm_probe_result* out) {
  PM_REQUIRE(args != nullptr && out != nullptr, PM_EINVAL, "args or out is NULL");
  NvtxRange nvtx("pm_probe_run");
  PM_REQUIRE(warmup >= 0 && reps >= 1 && reps <= 100000, PM_EINVAL, "warmup >= 0 and 1 <= reps <= 1e5 required");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // pointer chase: every launch after the first continues the walk
  pm_probe_args cont = *args;
  if (args->kind == PM_PROBE_PCHASE) cont.start = kContinue;
  int launches = 0;
  for (int i = 0; i < warmup; ++i, ++launches) {
    pm_status st = probe_launch(launches == 0 ? args : &cont, buf0, buf1, buf2, s);
    if (st != PM_OK) return st;
  }
  std::vector<cudaEvent_t> ev(2 * (size_t)reps);
  for (auto& e : ev) PM_CUDA(cudaEventCreate(&e));
  pm_status st = PM_OK;
  pm_clock c0, c1;
  read_clock(&c0);
  for (int i = 0; i < reps && st == PM_OK; ++i, ++launches) {
    cudaEventRecord(ev[2 * i], s);
    st = probe_launch(launches == 0 ? args : &cont, buf0, buf1, buf2, s);
    cudaEventRecord(ev[2 * i + 1], s);
  }
  cudaError_t e = cudaStreamSynchronize(s);
  read_clock(&c1);
  std::vector<double> t;
  if (st == PM_OK && e == cudaSuccess) {
    for (int i = 0; i < reps; ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
      t.push_back(ms * 1e-3);
    }
  }
  for (auto& x : ev) cudaEventDestroy(x);
  if (st != PM_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  std::sort(t.begin(), t.end());
  auto q = [&](double f) {
    const double pos = f * (t.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, t.size() - 1);
    return t[lo] + (pos - lo) * (t[hi] - t[lo]);
  };
  out->median_s = q(0.5);
  out->p25_s = q(0.25);
  out->p75_s = q(0.75);
  out->min_s = t.front();
  out->bytes = probe_bytes(args);
  out->final_index = 0;
  clock_record(out, c0, c1);
  if (args->kind == PM_PROBE_PCHASE || args->kind == PM_PROBE_MBAR) {
    uint32_t fi = 0;
    PM_CUDA(cudaMemcpy(&fi, args->kind == PM_PROBE_PCHASE ? buf1 : buf0, 4, cudaMemcpyDeviceToHost));
    out->final_index = fi;
  }
  if (args->kind == PM_PROBE_TMA2D || args->kind == PM_PROBE_MMA || args->kind == PM_PROBE_MBAR) {
    unsigned int* w = watchdog_word();
    unsigned int h[2] = {0, 0};
    PM_CUDA(cudaMemcpy(h, w, sizeof(h), cudaMemcpyDeviceToHost));
    if (h[0] != 0) {
      PM_CUDA(cudaMemset(w, 0, 4 * sizeof(unsigned int)));
      set_error("device watchdog expired at site %u", h[1]);
      return PM_ETIMEOUT;
    }
  }
  return PM_OK;
}

// ------------------------------------------------ concurrent-stream probe
// Sec. III-A.6: N_c kernels in flight on N_c streams of one GPU take the
// single-stream time plus (N_c - 1) tau_c.  The probe launches one copy of a
// probe kernel on each of n_streams library-owned non-blocking streams, all
// released by one event recorded on the caller's stream and joined back on
// it, and times the makespan between the two events.
namespace pm {
constexpr int kMaxConcStreams = 8;
struct ConcStreams {
  bool made = false;
  cudaStream_t s[kMaxConcStreams];
};
static std::mutex g_conc_mu;
static ConcStreams g_conc[64];

void release_stream_pool() {
  std::lock_guard<std::mutex> lk(g_conc_mu);
  int cur = -1;
  cudaGetDevice(&cur);
  for (int dev = 0; dev < 64; ++dev) {
    ConcStreams& c = g_conc[dev];
    if (!c.made) continue;
    if (cudaSetDevice(dev) == cudaSuccess)
      for (int i = 0; i < kMaxConcStreams; ++i) cudaStreamDestroy(c.s[i]);
    c.made = false;
  }
  if (cur >= 0) cudaSetDevice(cur);
}

static pm_status conc_streams(cudaStream_t** out) {
  int dev = 0;
  PM_CUDA(cudaGetDevice(&dev));
  PM_REQUIRE(dev >= 0 && dev < 64, PM_EINVAL, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_conc_mu);
  ConcStreams& c = g_conc[dev];
  if (!c.made) {
    for (int i = 0; i < kMaxConcStreams; ++i) PM_CUDA(cudaStreamCreateWithFlags(&c.s[i], cudaStreamNonBlocking));
    c.made = true;
  }
  *out = c.s;
  return PM_OK;
}
}  // namespace pm

extern "C" pm_status pm_streams_run(const pm_probe_args* per_stream, int32_t n_streams, void* const* buf0,
                                    void* const* buf1, void* const* buf2, int warmup, int reps, void* stream,
                                    pm_probe_result* out) {
  using namespace pm;
  PM_REQUIRE(per_stream != nullptr && out != nullptr && buf0 != nullptr, PM_EINVAL, "null argument");
  PM_REQUIRE(n_streams >= 1 && n_streams <= kMaxConcStreams, PM_EINVAL, "n_streams %d outside [1, %d]", n_streams,
             kMaxConcStreams);
  const int k = per_stream->kind;
  PM_REQUIRE(k == PM_PROBE_COPY || k == PM_PROBE_TRIAD || k == PM_PROBE_MMA, PM_EINVAL,
             "concurrent-stream probe runs COPY, TRIAD or MMA kernels (kind %d)", k);
  PM_REQUIRE(k == PM_PROBE_MMA || buf1 != nullptr, PM_EINVAL, "copy/triad need buf1 arrays");
  PM_REQUIRE(k != PM_PROBE_TRIAD || buf2 != nullptr, PM_EINVAL, "triad needs buf2 arrays");
  PM_REQUIRE(warmup >= 0 && reps >= 1 && reps <= 100000, PM_EINVAL, "warmup >= 0 and 1 <= reps <= 1e5 required");
  NvtxRange nvtx("pm_streams_run");
  cudaStream_t* cs = nullptr;
  pm_status st = conc_streams(&cs);
  if (st != PM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int total = warmup + reps;
  std::vector<cudaEvent_t> ev(2 * (size_t)total), done((size_t)total * n_streams);
  for (auto& e : ev) PM_CUDA(cudaEventCreate(&e));
  for (auto& e : done) PM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  pm_clock c0, c1;
  read_clock(&c0);
  for (int r = 0; r < total && st == PM_OK; ++r) {
    cudaEventRecord(ev[2 * r], s);
    for (int i = 0; i < n_streams && st == PM_OK; ++i) {
      cudaStreamWaitEvent(cs[i], ev[2 * r], 0);
      st = probe_launch(per_stream, buf0[i], buf1 ? buf1[i] : nullptr, buf2 ? buf2[i] : nullptr, cs[i]);
      cudaEventRecord(done[(size_t)r * n_streams + i], cs[i]);
      cudaStreamWaitEvent(s, done[(size_t)r * n_streams + i], 0);
    }
    cudaEventRecord(ev[2 * r + 1], s);
  }
  cudaError_t e = cudaStreamSynchronize(s);
  read_clock(&c1);
  std::vector<double> t;
  if (st == PM_OK && e == cudaSuccess) {
    for (int r = warmup; r < total; ++r) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[2 * r], ev[2 * r + 1]);
      t.push_back(ms * 1e-3);
    }
  }
  for (auto& x : ev) cudaEventDestroy(x);
  for (auto& x : done) cudaEventDestroy(x);
  if (st != PM_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  std::sort(t.begin(), t.end());
  auto q = [&](double f) {
    const double pos = f * (t.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, t.size() - 1);
    return t[lo] + (pos - lo) * (t[hi] - t[lo]);
  };
  out->median_s = q(0.5);
  out->p25_s = q(0.25);
  out->p75_s = q(0.75);
  out->min_s = t.front();
  out->bytes = (double)n_streams * probe_bytes(per_stream);
  out->final_index = 0;
  clock_record(out, c0, c1);
  if (k == PM_PROBE_MMA) {
    unsigned int* w = watchdog_word();
    unsigned int h[2] = {0, 0};
    PM_CUDA(cudaMemcpy(h, w, sizeof(h), cudaMemcpyDeviceToHost));
    if (h[0] != 0) {
      PM_CUDA(cudaMemset(w, 0, 4 * sizeof(unsigned int)));
      set_error("device watchdog expired at site %u", h[1]);
      return PM_ETIMEOUT;
    }
  }
  return PM_OK;
}
