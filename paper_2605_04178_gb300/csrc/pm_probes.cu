// Calibration probes (arxiv 2605.04178, Sec. V-A microbenchmarks, re-targeted
// to GB300): STREAM-style copy and triad for the memory-bound class (Eq. 16),
// a TMA 2D tile copy for L_TMA / B_TMA (Eq. 4), and a pointer chase for the
// latency of each memory level (Sec. III-B cites Mei & Chu's p-chase).
#include <algorithm>
#include <vector>

#include "pm_internal.cuh"

namespace pm {

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
  for (int i = 0; i < reps && st == PM_OK; ++i, ++launches) {
    cudaEventRecord(ev[2 * i], s);
    st = probe_launch(launches == 0 ? args : &cont, buf0, buf1, buf2, s);
    cudaEventRecord(ev[2 * i + 1], s);
  }
  cudaError_t e = cudaStreamSynchronize(s);
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
  if (args->kind == PM_PROBE_PCHASE) {
    uint32_t fi = 0;
    PM_CUDA(cudaMemcpy(&fi, buf1, 4, cudaMemcpyDeviceToHost));
    out->final_index = fi;
  }
  if (args->kind == PM_PROBE_TMA2D) {
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
