// Internal declarations and sm_103a PTX wrappers of libperfmodel.so.
//
// Everything device-side here is inline PTX for the Blackwell asynchronous
// machinery the stage model of arxiv 2605.04178 (Sec. III-A) is built on:
// mbarriers (T_sync = N_bar * L_mbar), TMA bulk tensor copies (Eq. 4),
// tensor memory allocation and tcgen05.mma / tcgen05.ld (Eqs. 2-3, 6).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/perfmodel.h"

namespace pm {

// ------------------------------------------------------------------ host side
void set_error(const char* fmt, ...);
pm_status cuda_fail(cudaError_t e, const char* what);
// Device watchdog word of the current device (4 x uint32: status, site, -, -).
unsigned int* watchdog_word();
// Limit of every bounded device wait, nanoseconds (env PM_WATCHDOG_MS, default 2000).
unsigned long long watchdog_limit_ns();
// Number of SMs of the current device.
int sm_count();
// Resources pm_shutdown releases: the library's stream pool (all devices), and
// the calling thread's host-transfer pipeline and tensor-map caches.
void release_stream_pool();
void release_host_pipe_this_thread();
void clear_tmap_caches_this_thread();
void clear_probe_tmap_cache_this_thread();
// Read-only NVML sample of the current device (false: NVML unavailable), and
// the timed region's clock record in a harness result.
bool read_clock(pm_clock* c);
void clock_record(pm_probe_result* out, const pm_clock& begin, const pm_clock& end);

// Named NVTX range over a scope (timing harnesses and pipelines); free when
// no profiler is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
// 2D tiled tensor map over a row-major [rows, cols] matrix of elem_bytes-wide
// elements, box box_cols x box_rows, swizzle 0/32/64/128 bytes.
pm_status make_tmap_2d(CUtensorMap* map, const void* base, int dtype_code, uint64_t rows, uint64_t cols,
                       uint32_t box_rows, uint32_t box_cols, int swizzle_bytes);
enum { TMAP_F32 = 0, TMAP_BF16 = 1, TMAP_U8 = 2 };

#define PM_CUDA(call)                                      \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return pm::cuda_fail(e_, #call); \
  } while (0)

#define PM_REQUIRE(cond, code, ...)  \
  do {                               \
    if (!(cond)) {                   \
      pm::set_error(__VA_ARGS__);    \
      return (code);                 \
    }                                \
  } while (0)

// Launch-error check after an async launch.
inline pm_status launch_status(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, what);
  return PM_OK;
}

// ------------------------------------------------------------- device helpers
struct Watchdog {
  unsigned int* word;
  unsigned long long limit_ns;
};

enum WatchSite : unsigned {
  SITE_SELFTEST = 1, SITE_TMA_PROBE = 2, SITE_GEMM_PRODUCER = 3, SITE_GEMM_MMA = 4,
  SITE_GEMM_EPILOGUE = 5, SITE_GEMM_TEARDOWN = 6, SITE_MMA_PROBE = 7, SITE_MBAR_PROBE = 8
};

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with this parity.  Gives up when the watchdog
// limit passes or when another role of the CTA already gave up (abort flag in
// shared memory); records PM_ETIMEOUT and the site in the device word.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const Watchdog& wd,
                                          volatile int* abort_flag, unsigned site) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (abort_flag != nullptr && *abort_flag) return false;
    if (globaltimer() - t0 > wd.limit_ns) {
      atomicCAS(&wd.word[0], 0u, (unsigned)(-PM_ETIMEOUT));
      atomicCAS(&wd.word[1], 0u, site);
      if (abort_flag != nullptr) *abort_flag = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Cluster-scope variants on an mbarrier given by its shared::cluster address.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cbar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cbar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx_cluster(uint32_t cbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cluster.shared::cluster.b64 _, [%0], %1;" ::"r"(cbar), "r"(bytes)
               : "memory");
}

// shared::cluster address of the same shared variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// TMA: 2D tile load into this CTA's shared memory, completion on an mbarrier
// of this CTA (bar given as a shared::cta address).
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int32_t x,
                                            int32_t y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

// TMA load whose completion is signalled on an mbarrier of either CTA of a
// CTA pair (bar given as a shared::cluster address).
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, uint32_t cbar, int32_t x,
                                                 int32_t y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4}], [%2];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(cbar), "r"(x), "r"(y)
      : "memory");
}

// TMA: 2D tile store from shared memory (bulk-group completion).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int32_t x, int32_t y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%2, %3}], [%1];"
               ::"l"(reinterpret_cast<uint64_t>(map)), "r"(src), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ------------------------------------------------------------- tensor memory
template <int CG>
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  if constexpr (CG == 1)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
  else
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}
template <int CG>
__device__ __forceinline__ void tmem_relinquish() {
  if constexpr (CG == 1)
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  else
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
template <int CG>
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  if constexpr (CG == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
  else
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// tcgen05.mma kinds: 0 = f16 (BF16 operands), 1 = tf32, 2 = f8f6f4 (e4m3).
// `issue` predicates the instruction: a converged warp can run the issue
// sequence together (its operands then stay warp-uniform) while one lane
// (issue != 0) issues.
template <int CG, int KIND>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                     uint32_t accumulate, uint32_t issue = 1u) {
// No "memory" clobber: the MMA reads shared memory through the async proxy,
// ordered after the barrier wait by the volatile asm sequence itself.
#define PM_UMMA(CGS, KS)                                                                        \
  asm volatile(                                                                                 \
      "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %4, 0;\n\tsetp.ne.b32 q, %5, 0;\n\t"              \
      "@q tcgen05.mma.cta_group::" CGS ".kind::" KS " [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem), \
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate), "r"(issue))
  if constexpr (CG == 1) {
    if constexpr (KIND == 0) PM_UMMA("1", "f16");
    else if constexpr (KIND == 1) PM_UMMA("1", "tf32");
    else PM_UMMA("1", "f8f6f4");
  } else {
    if constexpr (KIND == 0) PM_UMMA("2", "f16");
    else if constexpr (KIND == 1) PM_UMMA("2", "tf32");
    else PM_UMMA("2", "f8f6f4");
  }
#undef PM_UMMA
}

// TMEM strategy B (Sec. III-A.1): the A operand is read from tensor memory
// (128 lanes = rows, 32-bit columns packing K) instead of shared memory.
// One SM (cta_group::1); B still comes from a shared-memory descriptor.
template <int KIND>
__device__ __forceinline__ void umma_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate, uint32_t issue = 1u) {
#define PM_UMMA_TA(KS)                                                                            \
  asm volatile(                                                                                   \
      "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %4, 0;\n\tsetp.ne.b32 q, %5, 0;\n\t"                \
      "@q tcgen05.mma.cta_group::1.kind::" KS " [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),      \
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate), "r"(issue))
  if constexpr (KIND == 0) PM_UMMA_TA("f16");
  else if constexpr (KIND == 1) PM_UMMA_TA("tf32");
  else PM_UMMA_TA("f8f6f4");
#undef PM_UMMA_TA
}

// Copy a 128-row x 32-byte shared-memory matrix (described like an MMA
// operand) into 128 lanes x 8 columns of tensor memory.  Asynchronous; a
// later tcgen05.mma of the same thread sees the data, and tcgen05.commit
// tracks its completion together with the MMAs.
__device__ __forceinline__ void tmem_cp_128x256b(uint32_t taddr, uint64_t sdesc, uint32_t issue = 1u) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q tcgen05.cp.cta_group::1.128x256b [%0], %1;\n\t}"
               ::"r"(taddr), "l"(sdesc), "r"(issue));
}

// Arrive once on an mbarrier when all prior tcgen05.mma of this thread are done.
__device__ __forceinline__ void umma_commit(uint32_t bar, uint32_t issue = 1u) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %1, 0;\n\t"
               "@q tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}"
               ::"r"(bar), "r"(issue) : "memory");
}
// CTA-pair form: arrive on the mbarrier at the same offset in every CTA of mask.
__device__ __forceinline__ void umma_commit_pair(uint32_t bar, uint16_t mask, uint32_t issue = 1u) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t"
      "@q tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;\n\t}"
      ::"r"(bar), "h"(mask), "r"(issue)
      : "memory");
}

// 32 lanes x 32 bits, 32 consecutive columns: thread i of the warp gets TMEM
// lane (quarter*32 + i), columns [col, col+32).
__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 lanes x 32 bits, 32 consecutive columns from registers into TMEM.
__device__ __forceinline__ void tmem_st_32x32b_x32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
      ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
        "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
        "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor (tcgen05 format): start address, leading
// byte offset, stride byte offset (8-row group pitch), fixed version bits
// 46-48 = 0b001, swizzle mode in bits 61-63 (2 = 128B, 4 = 64B, 6 = 32B).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t sbo_bytes, uint32_t swizzle_code) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                                   // LBO (unused for swizzled K-major)
  d |= (uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)swizzle_code << 61;
  return d;
}

// Instruction descriptor: D format F32, A/B formats, both operands K-major,
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ __forceinline__ uint32_t instr_desc(uint32_t ab_fmt, uint32_t M, uint32_t N) {
  return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

}  // namespace pm
