// Runtime glue of libperfmodel.so: error reporting, the per-device watchdog
// word, TMA descriptor encoding, device queries and the watchdog self-test.
#include <cudaTypedefs.h>
#include <dlfcn.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>

#include <chrono>
#include <mutex>

#include "pm_internal.cuh"

namespace pm {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

pm_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s failed: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
  return PM_ECUDA;
}

// The watchdog word: status and site of the first bounded wait that expired.
static __device__ unsigned int g_watchdog_word[4];
static const int kMaxDevices = 64;
static unsigned int* g_wd_ptr[kMaxDevices];
static int g_sm_count[kMaxDevices];
static std::mutex g_mu;

static int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  return dev;
}

unsigned int* watchdog_word() {
  const int dev = current_device();
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_wd_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_watchdog_word) != cudaSuccess) return nullptr;
    g_wd_ptr[dev] = static_cast<unsigned int*>(p);
  }
  return g_wd_ptr[dev];
}

// The allocation-free gradient's scratch address cache (pm_model.cu).
void clear_grad_scratch_cache();

// Forget the per-device addresses of the library's static device arrays and
// the cached SM counts; the next call looks them up again.  A device reset
// reloads the module, after which a cached address would be stale.
void clear_device_address_caches() {
  std::lock_guard<std::mutex> lk(g_mu);
  for (int d = 0; d < kMaxDevices; ++d) {
    g_wd_ptr[d] = nullptr;
    g_sm_count[d] = 0;
  }
}

unsigned long long watchdog_limit_ns() {
  static unsigned long long v = [] {
    const char* s = getenv("PM_WATCHDOG_MS");
    long ms = s ? strtol(s, nullptr, 10) : 2000;
    if (ms <= 0) ms = 2000;
    return (unsigned long long)ms * 1000000ull;
  }();
  return v;
}

int sm_count() {
  const int dev = current_device();
  if (dev < 0 || dev >= kMaxDevices) return 0;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_sm_count[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    g_sm_count[dev] = n;
  }
  return g_sm_count[dev];
}

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

pm_status make_tmap_2d(CUtensorMap* map, const void* base, int dtype_code, uint64_t rows, uint64_t cols,
                       uint32_t box_rows, uint32_t box_cols, int swizzle_bytes) {
  auto enc = get_encode();
  PM_REQUIRE(enc != nullptr, PM_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  CUtensorMapDataType dt;
  uint64_t esize;
  switch (dtype_code) {
    case TMAP_F32: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; esize = 4; break;
    case TMAP_BF16: dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; esize = 2; break;
    default: dt = CU_TENSOR_MAP_DATA_TYPE_UINT8; esize = 1; break;
  }
  CUtensorMapSwizzle sw;
  switch (swizzle_bytes) {
    case 128: sw = CU_TENSOR_MAP_SWIZZLE_128B; break;
    case 64: sw = CU_TENSOR_MAP_SWIZZLE_64B; break;
    case 32: sw = CU_TENSOR_MAP_SWIZZLE_32B; break;
    default: sw = CU_TENSOR_MAP_SWIZZLE_NONE; break;
  }
  PM_REQUIRE(((uintptr_t)base & 15) == 0, PM_EINVAL, "TMA base address %p is not 16-byte aligned", base);
  PM_REQUIRE((cols * esize) % 16 == 0, PM_EINVAL, "row pitch %llu bytes is not a multiple of 16",
             (unsigned long long)(cols * esize));
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * esize};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  PM_REQUIRE(r == CUDA_SUCCESS, PM_EINVAL,
             "cuTensorMapEncodeTiled failed (%d): rows=%llu cols=%llu box=%ux%u swizzle=%d", (int)r,
             (unsigned long long)rows, (unsigned long long)cols, box_rows, box_cols, swizzle_bytes);
  return PM_OK;
}

// Clock and throttle state through NVML, read only.  The driver's NVML
// library is opened at run time (no link dependency: the library also loads
// on machines without a driver); the device is matched by PCI bus id, so
// the CUDA and NVML device orders need not agree.
namespace {
struct Nvml {
  bool ok = false;
  int (*init)() = nullptr;
  int (*by_pci)(const char*, void**) = nullptr;
  int (*clock)(void*, int, unsigned int*) = nullptr;
  int (*max_clock)(void*, int, unsigned int*) = nullptr;
  int (*reasons)(void*, unsigned long long*) = nullptr;
  int (*power)(void*, unsigned int*) = nullptr;
  void* dev[kMaxDevices] = {};
};
Nvml g_nvml;
std::once_flag g_nvml_once;
std::mutex g_nvml_mu;

void nvml_open() {
  void* h = dlopen("libnvidia-ml.so.1", RTLD_NOW | RTLD_LOCAL);
  if (!h) return;
  auto sym = [&](const char* name) { return dlsym(h, name); };
  g_nvml.init = reinterpret_cast<int (*)()>(sym("nvmlInit_v2"));
  g_nvml.by_pci = reinterpret_cast<int (*)(const char*, void**)>(sym("nvmlDeviceGetHandleByPciBusId_v2"));
  g_nvml.clock = reinterpret_cast<int (*)(void*, int, unsigned int*)>(sym("nvmlDeviceGetClockInfo"));
  g_nvml.max_clock = reinterpret_cast<int (*)(void*, int, unsigned int*)>(sym("nvmlDeviceGetMaxClockInfo"));
  void* r = sym("nvmlDeviceGetCurrentClocksEventReasons");
  if (!r) r = sym("nvmlDeviceGetCurrentClocksThrottleReasons");
  g_nvml.reasons = reinterpret_cast<int (*)(void*, unsigned long long*)>(r);
  g_nvml.power = reinterpret_cast<int (*)(void*, unsigned int*)>(sym("nvmlDeviceGetPowerUsage"));
  g_nvml.ok = g_nvml.init && g_nvml.by_pci && g_nvml.clock && g_nvml.max_clock && g_nvml.reasons &&
              g_nvml.power && g_nvml.init() == 0;
}

void* nvml_device() {
  std::call_once(g_nvml_once, nvml_open);
  if (!g_nvml.ok) return nullptr;
  const int d = current_device();
  if (d < 0 || d >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_nvml_mu);
  if (!g_nvml.dev[d]) {
    char bus[32] = {0};
    if (cudaDeviceGetPCIBusId(bus, sizeof(bus), d) != cudaSuccess) return nullptr;
    void* h = nullptr;
    if (g_nvml.by_pci(bus, &h) != 0) return nullptr;
    g_nvml.dev[d] = h;
  }
  return g_nvml.dev[d];
}
}  // namespace

bool read_clock(pm_clock* c) {
  *c = pm_clock{};
  c->host_time_s = std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
  void* d = nvml_device();
  if (!d) return false;
  unsigned int v = 0;
  unsigned long long r = 0;
  bool ok = g_nvml.clock(d, 1 /* SM */, &v) == 0;
  c->sm_mhz = v;
  ok = ok && g_nvml.max_clock(d, 1, &v) == 0;
  c->sm_max_mhz = v;
  if (g_nvml.clock(d, 2 /* memory */, &v) == 0) c->mem_mhz = v;
  if (g_nvml.power(d, &v) == 0) c->power_mw = v;
  ok = ok && g_nvml.reasons(d, &r) == 0;
  c->reasons = r;
  return ok;
}

void clock_record(pm_probe_result* out, const pm_clock& begin, const pm_clock& end) {
  out->sm_mhz_begin = begin.sm_mhz;
  out->sm_mhz_end = end.sm_mhz;
  out->sm_max_mhz = end.sm_max_mhz ? end.sm_max_mhz : begin.sm_max_mhz;
  out->clock_reasons = begin.reasons | end.reasons;
}

// Waits on an mbarrier that nothing ever completes; the bounded wait gives up
// after the limit and records PM_ETIMEOUT.
__global__ void watchdog_selftest_kernel(Watchdog wd) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = smem_u32(&bar);
  if (threadIdx.x == 0) {
    mbar_init(b, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(b, 0, wd, nullptr, SITE_SELFTEST);
}

}  // namespace pm

using namespace pm;

extern "C" const char* pm_last_error(void) { return pm::g_err; }

extern "C" int32_t pm_version(void) { return 10000; }

extern "C" pm_status pm_device_status(int clear) {
  unsigned int* w = watchdog_word();
  PM_REQUIRE(w != nullptr, PM_ECUDA, "no CUDA device");
  PM_CUDA(cudaDeviceSynchronize());
  unsigned int h[4];
  PM_CUDA(cudaMemcpy(h, w, sizeof(h), cudaMemcpyDeviceToHost));
  if (clear) PM_CUDA(cudaMemset(w, 0, sizeof(h)));
  if (h[0] != 0) {
    set_error("device watchdog expired at site %u", h[1]);
    return (pm_status)(-(int)h[0]);
  }
  return PM_OK;
}

extern "C" pm_status pm_watchdog_selftest(int32_t limit_us, void* stream) {
  PM_REQUIRE(limit_us > 0 && limit_us <= 10000000, PM_EINVAL, "limit_us must be in (0, 1e7]");
  unsigned int* w = watchdog_word();
  PM_REQUIRE(w != nullptr, PM_ECUDA, "no CUDA device");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PM_CUDA(cudaMemsetAsync(w, 0, 4 * sizeof(unsigned int), s));
  Watchdog wd{w, (unsigned long long)limit_us * 1000ull};
  watchdog_selftest_kernel<<<1, 32, 0, s>>>(wd);
  pm_status st = launch_status("watchdog_selftest_kernel");
  if (st != PM_OK) return st;
  PM_CUDA(cudaStreamSynchronize(s));
  unsigned int h[4];
  PM_CUDA(cudaMemcpy(h, w, sizeof(h), cudaMemcpyDeviceToHost));
  PM_CUDA(cudaMemset(w, 0, sizeof(h)));
  if (h[0] != 0) {
    set_error("device watchdog expired at site %u", h[1]);
    return (pm_status)(-(int)h[0]);
  }
  return PM_OK;
}

extern "C" pm_status pm_clock_sample(pm_clock* out) {
  PM_REQUIRE(out != nullptr, PM_EINVAL, "out is NULL");
  PM_REQUIRE(pm::read_clock(out), PM_EUNSUPPORTED, "NVML clock query unavailable for the current device");
  return PM_OK;
}

extern "C" pm_status pm_shutdown(void) {
  pm::release_stream_pool();
  pm::release_host_pipe_this_thread();
  pm::clear_tmap_caches_this_thread();
  pm::clear_device_address_caches();
  pm::clear_grad_scratch_cache();
  return PM_OK;
}
