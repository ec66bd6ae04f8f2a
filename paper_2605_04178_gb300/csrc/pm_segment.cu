// Generic roofline path of arxiv 2605.04178 (Sec. III-E): workload segments
// outside the stage model, timed as launches + a class-scaled roofline with
// the working-set bandwidth of Eq. 16 + host transfers (Eq. 15) +
// synchronisation points (+ (N_c - 1) tau_c for N_c concurrent copies, Sec.
// III-A.6), times the segment's executions.  One thread per
// segment, FP64 (segment sizes span many decades).
#include <math.h>

#include "pm_internal.cuh"

namespace pm {

struct SegParams {
  double th[PM_NPARAMS];   // stage-model theta (T_launch, B_sus, B_peak, w0, R_TC ...)
  double psi[PM_NPSI];     // class scales, precision efficiencies, host link, sync, stream interference
};

__device__ __forceinline__ double seg_time(const pm_segment& g, const SegParams& p, int n_sm) {
  if (g.cls < PM_SEG_MEMORY || g.cls > PM_SEG_STENCIL || g.precision < PM_FP32 || g.precision > PM_FP8E4M3 ||
      g.kernels < 0 || g.syncs < 0 || g.execs < 1 || g.streams < 0 || !(g.flops >= 0.0) || !(g.bytes >= 0.0) ||
      !(g.working_set >= 0.0) || !(g.h2d_bytes >= 0.0) || !(g.d2h_bytes >= 0.0))
    return __longlong_as_double(0x7ff8000000000000ll);
  double t = 0.0;
  if (g.kernels > 0) {
    // Eq. 16 working-set bandwidth (w0 <= 0 disables the blend)
    const double b_eff = p.th[3] > 0.0 ? p.th[1] + (p.th[2] - p.th[1]) * exp(-g.working_set / p.th[3]) : p.th[1];
    const double rate = (double)n_sm * p.th[6 + g.precision] * p.psi[4 + g.precision];
    const double launches = (double)g.kernels * p.th[0];
    const double roof = p.psi[g.cls] * fmax(g.flops / rate, g.bytes / b_eff);
    t += launches + roof;
    // N_c concurrent copies (Sec. III-A.6): (N_c - 1) tau_c more
    if (g.streams > 1) t += (double)(g.streams - 1) * (p.psi[16] * launches + p.psi[12 + g.cls] * roof);
  }
  if (g.h2d_bytes > 0.0) t += g.h2d_bytes / p.psi[7] + p.psi[8];     // Eq. 15, host to device
  if (g.d2h_bytes > 0.0) t += g.d2h_bytes / p.psi[9] + p.psi[10];    // Eq. 15, device to host
  t += (double)g.syncs * p.psi[11];
  return (double)g.execs * t;
}

__global__ void __launch_bounds__(256) segment_predict_kernel(const pm_segment* __restrict__ segs, int64_t n,
                                                              SegParams p, int n_sm, double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = seg_time(segs[i], p, n_sm);
}

}  // namespace pm

using namespace pm;

extern "C" pm_status pm_segment_predict(const pm_segment* segs_dev, int64_t n, const pm_params* theta_host,
                                        const pm_segment_params* psi_host, int32_t n_sm, double* t_out_dev,
                                        void* stream) {
  PM_REQUIRE(n >= 0, PM_EINVAL, "n < 0");
  if (n == 0) return PM_OK;
  PM_REQUIRE(segs_dev && theta_host && psi_host && t_out_dev && n_sm > 0, PM_EINVAL, "null pointer or n_sm <= 0");
  PM_REQUIRE(((uintptr_t)segs_dev & 7) == 0 && ((uintptr_t)t_out_dev & 7) == 0, PM_EINVAL,
             "segs_dev and t_out_dev must be 8-byte aligned");
  SegParams p;
  for (int j = 0; j < PM_NPARAMS; ++j) p.th[j] = theta_host->v[j];
  for (int j = 0; j < PM_NPSI; ++j) p.psi[j] = psi_host->v[j];
  const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)std::max(1, sm_count()) * 8);
  segment_predict_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(segs_dev, n, p, n_sm, t_out_dev);
  return launch_status("segment_predict_kernel");
}
