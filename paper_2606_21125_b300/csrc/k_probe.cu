// FP64 issue-rate probe: the measured FP64 peak that the roofline fractions of the FP64-ALU-bound
// kernels (the LCFO basis step, the subspace solve) are quoted against.  Each thread runs eight
// independent FMA chains, so the FP64 pipe, not the latency of one chain, sets the rate.
#include "dc_internal.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(kProbeThreads) k_fp64_fma(long long iters, double a, double b, double *sink) {
  double x[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += x[k];
  if (s == 12345.678) sink[0] = s;  // keeps the chains live; never true for the inputs used
}

}  // namespace

extern "C" int dc_fp64_fma_probe(int64_t iters, double *d_sink, int64_t *h_fmas, void *stream) {
  if (iters < 1 || !d_sink || !h_fmas) {
    dc_set_error("dc_fp64_fma_probe: iters >= 1, d_sink and h_fmas required");
    return DC_ERR_ARG;
  }
  int dev = 0, sms = 0, per_sm = 0;
  DC_CUDA(cudaGetDevice(&dev));
  DC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_fma, kProbeThreads, 0));
  if (per_sm < 1) per_sm = 1;
  const long long blocks = (long long)sms * per_sm;
  k_fp64_fma<<<(unsigned)blocks, kProbeThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      (long long)iters, 0.999999999, 1e-9, d_sink);
  DC_CUDA(cudaGetLastError());
  *h_fmas = blocks * kProbeThreads * kProbeChains * (int64_t)iters;
  return DC_OK;
}
