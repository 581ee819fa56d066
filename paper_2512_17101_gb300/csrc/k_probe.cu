// Measured FP64 FMA throughput of the current device: the denominator beside the nominal FP64
// peak for the kernels that the FP64 pipe bounds.  Every thread runs eight independent FMA
// chains (enough to cover the pipe's latency) on values that stay near 1; the result is stored
// only under a condition that the values never meet, so the chains cannot be removed.
#include <algorithm>

#include "dg_internal.h"

namespace dg {
namespace {

constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, double seed, double* __restrict__ sink) {
  double a[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) a[c] = seed + 1e-3 * (threadIdx.x + c);
  const double m = 1.0 + 1e-9, d = 1e-12;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) a[c] = fma(a[c], m, d);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += a[c];
  if (s < 0.0) sink[0] = s;  // never true: the values stay near kProbeChains
}

}  // namespace
}  // namespace dg

extern "C" int dg_fp64_fma_rate(double* tflops_host) {
  using dg::fail;
  if (!tflops_host) return fail(DG_ERR_INVALID_ARG, "NULL output");
  *tflops_host = 0.0;
  const int blocks = dg::device_sms() * 8, threads = 256, iters = 1 << 14;
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc((void**)&sink, sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.0f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch is a warm-up
    e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) {
      dg::fma_probe_kernel<<<blocks, threads>>>(iters, 1.0, sink);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && ms > 0.0f) {
      const float rate = (float)(2.0 * dg::kProbeChains * iters * (double)blocks * threads / (ms * 1e-3) / 1e12);
      best = std::max(best, rate);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return dg::cuda_fail(e, "FP64 FMA probe");
  *tflops_host = best;
  return DG_OK;
}
