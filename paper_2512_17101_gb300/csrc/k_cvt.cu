// Element-wise entry points of the integer-pipe precision conversions (dg_cvt.cuh).
#include "dg_cvt.cuh"
#include "dg_internal.h"

namespace dg {
namespace {

__global__ void round_kernel(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = cvt::narrow(x[i]);
}

__global__ void widen_kernel(const float* __restrict__ x, double* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = cvt::widen(x[i]);
}

__global__ void split_kernel(const double* __restrict__ x, float* __restrict__ hi, float* __restrict__ lo, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 s = cvt::split(x[i]);
    hi[i] = s.x;
    lo[i] = s.y;
  }
}

int grid(int64_t n) {
  const int64_t want = (n + 255) / 256, cap = (int64_t)device_sms() * 16;
  return (int)(want < cap ? want : cap);
}

}  // namespace
}  // namespace dg

extern "C" {

int dg_round_to_float(const double* x, float* y, int64_t n, void* stream) {
  if (n < 0) return dg::fail(DG_ERR_INVALID_ARG, "n must be >= 0");
  if (n == 0) return DG_OK;
  if (!x || !y) return dg::fail(DG_ERR_INVALID_ARG, "NULL array");
  dg::round_kernel<<<dg::grid(n), 256, 0, (cudaStream_t)stream>>>(x, y, n);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DG_OK : dg::cuda_fail(e, "conversion kernel");
}

int dg_widen_to_double(const float* x, double* y, int64_t n, void* stream) {
  if (n < 0) return dg::fail(DG_ERR_INVALID_ARG, "n must be >= 0");
  if (n == 0) return DG_OK;
  if (!x || !y) return dg::fail(DG_ERR_INVALID_ARG, "NULL array");
  dg::widen_kernel<<<dg::grid(n), 256, 0, (cudaStream_t)stream>>>(x, y, n);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DG_OK : dg::cuda_fail(e, "conversion kernel");
}

int dg_split_to_float_pair(const double* x, float* hi, float* lo, int64_t n, void* stream) {
  if (n < 0) return dg::fail(DG_ERR_INVALID_ARG, "n must be >= 0");
  if (n == 0) return DG_OK;
  if (!x || !hi || !lo) return dg::fail(DG_ERR_INVALID_ARG, "NULL array");
  dg::split_kernel<<<dg::grid(n), 256, 0, (cudaStream_t)stream>>>(x, hi, lo, n);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DG_OK : dg::cuda_fail(e, "conversion kernel");
}

}  // extern "C"
