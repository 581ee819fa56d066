// Element gather / scatter for the halo exchange of partitioned meshes: the send buffer of a
// neighbour rank is the owned elements it holds as halo, [V][n][Np]; the receive buffer lands on
// the local halo elements.  One thread per (variable, element, node); node-contiguous runs keep
// both sides coalesced.  An element index outside [0, K) is skipped (nothing read or written).
#include "dg_internal.h"

namespace {

__global__ void gather_kernel(const double* __restrict__ src, int V, int64_t K, int Np,
                              const int32_t* __restrict__ elems, int n, double* __restrict__ dst) {
  const int64_t total = (int64_t)V * n * Np;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = t / ((int64_t)n * Np), r = t - v * n * Np, i = r / Np, node = r - i * Np;
    const int64_t e = elems[i];
    if (e >= 0 && e < K) dst[t] = src[(v * K + e) * Np + node];
  }
}

__global__ void scatter_kernel(const double* __restrict__ src, int V, int64_t K, int Np,
                               const int32_t* __restrict__ elems, int n, double* __restrict__ dst) {
  const int64_t total = (int64_t)V * n * Np;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = t / ((int64_t)n * Np), r = t - v * n * Np, i = r / Np, node = r - i * Np;
    const int64_t e = elems[i];
    if (e >= 0 && e < K) dst[(v * K + e) * Np + node] = src[t];
  }
}

int launch(bool gather, const double* src, int32_t V, int64_t K, int32_t Np, const int32_t* elems, int32_t n,
           double* dst, void* stream) {
  if (n == 0) return DG_OK;
  if (n < 0 || V < 1 || Np < 1 || K < 1 || !src || !dst || !elems)
    return dg::fail(DG_ERR_INVALID_ARG, "element gather/scatter: bad sizes or NULL pointers");
  const int64_t total = (int64_t)V * n * Np;
  const int blocks = (int)((total + 255) / 256 < 65535 ? (total + 255) / 256 : 65535);
  if (gather)
    gather_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(src, V, K, Np, elems, n, dst);
  else
    scatter_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(src, V, K, Np, elems, n, dst);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DG_OK : dg::cuda_fail(e, "element gather/scatter");
}

}  // namespace

extern "C" int dg_gather_elements(const double* src, int32_t V, int64_t K, int32_t Np, const int32_t* elems, int32_t n,
                                  double* dst, void* stream) {
  return launch(true, src, V, K, Np, elems, n, dst, stream);
}

extern "C" int dg_scatter_elements(const double* src, int32_t V, int64_t K, int32_t Np, const int32_t* elems,
                                   int32_t n, double* dst, void* stream) {
  return launch(false, src, V, K, Np, elems, n, dst, stream);
}
