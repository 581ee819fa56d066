// Mixed-precision path: split-FP16 operator tables (built once at upload) and the
// launchers of the tensor-core right-hand side / RK stage and its BR1 pass.
#include <vector>

#include "dg_mixed.cuh"

namespace dg {
namespace {

// words[r][c] = (fp16(x) | fp16(y) << 16) for (x, y) = M[r][2c], M[r][2c+1]; lo = residuals.
__global__ void split_table_kernel(const double* __restrict__ M, int rows, int cols, uint32_t* __restrict__ hi,
                                   uint32_t* __restrict__ lo) {
  const int half = cols / 2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows * half; i += gridDim.x * blockDim.x) {
    const int r = i / half, c = i - r * half;
    const double x = M[r * cols + 2 * c], y = M[r * cols + 2 * c + 1];
    const __half hx = __double2half(x), hy = __double2half(y);
    const __half lx = __double2half(x - (double)__half2float(hx)), ly = __double2half(y - (double)__half2float(hy));
    hi[i] = (uint32_t)__half_as_ushort(hx) | ((uint32_t)__half_as_ushort(hy) << 16);
    lo[i] = (uint32_t)__half_as_ushort(lx) | ((uint32_t)__half_as_ushort(ly) << 16);
  }
}

cudaError_t split_table(const std::vector<double>& host, int rows, int cols, uint32_t** hi, uint32_t** lo) {
  double* dM = nullptr;
  const size_t words = (size_t)rows * cols / 2;
  cudaError_t e = cudaMalloc((void**)&dM, sizeof(double) * host.size());
  if (e == cudaSuccess) e = cudaMemcpy(dM, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)hi, sizeof(uint32_t) * words);
  if (e == cudaSuccess) e = cudaMalloc((void**)lo, sizeof(uint32_t) * words);
  if (e == cudaSuccess) {
    split_table_kernel<<<64, 256>>>(dM, rows, cols, *hi, *lo);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(dM);
  return e;
}

template <int N>
cudaError_t build_t(MeshDev& m, const RefOps& o) {
  using M = mixk::MOrd<N>;
  const int Np = M::Np, NF = M::NF;
  const std::vector<double>* D[3] = {&o.Dr, &o.Ds, &o.Dt};
  std::vector<double> R((size_t)M::NPAD * M::KR, 0.0);
  for (int i = 0; i < Np; ++i) {
    for (int a = 0; a < 3; ++a)
      for (int j = 0; j < Np; ++j) R[(size_t)i * M::KR + a * Np + j] = -(*D[a])[i * Np + j];
    for (int k = 0; k < NF; ++k) R[(size_t)i * M::KR + 3 * Np + k] = o.LIFT[i * NF + k];
  }
  std::vector<double> Dm((size_t)M::ND * M::KW, 0.0);
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i < Np; ++i)
      for (int j = 0; j < Np; ++j) Dm[(size_t)(a * Np + i) * M::KW + j] = (*D[a])[i * Np + j];
  std::vector<double> L((size_t)M::NPAD * M::KJ, 0.0);
  for (int i = 0; i < Np; ++i)
    for (int k = 0; k < NF; ++k) L[(size_t)i * M::KJ + k] = o.LIFT[i * NF + k];
  cudaError_t e = split_table(R, M::NPAD, M::KR, &m.mx.rhs_hi, &m.mx.rhs_lo);
  if (e == cudaSuccess) e = split_table(Dm, M::ND, M::KW, &m.mx.d_hi, &m.mx.d_lo);
  if (e == cudaSuccess) e = split_table(L, M::NPAD, M::KJ, &m.mx.l_hi, &m.mx.l_lo);
  return e;
}

template <int N, int PHYS, bool RK>
cudaError_t launch_rhs_mixed_t(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k,
                               double a, double b, double dt, cudaStream_t s) {
  using M = mixk::MOrd<N>;
  constexpr size_t smem = mixk::rhs_mixed_smem<N, PHYS>();
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(mixk::rhs_mixed_kernel<N, PHYS, RK>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int blocks = (m.K + M::EPB - 1) / M::EPB;
  const mixk::MixedScratch sc = mixk::mixed_scratch(m.scratch, (size_t)m.K * M::Np);
  mixk::rhs_mixed_kernel<N, PHYS, RK><<<blocks, M::NT, smem, s>>>(q, out, k, m.mx.rhs_hi, m.mx.rhs_lo, m.fmask,
                                                                    m.geo32, m.vmapP, sc.qf, sc.p, sc.fv, g, m.K,
                                                                    a, b, (float)dt);
  return cudaGetLastError();
}

template <int PHYS>
cudaError_t dispatch_mixed(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k, bool rk,
                           double a, double b, double dt, cudaStream_t s) {
  switch (m.N) {
#define DG_CASE(NN)                                                                     \
  case NN:                                                                              \
    return rk ? launch_rhs_mixed_t<NN, PHYS, true>(m, g, q, out, k, a, b, dt, s)        \
              : launch_rhs_mixed_t<NN, PHYS, false>(m, g, q, out, k, a, b, dt, s);
    DG_CASE(1)
    DG_CASE(2)
    DG_CASE(3)
    DG_CASE(4)
#undef DG_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <int N>
cudaError_t launch_viscous_mixed_t(const MeshDev& m, const GasParams& g, const double* q, cudaStream_t s) {
  using M = mixk::MOrd<N>;
  constexpr size_t smem = mixk::viscous_mixed_smem<N>();
  static bool configured = false;
  if (!configured) {
    cudaError_t e =
        cudaFuncSetAttribute(mixk::viscous_mixed_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int blocks = (m.K + M::EPBV - 1) / M::EPBV;
  const mixk::MixedScratch sc = mixk::mixed_scratch(m.scratch, (size_t)m.K * M::Np);
  mixk::viscous_mixed_kernel<N><<<blocks, M::NTV, smem, s>>>(q, sc.qf, sc.T, sc.fv, m.mx.d_hi, m.mx.d_lo,
                                                             m.mx.l_hi, m.mx.l_lo, m.fmask, m.geo32, m.vmapP, g,
                                                             m.K);
  return cudaGetLastError();
}

}  // namespace

cudaError_t build_mixed_ops(MeshDev& m, const RefOps& ops) {
  switch (m.N) {
    case 1: return build_t<1>(m, ops);
    case 2: return build_t<2>(m, ops);
    case 3: return build_t<3>(m, ops);
    case 4: return build_t<4>(m, ops);
    default: return cudaErrorInvalidValue;
  }
}

void free_mixed_ops(MeshDev& m) {
  cudaFree(m.mx.rhs_hi);
  cudaFree(m.mx.rhs_lo);
  cudaFree(m.mx.d_hi);
  cudaFree(m.mx.d_lo);
  cudaFree(m.mx.l_hi);
  cudaFree(m.mx.l_lo);
  m.mx = MixedOps();
}

cudaError_t launch_rhs_mixed(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k, bool rk,
                             double a, double b, double dt, cudaStream_t s) {
  if (g.mu > 0) return dispatch_mixed<kern::NAVIER_STOKES>(m, g, q, out, k, rk, a, b, dt, s);
  return dispatch_mixed<kern::EULER>(m, g, q, out, k, rk, a, b, dt, s);
}

cudaError_t launch_prims_mixed(const MeshDev& m, const GasParams& g, const double* q, cudaStream_t s) {
  const size_t KNp = (size_t)m.K * m.Np;
  const mixk::MixedScratch sc = mixk::mixed_scratch(m.scratch, KNp);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t want = (KNp + 255) / 256;
  const int blocks = (int)(want < (size_t)sms * 16 ? want : (size_t)sms * 16);
  if (g.mu > 0)
    mixk::prims_kernel<true><<<blocks, 256, 0, s>>>(q, sc.qf, sc.p, sc.T, m.status, g, KNp);
  else
    mixk::prims_kernel<false><<<blocks, 256, 0, s>>>(q, sc.qf, sc.p, sc.T, m.status, g, KNp);
  return cudaGetLastError();
}

cudaError_t launch_viscous_mixed(const MeshDev& m, const GasParams& g, const double* q, cudaStream_t s) {
  switch (m.N) {
    case 1: return launch_viscous_mixed_t<1>(m, g, q, s);
    case 2: return launch_viscous_mixed_t<2>(m, g, q, s);
    case 3: return launch_viscous_mixed_t<3>(m, g, q, s);
    case 4: return launch_viscous_mixed_t<4>(m, g, q, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dg
