// Mixed-precision path: split-BF16 operator tables (built once at upload) and the
// launchers of the tensor-core right-hand side / RK stage and its BR1 pass.
#include <algorithm>
#include <vector>

#include "dg_mixed.cuh"

namespace dg {
namespace {

// table[term][r][c] = (t(x) | t(y) << 16) for (x, y) = M[r][2c], M[r][2c+1], t the bf16
// term: hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi - mid) (residuals in FP64).
__global__ void split_table_kernel(const double* __restrict__ M, int rows, int cols, uint32_t* __restrict__ out) {
  const int half = cols / 2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows * half; i += gridDim.x * blockDim.x) {
    const int r = i / half, c = i - r * half;
    double x[2] = {M[r * cols + 2 * c], M[r * cols + 2 * c + 1]};
    unsigned short t[3][2];
    for (int j = 0; j < 2; ++j) {
      double rem = x[j];
      for (int term = 0; term < 3; ++term) {
        const __nv_bfloat16 h = __double2bfloat16(rem);
        t[term][j] = __bfloat16_as_ushort(h);
        rem -= (double)__bfloat162float(h);
      }
    }
    for (int term = 0; term < 3; ++term)
      out[(size_t)term * rows * half + i] = (uint32_t)t[term][0] | ((uint32_t)t[term][1] << 16);
  }
}

cudaError_t split_table(const std::vector<double>& host, int rows, int cols, uint32_t** out) {
  double* dM = nullptr;
  const size_t words = (size_t)rows * cols / 2;
  cudaError_t e = cudaMalloc((void**)&dM, sizeof(double) * host.size());
  if (e == cudaSuccess) e = cudaMemcpy(dM, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)out, sizeof(uint32_t) * 3 * words);
  if (e == cudaSuccess) {
    split_table_kernel<<<64, 256>>>(dM, rows, cols, *out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(dM);
  return e;
}

template <int N>
cudaError_t build_t(MeshDev& m, const RefOps& o) {
  using M = mixk::MOrd<N>;
  const int Np = M::Np, NF = M::NF, Nfp = M::Nfp;
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
  std::vector<double> L((size_t)4 * M::NPAD * M::KF, 0.0);
  for (int f = 0; f < 4; ++f)
    for (int i = 0; i < Np; ++i)
      for (int jj = 0; jj < Nfp; ++jj) L[((size_t)f * M::NPAD + i) * M::KF + jj] = o.LIFT[i * NF + f * Nfp + jj];
  cudaError_t e = split_table(R, M::NPAD, M::KR, &m.mx.rhs);
  if (e == cudaSuccess) e = split_table(Dm, M::ND, M::KW, &m.mx.d);
  if (e == cudaSuccess) e = split_table(L, 4 * M::NPAD, M::KF, &m.mx.l);
  return e;
}

template <int N, int PHYS, bool RK>
cudaError_t launch_rhs_mixed_t(const MeshDev& m, const mixk::MixedCase& c, double a, double b, cudaStream_t s) {
  using T = mixk::RT<N, mixk::MOrd<N>::EPB>;
  const size_t smem = T::smem(PHYS == kern::NAVIER_STOKES);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(mixk::rhs_mixed_kernel<N, PHYS, RK>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  static int grid_cap = 0;
  if (!grid_cap) grid_cap = resident_blocks((const void*)mixk::rhs_mixed_kernel<N, PHYS, RK>, T::NT, smem) * device_sms();
  const int tiles = (m.K + T::EPB - 1) / T::EPB;
  mixk::rhs_mixed_kernel<N, PHYS, RK><<<std::min(tiles, grid_cap), T::NT, smem, s>>>(c, m.mx.rhs, m.fmask, a, b);
  return cudaGetLastError();
}

template <int PHYS>
cudaError_t dispatch_mixed(const MeshDev& m, const mixk::MixedCase& c, bool rk, double a, double b,
                           cudaStream_t s) {
  switch (m.N) {
#define DG_CASE(NN)                                                                           \
  case NN:                                                                                    \
    return rk ? launch_rhs_mixed_t<NN, PHYS, true>(m, c, a, b, s) : launch_rhs_mixed_t<NN, PHYS, false>(m, c, a, b, s);
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
cudaError_t launch_viscous_mixed_t(const MeshDev& m, const mixk::MixedCase& c, cudaStream_t s) {
  using T = mixk::VT<N, mixk::MOrd<N>::EPBV>;
  const size_t smem = T::smem();
  static bool configured = false;
  if (!configured) {
    cudaError_t e =
        cudaFuncSetAttribute(mixk::viscous_mixed_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  static int grid_cap = 0;
  if (!grid_cap) grid_cap = resident_blocks((const void*)mixk::viscous_mixed_kernel<N>, T::NT, smem) * device_sms();
  const int tiles = (m.K + T::EPB - 1) / T::EPB;
  mixk::viscous_mixed_kernel<N><<<std::min(tiles, grid_cap), T::NT, smem, s>>>(c, m.mx.d, m.mx.l, m.fmask);
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
  cudaFree(m.mx.rhs);
  cudaFree(m.mx.d);
  cudaFree(m.mx.l);
  cudaFree(m.mx.tc_rhs);
  cudaFree(m.mx.tc_vis);
  m.mx = MixedOps();
}

mixk::MixedCase make_mixed_case(const MeshDev& m, const GasParams& g, const double* qin, double* out, double* k,
                                double dt) {
  const mixk::MixedScratch sc = mixk::mixed_scratch(m.scratch, (size_t)m.K * m.Np);
  mixk::MixedCase c;
  c.q[0] = const_cast<double*>(qin);
  c.q[1] = out;
  c.k = k;
  c.qf = sc.qf;
  c.p = sc.p;
  c.T = sc.T;
  c.fv = sc.fv;
  c.geo = m.geo32;
  c.vmapP = m.vmapP;
  c.K = m.K;
  c.Np = m.Np;
  c.dt = dt;
  c.gas = mixk::MixedGas{g.gamma, g.R, g.mu, g.kappa};
  return c;
}

cudaError_t launch_rhs_mixed(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k, bool rk,
                             double a, double b, double dt, cudaStream_t s) {
  const mixk::MixedCase c = make_mixed_case(m, g, q, out, k, dt);
  if (g.mu > 0) return dispatch_mixed<kern::NAVIER_STOKES>(m, c, rk, a, b, s);
  return dispatch_mixed<kern::EULER>(m, c, rk, a, b, s);
}

cudaError_t launch_prims_mixed(const MeshDev& m, const GasParams& g, const double* q, cudaStream_t s) {
  const size_t KNp = (size_t)m.K * m.Np;
  const mixk::MixedCase c = make_mixed_case(m, g, q, nullptr, nullptr, 0.0);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t want = (KNp + 255) / 256;
  const int blocks = (int)(want < (size_t)sms * 16 ? want : (size_t)sms * 16);
  mixk::prims_kernel<<<blocks, 256, 0, s>>>(c, q, KNp, m.status);
  return cudaGetLastError();
}

cudaError_t launch_viscous_mixed(const MeshDev& m, const GasParams& g, const double* q, cudaStream_t s) {
  const mixk::MixedCase c = make_mixed_case(m, g, q, nullptr, nullptr, 0.0);
  switch (m.N) {
    case 1: return launch_viscous_mixed_t<1>(m, c, s);
    case 2: return launch_viscous_mixed_t<2>(m, c, s);
    case 3: return launch_viscous_mixed_t<3>(m, c, s);
    case 4: return launch_viscous_mixed_t<4>(m, c, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dg
