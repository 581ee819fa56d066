// tcgen05 path of the mixed-precision right-hand side: the operator table in the UMMA layout
// (built once at upload) and the launchers.
#include <algorithm>
#include <vector>

#include "dg_tc.cuh"

namespace dg {
namespace {

// out[term] = UMMA K-major image (core matrices 128 B apart in K, sbo between 8-row groups)
// of the term-th BF16 part of M[rows][cols]: hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi - mid).
__global__ void umma_table_kernel(const double* __restrict__ M, int rows, int cols, int sbo, int term_bytes,
                                  unsigned char* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows * cols; i += gridDim.x * blockDim.x) {
    const int r = i / cols, k = i - r * cols;
    const int off = (r >> 3) * sbo + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
    double rem = M[i];
    for (int term = 0; term < 3; ++term) {
      const __nv_bfloat16 h = __double2bfloat16(rem);
      *reinterpret_cast<__nv_bfloat16*>(out + (size_t)term * term_bytes + off) = h;
      rem -= (double)__bfloat162float(h);
    }
  }
}

// Device copy of the three-term UMMA image of a row-major double matrix.
cudaError_t upload_table(const std::vector<double>& host, int rows, int cols, int sbo, int term_bytes,
                         unsigned char** out) {
  double* dM = nullptr;
  cudaError_t e = cudaMalloc((void**)&dM, sizeof(double) * host.size());
  if (e == cudaSuccess) e = cudaMemcpy(dM, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)out, 3 * (size_t)term_bytes);
  if (e == cudaSuccess) e = cudaMemset(*out, 0, 3 * (size_t)term_bytes);
  if (e == cudaSuccess) {
    umma_table_kernel<<<64, 256>>>(dM, rows, cols, sbo, term_bytes, *out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(dM);
  return e;
}

template <int N>
cudaError_t build_t(MeshDev& m, const RefOps& o) {
  using C = tc::Cfg<N>;
  const int Np = C::Np, NF = C::NF, KV = C::KV;
  const std::vector<double>* D[3] = {&o.Dr, &o.Ds, &o.Dt};
  std::vector<double> R((size_t)C::NPAD * C::KB, 0.0);
  for (int i = 0; i < Np; ++i) {
    for (int a = 0; a < 3; ++a)
      for (int j = 0; j < Np; ++j) R[(size_t)i * C::KB + a * KV + j] = -(*D[a])[i * Np + j];
    for (int mm = 0; mm < NF; ++mm) R[(size_t)i * C::KB + 3 * KV + mm] = o.LIFT[i * NF + mm];
  }
  cudaError_t e = upload_table(R, C::NPAD, C::KB, C::B_SBO, C::B_TERM, &m.mx.tc_rhs);
  if (e != cudaSuccess) return e;
  // BR1: rows (a, i) = [D_a[i][:] | 1/2 sum_f c_{f,a} LIFT[i][face f block]], c the reference
  // outward normals of faces t = -1, s = -1, r + s + t = -1, r = -1 (Nanson's relation)
  using V = tc::VCfg<N>;
  constexpr double cfa[4][3] = {{0, 0, -1}, {0, -1, 0}, {1, 1, 1}, {-1, 0, 0}};
  std::vector<double> Rv((size_t)V::NOUT * V::KB, 0.0);
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i < Np; ++i) {
      double* row = &Rv[(size_t)(a * V::NPAD + i) * V::KB];
      for (int j = 0; j < Np; ++j) row[j] = (*D[a])[i * Np + j];
      for (int mm = 0; mm < NF; ++mm) row[V::KV + mm] = 0.5 * cfa[mm / C::Nfp][a] * o.LIFT[i * NF + mm];
    }
  return upload_table(Rv, V::NOUT, V::KB, V::B_SBO, V::B_TERM, &m.mx.tc_vis);
}

template <int N, int PHYS, bool RK>
cudaError_t launch_t(const MeshDev& m, const mixk::MixedCase& c, double a, double b, cudaStream_t s) {
  constexpr int NT = PHYS == kern::MIXTURE ? tc::mixture_nt(N) : tc::default_nt(N);
  using C = tc::Cfg<N, NT, tc::tile_v(PHYS)>;
  auto kern_fn = tc::rhs_tc_kernel<N, NT, PHYS, RK>;
  static int grid_cap = 0;
  if (!grid_cap) {
    cudaError_t e = cudaFuncSetAttribute(kern_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    grid_cap = resident_blocks((const void*)kern_fn, C::NT, C::SMEM, C::TMEM_COLS) * device_sms();
  }
  const int tiles = (m.K + C::E - 1) / C::E;
  kern_fn<<<std::min(tiles, grid_cap), C::NT, C::SMEM, s>>>(c, reinterpret_cast<const uint4*>(m.mx.tc_rhs),
                                                              m.fmask, a, b, m.status);
  return cudaGetLastError();
}

template <int PHYS>
cudaError_t dispatch(const MeshDev& m, const mixk::MixedCase& c, bool rk, double a, double b, cudaStream_t s) {
  switch (m.N) {
#define DG_CASE(NN) \
  case NN:          \
    return rk ? launch_t<NN, PHYS, true>(m, c, a, b, s) : launch_t<NN, PHYS, false>(m, c, a, b, s);
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
cudaError_t launch_vis_t(const MeshDev& m, const mixk::MixedCase& c, cudaStream_t s) {
  using C = tc::VCfg<N>;
  auto kern_fn = tc::vis_tc_kernel<N, C::NT>;
  static int grid_cap = 0;
  if (!grid_cap) {
    cudaError_t e = cudaFuncSetAttribute(kern_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    grid_cap = resident_blocks((const void*)kern_fn, C::NT, C::SMEM, C::TMEM_COLS) * device_sms();
  }
  const int tiles = (m.K + C::E - 1) / C::E;
  kern_fn<<<std::min(tiles, grid_cap), C::NT, C::SMEM, s>>>(c, reinterpret_cast<const uint4*>(m.mx.tc_vis), m.fmask,
                                                              m.status);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_viscous_tc(const MeshDev& m, const GasParams& g, const double* q, cudaStream_t s,
                              int wait_polls) {
  mixk::MixedCase c = make_mixed_case(m, g, q, nullptr, nullptr, 0.0);
  c.wait_polls = wait_polls;
  switch (m.N) {
    case 1: return launch_vis_t<1>(m, c, s);
    case 2: return launch_vis_t<2>(m, c, s);
    case 3: return launch_vis_t<3>(m, c, s);
    case 4: return launch_vis_t<4>(m, c, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t build_tc_ops(MeshDev& m, const RefOps& ops) {
  switch (m.N) {
    case 1: return build_t<1>(m, ops);
    case 2: return build_t<2>(m, ops);
    case 3: return build_t<3>(m, ops);
    case 4: return build_t<4>(m, ops);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_rhs_tc(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k, bool rk,
                          double a, double b, double dt, cudaStream_t s, int wait_polls) {
  mixk::MixedCase c = make_mixed_case(m, g, q, out, k, dt);
  c.wait_polls = wait_polls;
  if (g.model == DG_GAS_NASA7) return dispatch<kern::MIXTURE>(m, c, rk, a, b, s);
  const bool av = m.av.eps0 > 0;  // the AV passes have filled m.av_eps and m.av_sig
  if (g.mu > 0) return av ? dispatch<kern::NS_AV>(m, c, rk, a, b, s) : dispatch<kern::NAVIER_STOKES>(m, c, rk, a, b, s);
  return av ? dispatch<kern::EULER_AV>(m, c, rk, a, b, s) : dispatch<kern::EULER>(m, c, rk, a, b, s);
}

}  // namespace dg
