// Shock capturing by artificial viscosity on the FP64 tetrahedral path (the paper names
// artificial viscosity among the stabilisations of its shock cases, Sec. 5.3; the method here is
// the sub-cell shock capturing of Persson and Peraire, 2006):
//   * smoothness indicator of the density per element, S = (energy of its orthonormal modes of
//     total degree N) / (its total energy), s = log10 S;
//   * eps = 0 (s < s0 - kappa), eps0 (s > s0 + kappa), eps0/2 (1 + sin(pi (s - s0) / (2 kappa)));
//   * flux sigma_v = eps grad q_v for every conserved variable, BR1 gradient with the central
//     flux (exterior values from the ghost states at boundary faces), added to the right-hand
//     side through the central flux (rhs_kernel<EULER_AV / NS_AV>).
#include <algorithm>
#include <cmath>

#include "dg_kernels.cuh"

namespace dg {
namespace kern {

// One thread per (element, mode): the mode's coefficient from the element's nodal densities;
// then one thread per element sums the energies.
// list (may be null): [0] a count the caller has zeroed, then the elements with eps > 0 in any order.
// R: the arithmetic type, double for the FP64 form, float for the mixed-precision form (whose
// right-hand side takes the AV flux as one of its FP32 terms); eps is stored as a double.
template <int N, typename R>
__global__ void __launch_bounds__(Ord<N>::NT) av_sensor_kernel(const double* __restrict__ q,
                                                               const double* __restrict__ modal_g, const int ntop,
                                                               const AvParams av, const int K,
                                                               double* __restrict__ eps, int* __restrict__ list) {
  using O = Ord<N>;
  constexpr int Np = O::Np, EPB = O::EPB, NODES = O::NODES;
  __shared__ R sH[Np * Np];
  __shared__ R sU[NODES];
  __shared__ R sC[NODES];
  const int tid = threadIdx.x;
  const int e0 = blockIdx.x * EPB;
  const int nel = min(EPB, K - e0);
  const int nn = nel * Np;
  const size_t base = (size_t)e0 * Np;
  for (int i = tid; i < Np * Np; i += blockDim.x) sH[i] = (R)modal_g[i];
  if (tid < nn) sU[tid] = (R)q[base + tid];  // density, variable 0
  __syncthreads();
  if (tid < nn) {
    const int e = tid / Np, m = tid - e * Np;
    R c = 0;
#pragma unroll 5
    for (int j = 0; j < Np; ++j) c = fma(sH[m * Np + j], sU[e * Np + j], c);
    sC[tid] = c * c;
  }
  __syncthreads();
  if (tid < nel) {
    R den = 0, num = 0;
    for (int m = 0; m < Np; ++m) {
      const R c2 = sC[tid * Np + m];
      den += c2;
      if (m >= Np - ntop) num += c2;
    }
    double e = 0.0;
    if (num > 0 && den > 0) {
      const R sv = log10(num / den);
      if (sv > (R)(av.s0 + av.kappa))
        e = av.eps0;
      else if (sv >= (R)(av.s0 - av.kappa))
        e = 0.5 * av.eps0 *
            (1.0 + (double)sin((R)3.141592653589793 * (sv - (R)av.s0) / ((R)2 * (R)av.kappa)));
    }
    eps[e0 + tid] = e;
    if (list && e > 0.0) list[1 + atomicAdd(list, 1)] = e0 + tid;
  }
}

// BR1 gradient of the five conserved variables, times the element viscosity:
//   grad_d q = sum_a (dr_a/dx_d) D_a q + sum_f n_d,f LIFT_f (Fscale (q+ - q-)/2),
//   sig[(5 d + v)][K][Np] = eps_e grad_d q_v,
// for the elements of the sensor's list only (sigma = 0 wherever eps = 0, and the right-hand sides
// read sigma only where eps > 0).  Persistent: each block takes groups of EPB listed elements.
// Shared memory of av_flux_kernel<N, R>: the geometry in FP64, the operators, state and face jumps
// in R, the face-node map and the group's element indices.
template <int N, typename R>
constexpr size_t av_flux_smem() {
  using O = Ord<N>;
  return sizeof(double) * O::EPB * GS + sizeof(R) * (O::OPS + 5 * O::NODES + 5 * O::EPB * O::NF + O::EPB * GS) +
         sizeof(int) * (O::NF + O::EPB);
}

template <int N, typename R>
__global__ void __launch_bounds__(Ord<N>::NT) av_flux_kernel(
    const double* __restrict__ q, const double* __restrict__ eps, double* __restrict__ sig,
    const double* __restrict__ ops_g, const int32_t* __restrict__ fmask_g, const double* __restrict__ geo_g,
    const int32_t* __restrict__ vmapP, const BcParams bc, const int K, const int* __restrict__ list) {
  using O = Ord<N>;
  constexpr int Np = O::Np, Nfp = O::Nfp, NF = O::NF, EPB = O::EPB, NODES = O::NODES;
  constexpr int W = 5;
  extern __shared__ double smem[];
  double* sGeo = smem;
  R* sOps = reinterpret_cast<R*>(sGeo + EPB * GS);
  R* sW = sOps + O::OPS;
  R* sJ = sW + W * NODES;
  R* sGr = sJ + W * EPB * NF;  // the geometry converted once per element, for the node loop
  int* sFm = reinterpret_cast<int*>(sGr + EPB * GS);
  int* sE = sFm + NF;  // [EPB]: the group's element indices

  const int tid = threadIdx.x;
  const size_t KNp = (size_t)K * Np;
  const int count = list[0];
  for (int i = tid; i < O::OPS; i += blockDim.x) sOps[i] = (R)ops_g[i];
  for (int i = tid; i < NF; i += blockDim.x) sFm[i] = fmask_g[i];
  for (int g0 = blockIdx.x * EPB; g0 < count; g0 += gridDim.x * EPB) {
  const int nel = min(EPB, count - g0);
  const int nn = nel * Np;
  __syncthreads();  // the previous group's reads of sE, sGeo, sW and sJ are done
  if (tid < nel) sE[tid] = list[1 + g0 + tid];
  __syncthreads();
  for (int i = tid; i < nel * GS; i += blockDim.x) {
    const double gv = geo_g[(size_t)sE[i / GS] * GS + i % GS];
    sGeo[i] = gv;
    sGr[i] = (R)gv;
  }
#pragma unroll
  for (int v = 0; v < W; ++v)
    for (int i = tid; i < nn; i += blockDim.x) sW[v * NODES + i] = (R)q[v * KNp + (size_t)sE[i / Np] * Np + i % Np];
  __syncthreads();

  for (int j = tid; j < nel * NF; j += blockDim.x) {
    const int e = j / NF, m = j - e * NF, f = m / Nfp;
    const double* G = sGeo + e * GS;
    const double hf = 0.5 * G[12 + 4 * f];
    const int P = vmapP[(size_t)sE[e] * NF + m];  // < 0: boundary face node, -DG_BC_* code
    const size_t Pn = P >= 0 ? (size_t)P : (size_t)sE[e] * Np + sFm[m];  // a boundary node gathers its own trace
    double qm[W], qp[W];  // the traces and the ghost state in FP64, the jump stored in R
#pragma unroll
    for (int v = 0; v < W; ++v) {
      qm[v] = q[v * KNp + (size_t)sE[e] * Np + sFm[m]];
      qp[v] = q[v * KNp + Pn];
    }
    if (P < 0) ghost_state<W>(-P, qm, G[9 + 4 * f], G[10 + 4 * f], G[11 + 4 * f], bc, W, qp);
#pragma unroll
    for (int v = 0; v < W; ++v) sJ[v * EPB * NF + j] = (R)(hf * (qp[v] - qm[v]));
  }
  __syncthreads();

  if (tid < nn) {
    const int e = tid / Np, i = tid - e * Np;
    const R* G = sGr + e * GS;
    const R* Dr = sOps + i * Np;
    const R* Ds = sOps + Np * Np + i * Np;
    const R* Dt = sOps + 2 * Np * Np + i * Np;
    const R* L = sOps + 3 * Np * Np + i * NF;
    R dref[3][W];
#pragma unroll
    for (int v = 0; v < W; ++v) dref[0][v] = dref[1][v] = dref[2][v] = 0;
#pragma unroll 4
    for (int jn = 0; jn < Np; ++jn) {
      const R dr = Dr[jn], ds = Ds[jn], dtt = Dt[jn];
#pragma unroll
      for (int v = 0; v < W; ++v) {
        const R w = sW[v * NODES + e * Np + jn];
        dref[0][v] = fma(dr, w, dref[0][v]);
        dref[1][v] = fma(ds, w, dref[1][v]);
        dref[2][v] = fma(dtt, w, dref[2][v]);
      }
    }
    R grad[3][W];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int v = 0; v < W; ++v)
        grad[d][v] = fma(G[d], dref[0][v], fma(G[3 + d], dref[1][v], G[6 + d] * dref[2][v]));
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      R lf[W];
#pragma unroll
      for (int v = 0; v < W; ++v) lf[v] = 0;
#pragma unroll 5
      for (int jj = 0; jj < Nfp; ++jj) {
        const R l = L[f * Nfp + jj];
        const int col = e * NF + f * Nfp + jj;
#pragma unroll
        for (int v = 0; v < W; ++v) lf[v] = fma(l, sJ[v * EPB * NF + col], lf[v]);
      }
      const R nf[3] = {G[9 + 4 * f], G[10 + 4 * f], G[11 + 4 * f]};
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < W; ++v) grad[d][v] = fma(nf[d], lf[v], grad[d][v]);
    }
    const R ee = (R)eps[sE[e]];
    const size_t gi = (size_t)sE[e] * Np + i;
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int v = 0; v < W; ++v) sig[(5 * d + v) * KNp + gi] = (double)(ee * grad[d][v]);
  }
  }
}

template <int N, typename R>
cudaError_t launch_sensor_t(const MeshDev& m, const double* q, double* eps, int* list, cudaStream_t s) {
  using O = Ord<N>;
  const int blocks = (m.K + O::EPB - 1) / O::EPB;
  if (list) {
    cudaError_t e = cudaMemsetAsync(list, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
  }
  av_sensor_kernel<N, R><<<blocks, O::NT, 0, s>>>(q, m.modal, m.ntop, m.av, m.K, eps, list);
  return cudaGetLastError();
}

template <int N, typename R>
cudaError_t launch_flux_t(const MeshDev& m, const double* q, cudaStream_t s) {
  using O = Ord<N>;
  constexpr size_t smem = av_flux_smem<N, R>();
  static int grid_cap = 0;
  if (!grid_cap) {  // a persistent grid: the blocks that fit on the device at once
    cudaError_t e = cudaFuncSetAttribute(av_flux_kernel<N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, av_flux_kernel<N, R>, O::NT, smem);
    if (e != cudaSuccess) return e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid_cap = std::max(1, per_sm) * sms;
  }
  const int blocks = std::min((m.K + O::EPB - 1) / O::EPB, grid_cap);
  av_flux_kernel<N, R><<<blocks, O::NT, smem, s>>>(q, m.av_eps, m.av_sig, m.ops, m.fmask, m.geo, m.vmapP, m.bc, m.K,
                                                    m.av_list);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_sensor_r(const MeshDev& m, const double* q, double* eps, cudaStream_t s, int* list) {
  switch (m.N) {
    case 1: return launch_sensor_t<1, R>(m, q, eps, list, s);
    case 2: return launch_sensor_t<2, R>(m, q, eps, list, s);
    case 3: return launch_sensor_t<3, R>(m, q, eps, list, s);
    case 4: return launch_sensor_t<4, R>(m, q, eps, list, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R>
cudaError_t launch_flux_r(const MeshDev& m, const double* q, cudaStream_t s) {
  switch (m.N) {
    case 1: return launch_flux_t<1, R>(m, q, s);
    case 2: return launch_flux_t<2, R>(m, q, s);
    case 3: return launch_flux_t<3, R>(m, q, s);
    case 4: return launch_flux_t<4, R>(m, q, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace kern

cudaError_t launch_av_sensor(const MeshDev& m, const double* q, double* eps, cudaStream_t s, int* list, bool fp32) {
  return fp32 ? kern::launch_sensor_r<float>(m, q, eps, s, list) : kern::launch_sensor_r<double>(m, q, eps, s, list);
}

cudaError_t launch_av_flux(const MeshDev& m, const GasParams&, const double* q, cudaStream_t s, bool fp32) {
  return fp32 ? kern::launch_flux_r<float>(m, q, s) : kern::launch_flux_r<double>(m, q, s);
}

cudaError_t launch_rhs_av(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k, bool rk,
                          double a, double b, double dt, cudaStream_t s) {
  if (g.mu > 0) return kern::dispatch_rhs<5, kern::NS_AV>(m, g, q, out, k, nullptr, rk, a, b, dt, s);
  return kern::dispatch_rhs<5, kern::EULER_AV>(m, g, q, out, k, nullptr, rk, a, b, dt, s);
}

}  // namespace dg
