// The two global reductions of a run: integrals of the conserved variables (conservation
// diagnostics) and the largest stability rate (the time step is CFL / rate).  A partitioned run
// reduces each rank's value over its owned elements, which come first in its local mesh, and
// combines the ranks' values itself (sum, max).
//   integral of q_v = sum_e J_e sum_i w_i q_v(e, i),  w_i = integral of the i-th nodal basis
//     function over the reference element;
//   rate = max_e max_i [ (N+1)^2/2 F_e (|u| + c) + (N+1)^4/4 F_e^2 nu ],  F_e = max_f Fscale_{e,f},
//     nu = (mu / rho) max(4/3, gamma / Pr) (0 without viscosity): the nodal-DG step estimate of
//     Hesthaven and Warburton with 1/h read as F_e / 2.
// Both run a fixed grid and combine the block partials in a fixed order, so a result does not
// depend on the device or on timing (bitwise reproducible).
#include <cmath>

#include "dg_internal.h"

namespace {

using dg::kDiagBlocks;
using dg::kDiagMaxV;
using dg::kDiagThreads;
constexpr int GS = DG_GEO_STRIDE, GEO_J = 25, GEO_FSCALE = 12;

template <bool MAX>
__device__ __forceinline__ double combine(double a, double b) {
  return MAX ? fmax(a, b) : a + b;
}

// Tree over the block's threads in shared memory; thread 0 returns the result.
template <bool MAX>
__device__ double block_reduce(double v, double* red) {
  const int tid = threadIdx.x;
  red[tid] = v;
  __syncthreads();
#pragma unroll
  for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
    if (tid < w) red[tid] = combine<MAX>(red[tid], red[tid + w]);
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kDiagThreads) integrals_partial(const double* __restrict__ q, int nvar, int64_t KNp,
                                                                  int64_t nodes, int Np,
                                                                  const double* __restrict__ geo,
                                                                  const double* __restrict__ wq,
                                                                  double* __restrict__ part) {
  __shared__ double red[kDiagThreads];
  double acc[kDiagMaxV];
#pragma unroll
  for (int v = 0; v < kDiagMaxV; ++v) acc[v] = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)kDiagThreads + threadIdx.x; t < nodes; t += (int64_t)kDiagBlocks * kDiagThreads) {
    const int64_t e = t / Np;
    const double wJ = geo[e * GS + GEO_J] * wq[t - e * Np];
#pragma unroll
    for (int v = 0; v < kDiagMaxV; ++v)
      if (v < nvar) acc[v] = fma(wJ, q[v * KNp + t], acc[v]);
  }
#pragma unroll
  for (int v = 0; v < kDiagMaxV; ++v) {  // unrolled: acc stays in registers (nvar is block-uniform)
    if (v >= nvar) break;
    const double r = block_reduce<false>(acc[v], red);
    if (threadIdx.x == 0) part[blockIdx.x * kDiagMaxV + v] = r;
  }
}

__global__ void __launch_bounds__(kDiagThreads) rate_partial(const double* __restrict__ q, int64_t KNp, int64_t nodes,
                                                             int Np, const double* __restrict__ geo, double A, double B,
                                                             double gamma, double mu, double visc_coef,
                                                             unsigned* __restrict__ status, double* __restrict__ part) {
  __shared__ double red[kDiagThreads];
  double best = 0.0;
  bool bad = false;
  for (int64_t t = blockIdx.x * (int64_t)kDiagThreads + threadIdx.x; t < nodes; t += (int64_t)kDiagBlocks * kDiagThreads) {
    const int64_t e = t / Np;
    const double* G = geo + e * GS + GEO_FSCALE;
    const double F = fmax(fmax(G[0], G[4]), fmax(G[8], G[12]));
    const double rho = q[t], mx = q[KNp + t], my = q[2 * KNp + t], mz = q[3 * KNp + t], E = q[4 * KNp + t];
    const double ux = mx / rho, uy = my / rho, uz = mz / rho;
    const double u2 = ux * ux + uy * uy + uz * uz;
    const double p = (gamma - 1.0) * (E - 0.5 * rho * u2);
    double r;
    if (rho > 0.0 && p > 0.0) {
      const double speed = sqrt(u2) + sqrt(gamma * p / rho);
      const double nu = mu > 0.0 ? (mu / rho) * visc_coef : 0.0;
      r = A * F * speed + B * F * F * nu;
    } else {
      r = INFINITY;
      bad = true;
    }
    best = fmax(best, r);
  }
  if (bad) atomicOr(status, (unsigned)DG_STATUS_NONPHYSICAL);
  const double r = block_reduce<true>(best, red);
  if (threadIdx.x == 0) part[blockIdx.x * kDiagMaxV] = r;
}

// out[v] <- the kDiagBlocks partials of variable v combined (block of kDiagThreads threads).
template <bool MAX>
__global__ void __launch_bounds__(kDiagThreads) finish(const double* __restrict__ part, int nvar,
                                                       double* __restrict__ out) {
  __shared__ double red[kDiagThreads];
  for (int v = 0; v < nvar; ++v) {
    double a = 0.0;  // the identity of both: sums start at 0, rates are >= 0
    for (int b = threadIdx.x; b < kDiagBlocks; b += kDiagThreads) a = combine<MAX>(a, part[b * kDiagMaxV + v]);
    const double r = block_reduce<MAX>(a, red);
    if (threadIdx.x == 0) out[v] = r;
  }
}

int check_common(dg_mesh mesh, const void* q, int64_t K_count, const void* out) {
  if (!mesh || !q || !out) return dg::fail(DG_ERR_INVALID_ARG, "NULL mesh, state or output");
  if (!mesh->d.ops) return dg::fail(DG_ERR_INVALID_ARG, "the mesh was built with DG_MESH_HOST_ONLY");
  if (K_count < 0 || K_count > mesh->d.K) return dg::fail(DG_ERR_INVALID_ARG, "K_count must be in [0, K]");
  return DG_OK;
}

}  // namespace

extern "C" int dg_integrals(dg_mesh mesh, const double* q, int32_t nvar, int64_t K_count, double* out, void* stream) {
  if (int r = check_common(mesh, q, K_count, out)) return r;
  if (nvar < 1 || nvar > kDiagMaxV) return dg::fail(DG_ERR_INVALID_ARG, "nvar must be in 1..5+DG_MAX_SPECIES");
  const dg::MeshDev& m = mesh->d;
  cudaStream_t s = (cudaStream_t)stream;
  integrals_partial<<<kDiagBlocks, kDiagThreads, 0, s>>>(q, nvar, (int64_t)m.K * m.Np, K_count * m.Np, m.Np, m.geo,
                                                         m.wq, m.diag);
  finish<false><<<1, kDiagThreads, 0, s>>>(m.diag, nvar, out);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DG_OK : dg::cuda_fail(e, "integrals kernels");
}

extern "C" int dg_max_rate(dg_mesh mesh, dg_gas gas, const double* q, int64_t K_count, double* out, void* stream) {
  if (int r = check_common(mesh, q, K_count, out)) return r;
  if (!gas) return dg::fail(DG_ERR_INVALID_ARG, "NULL gas");
  if (gas->p.model != DG_GAS_PERFECT) return dg::fail(DG_ERR_UNSUPPORTED, "the stability rate needs a perfect gas");
  const dg::MeshDev& m = mesh->d;
  const dg::GasParams& g = gas->p;
  const double n1 = m.N + 1.0;
  const double A = n1 * n1 / 2.0, B = n1 * n1 * n1 * n1 / 4.0;
  const double vc = g.mu > 0 ? fmax(4.0 / 3.0, g.gamma / g.Pr) : 0.0;
  cudaStream_t s = (cudaStream_t)stream;
  rate_partial<<<kDiagBlocks, kDiagThreads, 0, s>>>(q, (int64_t)m.K * m.Np, K_count * m.Np, m.Np, m.geo, A, B, g.gamma,
                                                    g.mu, vc, m.status, m.diag);
  finish<true><<<1, kDiagThreads, 0, s>>>(m.diag, 1, out);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DG_OK : dg::cuda_fail(e, "stability-rate kernels");
}
