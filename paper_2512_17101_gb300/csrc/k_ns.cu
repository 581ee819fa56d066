// Navier-Stokes with BR1 (Sec. 5.3): the viscous-flux pass and the fused
// right-hand side / RK stage that consumes it.
#include "dg_kernels.cuh"

namespace dg {

cudaError_t launch_rhs_ns(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k,
                          bool rk, double a, double b, double dt, cudaStream_t s, ElemRange r) {
  return kern::dispatch_rhs<5, kern::NAVIER_STOKES>(m, g, q, out, k, nullptr, rk, a, b, dt, s, r);
}

namespace {

// Per-node primitives of a perfect gas for the FP64 kernels, once per node:
// prim[0][n] = 1/rho, prim[1][n] = p = (gamma - 1)(rho E - |rho u|^2 / (2 rho)), prim[2][n] = c =
// sqrt(gamma p / rho); a node with rho <= 0 or p <= 0 sets DG_STATUS_NONPHYSICAL.
constexpr int kPrimThreads = 256;
// Nodes [t0, t1) of the n = K Np (the stride between variables).
__global__ void __launch_bounds__(kPrimThreads) prims_fp64_kernel(const double* __restrict__ q,
                                                                  double* __restrict__ prim, const int64_t n,
                                                                  const int64_t t0, const int64_t t1,
                                                                  const double gamma,
                                                                  unsigned* __restrict__ status) {
  bool bad = false;
  for (int64_t t = t0 + blockIdx.x * (int64_t)kPrimThreads + threadIdx.x; t < t1;
       t += (int64_t)gridDim.x * kPrimThreads) {
    const double rho = q[t], mx = q[n + t], my = q[2 * n + t], mz = q[3 * n + t], E = q[4 * n + t];
    const double ir = 1.0 / rho;
    const double p = (gamma - 1.0) * (E - 0.5 * ir * (mx * mx + my * my + mz * mz));
    if (!(rho > 0.0) || !(p > 0.0)) bad = true;
    prim[t] = ir;
    prim[n + t] = p;
    prim[2 * n + t] = sqrt(gamma * p * ir);
  }
  if (bad) atomicOr(status, (unsigned)DG_STATUS_NONPHYSICAL);
}

template <int N>
cudaError_t launch_viscous_t(const MeshDev& m, const GasParams& g, const double* q, cudaStream_t s, ElemRange r) {
  using O = kern::Ord<N>;
  constexpr size_t smem = kern::viscous_smem<N>();
  static bool configured = false;
  if (!configured) {
    cudaError_t e =
        cudaFuncSetAttribute(kern::viscous_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int kb = r.begin, ke = r.end < 0 ? m.K : r.end;
  if (ke <= kb) return cudaSuccess;
  const int blocks = (ke - kb + O::EPB - 1) / O::EPB;
  kern::viscous_kernel<N><<<blocks, O::NT, smem, s>>>(q, m.scratch, m.prim, m.ops, m.fmask, m.geo, m.vmapP, m.status,
                                                      g, m.bc, m.K, kb, ke);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_prims_fp64(const MeshDev& m, const GasParams& g, const double* q, cudaStream_t s, ElemRange r) {
  const int64_t n = (int64_t)m.K * m.Np;
  const int64_t t0 = (int64_t)r.begin * m.Np, t1 = (int64_t)(r.end < 0 ? m.K : r.end) * m.Np;
  if (t1 <= t0) return cudaSuccess;
  const int64_t want = (t1 - t0 + kPrimThreads - 1) / kPrimThreads;
  const int blocks = (int)(want < 65535 ? want : 65535);
  prims_fp64_kernel<<<blocks, kPrimThreads, 0, s>>>(q, m.prim, n, t0, t1, g.gamma, m.status);
  return cudaGetLastError();
}

cudaError_t launch_viscous_flux(const MeshDev& m, const GasParams& g, const double* q, cudaStream_t s,
                                ElemRange r) {
  switch (m.N) {
    case 1: return launch_viscous_t<1>(m, g, q, s, r);
    case 2: return launch_viscous_t<2>(m, g, q, s, r);
    case 3: return launch_viscous_t<3>(m, g, q, s, r);
    case 4: return launch_viscous_t<4>(m, g, q, s, r);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dg
