// Navier-Stokes with BR1 (Sec. 5.3): the viscous-flux pass and the fused
// right-hand side / RK stage that consumes it.
#include "dg_kernels.cuh"

namespace dg {

cudaError_t launch_rhs_ns(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k,
                          bool rk, double a, double b, double dt, cudaStream_t s) {
  return kern::dispatch_rhs<5, kern::NAVIER_STOKES>(m, g, q, out, k, nullptr, rk, a, b, dt, s);
}

namespace {
template <int N>
cudaError_t launch_viscous_t(const MeshDev& m, const GasParams& g, const double* q, cudaStream_t s) {
  using O = kern::Ord<N>;
  constexpr size_t smem = kern::viscous_smem<N>();
  static bool configured = false;
  if (!configured) {
    cudaError_t e =
        cudaFuncSetAttribute(kern::viscous_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int blocks = (m.K + O::EPB - 1) / O::EPB;
  kern::viscous_kernel<N><<<blocks, O::NT, smem, s>>>(q, m.scratch, m.ops, m.fmask, m.geo, m.vmapP, m.status, g, m.bc,
                                                      m.K);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_viscous_flux(const MeshDev& m, const GasParams& g, const double* q, cudaStream_t s) {
  switch (m.N) {
    case 1: return launch_viscous_t<1>(m, g, q, s);
    case 2: return launch_viscous_t<2>(m, g, q, s);
    case 3: return launch_viscous_t<3>(m, g, q, s);
    case 4: return launch_viscous_t<4>(m, g, q, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dg
