// Euler right-hand side / RK stage for a perfect gas (Sec. 5.2), and the
// physics dispatch of dg_rhs / dg_rk_stage.
#include "dg_kernels.cuh"

namespace dg {

cudaError_t launch_rhs_ns(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k,
                          bool rk, double a, double b, double dt, cudaStream_t s, ElemRange r);
cudaError_t launch_rhs_mixture(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k,
                               const double* T, bool rk, double a, double b, double dt, cudaStream_t s);

cudaError_t launch_rhs(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k,
                       const double* T, bool rk, double a, double b, double dt, cudaStream_t s, ElemRange r) {
  if (g.model == DG_GAS_NASA7) return launch_rhs_mixture(m, g, q, out, k, T, rk, a, b, dt, s);
  if (g.mu > 0) return launch_rhs_ns(m, g, q, out, k, rk, a, b, dt, s, r);
  return kern::dispatch_rhs<5, kern::EULER>(m, g, q, out, k, nullptr, rk, a, b, dt, s, r);
}

}  // namespace dg
