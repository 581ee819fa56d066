// Euler right-hand side / RK stage for a NASA-7 mixture (multi-species,
// Sec. 4 / Sec. 5): up to DG_MAX_SPECIES passive species, node temperatures
// supplied by the Newton kernel.
#include "dg_kernels.cuh"

namespace dg {

cudaError_t launch_rhs_mixture(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k,
                               const double* T, bool rk, double a, double b, double dt, cudaStream_t s) {
  return kern::dispatch_rhs<5 + DG_MAX_SPECIES, kern::MIXTURE>(m, g, q, out, k, T, rk, a, b, dt, s);
}

}  // namespace dg
