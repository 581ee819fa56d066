// dg_rk_stage_noalloc: the viscous RK stage on caller-owned tables and buffers,
// with the BR1 viscous-flux scratch in a file-scope static device array, for
// callers that cannot allocate device memory.  No counterpart in the paper.
#include <cmath>
#include <cstring>
#include <string>

#include "dg_kernels.cuh"

namespace {

// 9 doubles per node: the viscous flux handed from the BR1 pass to the RHS kernel.
static __device__ __align__(256) double g_static_scratch[9 * (size_t)DG_STATIC_SCRATCH_NODES];

// Device address of g_static_scratch in the current context.  Looked up on every call rather
// than cached: cudaGetSymbolAddress is a host-side table lookup once the module is loaded, and a
// cached address would go stale after cudaDeviceReset or a reset of the primary context.  The
// first lookup in a context loads this file's module (lazy module loading) and commits the array.
cudaError_t scratch_address(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

template <int N>
cudaError_t stage_t(const dg::MeshDev& m, const dg::GasParams& g, const double* q, double* out, double* k, double a,
                    double b, double dt, cudaStream_t s) {
  using O = dg::kern::Ord<N>;
  constexpr size_t vs = dg::kern::viscous_smem<N>();
  constexpr size_t rs = dg::kern::rhs_smem<N, 5, dg::kern::NAVIER_STOKES>();
  cudaError_t e = cudaFuncSetAttribute(dg::kern::viscous_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)vs);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(dg::kern::rhs_kernel<N, 5, dg::kern::NAVIER_STOKES, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs);
  if (e != cudaSuccess) return e;
  const int blocks = (m.K + O::EPB - 1) / O::EPB;
  dg::kern::viscous_kernel<N><<<blocks, O::NT, vs, s>>>(q, m.scratch, nullptr, m.ops, m.fmask, m.geo, m.vmapP,
                                                        m.status, g, m.bc, m.K, 0, m.K);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dg::kern::rhs_kernel<N, 5, dg::kern::NAVIER_STOKES, true><<<blocks, O::NT, rs, s>>>(
      q, out, k, nullptr, nullptr, m.ops, m.fmask, m.geo, m.vmapP, m.scratch, nullptr, nullptr, m.status, g, m.bc, m.K,
      5, a, b, dt, 0, m.K);
  return cudaGetLastError();
}

}  // namespace

extern "C" int dg_rk_stage_noalloc(const dg_mesh_tables* t, const dg_gas_desc* gd, int32_t stage, double dt,
                                   const double* q_in, double* q_out, double* k, uint32_t* status, void* stream) {
  using dg::fail;
  if (!t || !gd) return fail(DG_ERR_INVALID_ARG, "NULL tables or gas description");
  if (t->K < 1 || t->N < 1 || t->N > DG_MAX_ORDER) return fail(DG_ERR_INVALID_ARG, "need K >= 1 and N in 1..4");
  const int Np = (t->N + 1) * (t->N + 2) * (t->N + 3) / 6;
  if ((int64_t)t->K * Np > DG_STATIC_SCRATCH_NODES)
    return fail(DG_ERR_INVALID_ARG, "K * Np = " + std::to_string((int64_t)t->K * Np) +
                                        " exceeds the static scratch of DG_STATIC_SCRATCH_NODES = " +
                                        std::to_string(DG_STATIC_SCRATCH_NODES) + " nodes");
  if (!t->ops_dev || !t->fmask_dev || !t->geo_dev || !t->vmapP_dev) return fail(DG_ERR_INVALID_ARG, "NULL table");
  if (!q_in || !q_out || !k || !status) return fail(DG_ERR_INVALID_ARG, "NULL state, output, k or status");
  if (stage < 0 || stage > 4) return fail(DG_ERR_INVALID_ARG, "stage must be in 0..4");
  if (!std::isfinite(dt)) return fail(DG_ERR_INVALID_ARG, "dt must be finite");
  if (gd->model != DG_GAS_PERFECT || !(gd->mu > 0) || !(gd->gamma > 1) || !(gd->R > 0) || !(gd->Pr > 0))
    return fail(DG_ERR_INVALID_ARG, "dg_rk_stage_noalloc needs a viscous perfect gas (gamma > 1, R, mu, Pr > 0)");
  const size_t n = (size_t)5 * t->K * Np;
  if (q_in == q_out || (q_in < q_out + n && q_out < q_in + n))
    return fail(DG_ERR_INVALID_ARG, "output overlaps the input state");
  dg::GasParams g;
  std::memset(&g, 0, sizeof(g));
  g.model = DG_GAS_PERFECT;
  g.gamma = gd->gamma;
  g.R = gd->R;
  g.mu = gd->mu;
  g.Pr = gd->Pr;
  g.cp = gd->gamma * gd->R / (gd->gamma - 1);
  g.kappa = gd->mu * g.cp / gd->Pr;
  dg::MeshDev m;
  m.K = t->K;
  m.N = t->N;
  m.Np = Np;
  m.Nfp = (t->N + 1) * (t->N + 2) / 2;
  m.ops = const_cast<double*>(t->ops_dev);
  m.fmask = const_cast<int32_t*>(t->fmask_dev);
  m.geo = const_cast<double*>(t->geo_dev);
  m.vmapP = const_cast<int32_t*>(t->vmapP_dev);
  m.status = status;
  cudaError_t e = scratch_address(&m.scratch);
  if (e != cudaSuccess) return dg::cuda_fail(e, "static scratch address");
  const double a = dg::kRK4A[stage], b = dg::kRK4B[stage];
  cudaStream_t s = (cudaStream_t)stream;
  switch (t->N) {
    case 1: e = stage_t<1>(m, g, q_in, q_out, k, a, b, dt, s); break;
    case 2: e = stage_t<2>(m, g, q_in, q_out, k, a, b, dt, s); break;
    case 3: e = stage_t<3>(m, g, q_in, q_out, k, a, b, dt, s); break;
    default: e = stage_t<4>(m, g, q_in, q_out, k, a, b, dt, s); break;
  }
  if (e != cudaSuccess) return dg::cuda_fail(e, "allocation-free stage kernels");
  return DG_OK;
}
