// Temperature of a NASA-7 mixture from internal energy and mass fractions, by
// Newton's method per node (the per-node solve that MIRGE-Com's multi-species
// model needs, Sec. 4 / Sec. 5), and the forward map e(T, Y).
//
// For fixed Y the mixture energy is a quintic in T,
//   e(T) = sum_k Y_k R_k (a1 T + a2 T^2/2 + a3 T^3/3 + a4 T^4/4 + a5 T^5/5 + a6 - T),
// so each node first folds the species sums into six coefficients; every
// Newton update then costs two Horner evaluations and a reciprocal:
//   T <- T - (e(T) - e) / cv(T),  cv = de/dT,  until |dT| < tol (capped)
// (dg_newton.cuh).  In the mixed-precision form the same kernel also writes the
// node's pressure, sound speed and float state copy; in the FP64 form 1/rho, p and c.
#include "dg_newton.cuh"

namespace dg {
namespace {

__global__ void temperature_kernel(const GasParams g, const int64_t n, const double* __restrict__ q,
                                   double* __restrict__ T, int32_t* __restrict__ iters, const int mode,
                                   const double t_const, unsigned* __restrict__ status, const MixturePrims mp) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double rho = q[i], ir = newton::rcp64(rho);
    const double mx = q[n + i], my = q[2 * n + i], mz = q[3 * n + i];
    const double e = q[4 * n + i] * ir - 0.5 * ir * ir * (mx * mx + my * my + mz * mz);
    double Y[DG_MAX_SPECIES];
#pragma unroll
    for (int k = 0; k < DG_MAX_SPECIES; ++k) Y[k] = k < g.ns ? q[(5 + k) * n + i] * ir : 0.0;
    double c[6], Rmix, cv;
    newton::fold(g, Y, c, Rmix);
    double t = mode == DG_TSEED_CONST ? t_const : T[i];
    int it;
    if (!newton::solve(c, e, t, g.newton_max_it, g.newton_tol, it, cv)) atomicOr(status, DG_STATUS_NO_CONVERGENCE);
    T[i] = t;
    if (iters) iters[i] = it;
    if (mp.rec) newton::store_prims(mp, g, q, n, i, rho, Rmix, t, cv);
    if (mp.prim) newton::store_prims64(mp, c, n, i, rho, Rmix, t);
  }
}

__global__ void mixture_energy_kernel(const GasParams g, const int64_t n, const double* __restrict__ T,
                                      const double* __restrict__ Y, double* __restrict__ e) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double t = T[i];
    double acc = 0.0;
    for (int k = 0; k < g.ns; ++k) {
      const double* a = g.a[k];
      const double hk = t * (a[0] + t * (a[1] * 0.5 + t * (a[2] * (1.0 / 3.0) + t * (a[3] * 0.25 + t * a[4] * 0.2)))) +
                        a[5];
      acc = fma(Y[k * n + i] * g.Rk[k], hk - t, acc);
    }
    e[i] = acc;
  }
}

int grid_for(int64_t n, int threads) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t want = (n + threads - 1) / threads;
  int64_t cap = (int64_t)sms * 16;
  return (int)(want < cap ? want : cap);
}

}  // namespace

cudaError_t launch_temperature(const GasParams& g, int64_t n, const double* q, double* T, int32_t* iters,
                               int seed_mode, double t_const, unsigned* status, cudaStream_t s,
                               const MixturePrims& mp) {
  if (n <= 0) return cudaSuccess;
  temperature_kernel<<<grid_for(n, 256), 256, 0, s>>>(g, n, q, T, iters, seed_mode, t_const, status, mp);
  return cudaGetLastError();
}

cudaError_t launch_mixture_energy(const GasParams& g, int64_t n, const double* T, const double* Y, double* e,
                                  cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  mixture_energy_kernel<<<grid_for(n, 256), 256, 0, s>>>(g, n, T, Y, e);
  return cudaGetLastError();
}

}  // namespace dg
