// Temperature of a NASA-7 mixture from internal energy and mass fractions, by
// Newton's method per node (the per-node solve that MIRGE-Com's multi-species
// model needs, Sec. 4 / Sec. 5), and the forward map e(T, Y).
//
// For fixed Y the mixture energy is a quintic in T,
//   e(T) = sum_k Y_k R_k (a1 T + a2 T^2/2 + a3 T^3/3 + a4 T^4/4 + a5 T^5/5 + a6 - T),
// so each node first folds the species sums into six coefficients; every
// Newton update then costs two Horner evaluations and a division:
//   T <- T - (e(T) - e) / cv(T),  cv = de/dT,  until |dT| < tol (capped).
#include "dg_internal.h"

namespace dg {
namespace {

__global__ void temperature_kernel(const GasParams g, const int64_t n, const double* __restrict__ q,
                                   double* __restrict__ T, int32_t* __restrict__ iters, const int mode,
                                   const double t_const, unsigned* __restrict__ status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double rho = q[i], ir = 1.0 / rho;
    const double mx = q[n + i], my = q[2 * n + i], mz = q[3 * n + i];
    const double e = q[4 * n + i] * ir - 0.5 * ir * ir * (mx * mx + my * my + mz * mz);
    double c[6] = {0, 0, 0, 0, 0, 0};
    for (int k = 0; k < g.ns; ++k) {
      const double yr = q[(5 + k) * n + i] * ir * g.Rk[k];
      const double* a = g.a[k];
      c[0] = fma(yr, a[5], c[0]);
      c[1] = fma(yr, a[0] - 1.0, c[1]);
      c[2] = fma(yr, a[1] * 0.5, c[2]);
      c[3] = fma(yr, a[2] * (1.0 / 3.0), c[3]);
      c[4] = fma(yr, a[3] * 0.25, c[4]);
      c[5] = fma(yr, a[4] * 0.2, c[5]);
    }
    double t = mode == DG_TSEED_CONST ? t_const : T[i];
    int it = 0;
    bool done = false;
    while (it < g.newton_max_it) {
      const double eT = c[0] + t * (c[1] + t * (c[2] + t * (c[3] + t * (c[4] + t * c[5]))));
      const double cv = c[1] + t * (2.0 * c[2] + t * (3.0 * c[3] + t * (4.0 * c[4] + t * 5.0 * c[5])));
      const double dT = (eT - e) / cv;
      t -= dT;
      ++it;
      if (fabs(dT) < g.newton_tol) {
        done = true;
        break;
      }
    }
    if (!done) atomicOr(status, DG_STATUS_NO_CONVERGENCE);
    T[i] = t;
    if (iters) iters[i] = it;
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
                               int seed_mode, double t_const, unsigned* status, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  temperature_kernel<<<grid_for(n, 256), 256, 0, s>>>(g, n, q, T, iters, seed_mode, t_const, status);
  return cudaGetLastError();
}

cudaError_t launch_mixture_energy(const GasParams& g, int64_t n, const double* T, const double* Y, double* e,
                                  cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  mixture_energy_kernel<<<grid_for(n, 256), 256, 0, s>>>(g, n, T, Y, e);
  return cudaGetLastError();
}

}  // namespace dg
