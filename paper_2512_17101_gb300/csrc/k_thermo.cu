// Temperature of a NASA-7 mixture from internal energy and mass fractions, by
// Newton's method per node (the per-node solve that MIRGE-Com's multi-species
// model needs, Sec. 4 / Sec. 5), and the forward map e(T, Y).
//
// For fixed Y the mixture energy is a quintic in T,
//   e(T) = sum_k Y_k R_k (a1 T + a2 T^2/2 + a3 T^3/3 + a4 T^4/4 + a5 T^5/5 + a6 - T),
// so each node first folds the species sums into six coefficients; every
// Newton update then costs two Horner evaluations and a reciprocal:
//   T <- T - (e(T) - e) / cv(T),  cv = de/dT,  until |dT| < tol (capped)
// (dg_newton.cuh; a block's nodes iterate in rounds, the unconverged ones packed
// onto the first threads after each round).  In the mixed-precision form the same
// kernel also writes the node's pressure, sound speed and float state copy; in the
// FP64 form 1/rho, p and c.
#include <algorithm>

#include "dg_newton.cuh"

namespace dg {
namespace {

constexpr int kNB = 128;  // nodes (threads) per block

// FP2FOLD: the mixed-precision form's float-pair species fold (dg_newton.cuh).
template <bool FP2FOLD>
__global__ void __launch_bounds__(kNB) temperature_kernel(const GasParams g, const int64_t n,
                                                          const double* __restrict__ q, double* __restrict__ T,
                                                          int32_t* __restrict__ iters, const int mode,
                                                          const double t_const, unsigned* __restrict__ status,
                                                          const MixturePrims mp) {
  __shared__ newton::Rounds<kNB> R;
  const int tid = threadIdx.x;
  const int64_t ntiles = (n + kNB - 1) / kNB;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t i = tile * kNB + tid;
    const bool valid = i < n;
    double rho = 1.0, ir = 1.0, rho_e = 0.0, C[6] = {0, 0, 0, 0, 0, 0}, rhoR = 0.0, seed = 0.0;
    if (valid) {
      double rhoY[DG_MAX_SPECIES];
      newton::load_node<FP2FOLD>(g, q, n, i, rho, ir, rho_e, C, rhoR, rhoY);
      seed = mode == DG_TSEED_CONST ? t_const : T[i];
    }
    newton::stage(R, valid, C, rho_e, seed);
    if (newton::rounds(R, g.newton_max_it, g.newton_tol) && tid == 0) atomicOr(status, DG_STATUS_NO_CONVERGENCE);
    if (!valid) continue;
    const double t = R.t[tid];
    T[i] = t;
    if (iters) iters[i] = R.it[tid];
    if (mp.rec || mp.prim) {
      const double rhocv = newton::heat_capacity(C, t);
      if (mp.rec) newton::store_prims(mp, g, q, n, i, rho, ir, rhoR, t, rhocv);
      if (mp.prim) newton::store_prims64(mp, n, i, rho, ir, rhoR, t, rhocv);
    }
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
  // the mixed-precision form (node records out) folds the species in float pairs
  const bool fp2 = mp.rec != nullptr;
  static int per_sm[2] = {0, 0};
  if (!per_sm[fp2])
    per_sm[fp2] = std::max(1, resident_blocks(fp2 ? (const void*)temperature_kernel<true>
                                                  : (const void*)temperature_kernel<false>, kNB, 0));
  const int64_t tiles = (n + kNB - 1) / kNB;
  const int blocks = (int)std::min<int64_t>(tiles, (int64_t)per_sm[fp2] * device_sms());
  if (fp2)
    temperature_kernel<true><<<blocks, kNB, 0, s>>>(g, n, q, T, iters, seed_mode, t_const, status, mp);
  else
    temperature_kernel<false><<<blocks, kNB, 0, s>>>(g, n, q, T, iters, seed_mode, t_const, status, mp);
  return cudaGetLastError();
}

cudaError_t launch_mixture_energy(const GasParams& g, int64_t n, const double* T, const double* Y, double* e,
                                  cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  mixture_energy_kernel<<<grid_for(n, 256), 256, 0, s>>>(g, n, T, Y, e);
  return cudaGetLastError();
}

}  // namespace dg
