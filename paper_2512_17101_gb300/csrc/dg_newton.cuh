// Per-node temperature Newton solve of a NASA-7 mixture, shared by the seeded kernel
// (k_thermo.cu) and the MLP-seeded kernel (k_mlp.cu), and the mixed-precision form's
// per-node outputs that the converged solve yields almost for free.
//
// For fixed Y the mixture internal energy is a quintic in T whose coefficients c[0..5]
// fold the species sums (sum_k Y_k R_k a_kj / (j+1), the -R_mix T of e = h - R T included);
// each Newton update evaluates e(T) and cv(T) = de/dT by Horner and takes
// T <- T - (e(T) - e) / cv(T) until |dT| < tol (capped).
// At the converged T: cp = cv + R_mix, p = rho R_mix T, c^2 = cp/cv p/rho = R_mix T (cv + R_mix)/cv.
#pragma once

#include "dg_cvt.cuh"
#include "dg_internal.h"

namespace dg {
namespace newton {

// FP64 reciprocal from an FP32 seed and one Newton step (relative error ~1e-14); the seed's
// conversions run on the integer pipe.
__device__ __forceinline__ double rcp64(double x) {
  const double r = cvt::widen(1.0f / cvt::narrow(x));
  return r * fma(-x, r, 2.0);
}

// Fold the species polynomials into the quintic e(T) = c0 + c1 T + ... + c5 T^5 (J/kg).
__device__ __forceinline__ void fold(const GasParams& g, const double* Y, double c[6], double& Rmix) {
#pragma unroll
  for (int j = 0; j < 6; ++j) c[j] = 0.0;
  Rmix = 0.0;
#pragma unroll
  for (int k = 0; k < DG_MAX_SPECIES; ++k) {
    if (k >= g.ns) break;
    const double yr = Y[k] * g.Rk[k];
    const double* a = g.a[k];
    Rmix += yr;
    c[0] = fma(yr, a[5], c[0]);
    c[1] = fma(yr, a[0] - 1.0, c[1]);
    c[2] = fma(yr, a[1] * 0.5, c[2]);
    c[3] = fma(yr, a[2] * (1.0 / 3.0), c[3]);
    c[4] = fma(yr, a[3] * 0.25, c[4]);
    c[5] = fma(yr, a[4] * 0.2, c[5]);
  }
}

// Newton from seed t; returns true when |dT| < tol was met within max_it updates.  On return
// t is the solution, it the updates taken and cv the heat capacity at the last iterate.
__device__ __forceinline__ bool solve(const double c[6], double e, double& t, int max_it, double tol, int& it,
                                      double& cv) {
  it = 0;
  cv = 1.0;
  while (it < max_it) {
    const double eT = c[0] + t * (c[1] + t * (c[2] + t * (c[3] + t * (c[4] + t * c[5]))));
    cv = c[1] + t * (2.0 * c[2] + t * (3.0 * c[3] + t * (4.0 * c[4] + t * 5.0 * c[5])));
    const double dT = (eT - e) * rcp64(cv);
    t -= dT;
    ++it;
    if (fabs(dT) < tol) return true;
  }
  return false;
}

// The mixed-precision form's node record from the converged temperature t (cv at the last
// iterate): the float state, p = rho R_mix t as a float pair, and the sound speed from c^2 formed
// in FP64 and rounded once.
__device__ __forceinline__ void store_prims(const MixturePrims& mp, const GasParams& g, const double* __restrict__ q,
                                            int64_t n, int64_t node, double rho, double Rmix, double t, double cv) {
  const int nvar = 5 + g.ns;
  float v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = 0.0f;
  const float2 rho2 = cvt::split(rho);
  const double p = rho * Rmix * t;
  const float2 p2 = cvt::split(p);
  if (!(rho2.x > 0.0f) || !(p2.x > 0.0f)) atomicOr(mp.status, DG_STATUS_NONPHYSICAL);
  v[0] = rho2.x;
  for (int j = 1; j < 4; ++j) v[j] = cvt::narrow(q[j * n + node]);
  v[4] = cvt::narrow(q[4 * n + node]);
  v[5] = p2.x;
  v[6] = p2.y;
  const double c2 = Rmix * t * fma(Rmix, rcp64(cv), 1.0);
  v[7] = sqrtf(cvt::narrow(c2));
  for (int k = 0; k < nvar - 5; ++k) v[8 + k] = cvt::narrow(q[(5 + k) * n + node]);
  float4* r = mp.rec + 4 * node;
  r[0] = make_float4(v[0], v[1], v[2], v[3]);
  r[1] = make_float4(v[4], v[5], v[6], v[7]);
  r[2] = make_float4(v[8], v[9], v[10], v[11]);
  r[3] = make_float4(v[12], v[13], v[14], v[15]);
}

// The FP64 form's primitives at the converged temperature t: 1/rho, p = rho R_mix t and
// c = sqrt(cp/cv p/rho), with cv = de/dT of the folded quintic at t and cp = cv + R_mix.
__device__ __forceinline__ void store_prims64(const MixturePrims& mp, const double c[6], int64_t n, int64_t node,
                                              double rho, double Rmix, double t) {
  const double cv = c[1] + t * (2.0 * c[2] + t * (3.0 * c[3] + t * (4.0 * c[4] + t * 5.0 * c[5])));
  const double ir = 1.0 / rho;
  const double p = rho * Rmix * t;
  if (!(rho > 0.0) || !(p > 0.0)) atomicOr(mp.status, DG_STATUS_NONPHYSICAL);
  mp.prim[node] = ir;
  mp.prim[n + node] = p;
  mp.prim[2 * n + node] = sqrt((cv + Rmix) / cv * p * ir);
}

}  // namespace newton
}  // namespace dg
