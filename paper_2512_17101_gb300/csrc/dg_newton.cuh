// Per-node temperature Newton solve of a NASA-7 mixture, shared by the seeded kernel
// (k_thermo.cu) and the MLP-seeded kernel (k_mlp.cu), and the per-node outputs that the
// converged solve yields almost for free.
//
// For fixed mass fractions the internal energy per unit volume is a quintic in T,
//   rho e(T) = sum_j C_j T^j,   C_j = sum_k (rho Y_k) fc[k][j]
// (fc folds R_k, the 1/(j+1) of the enthalpy integral and the -R_k T of e = h - R T; the gas
// precomputes it), so a node folds its species once and every Newton update evaluates the quintic
// and its derivative rho cv(T) by Horner:
//   T <- T - (rho e(T) - rho e) / (rho cv(T))   until |dT| < tol (capped).
// Working per unit volume leaves the iterates unchanged (numerator and denominator both carry rho)
// and saves the seven divisions of rho Y_k by rho.  At the converged T: p = rho R_mix T with
// rho R_mix = sum_k (rho Y_k) R_k, and c^2 = R_mix T (cv + R_mix) / cv.
//
// The block solve runs the updates in rounds: in each round every still-active node takes one
// update, and the nodes that have not converged are packed onto the first threads of the block for
// the next round.  A round costs ceil(active / 32) warp-updates, so the solve costs the mean number
// of updates per node rather than the maximum over each warp's 32 nodes.
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

// FP64 square root of x > 0 from an FP32 reciprocal-square-root seed y0: one Newton step for
// 1/sqrt(x) (y1 = y0 (3 - x y0^2) / 2), then s = x y1 corrected once by s + y1 (x - s^2) / 2
// (relative error ~1e-15); zero and negative inputs give the hardware result.
__device__ __forceinline__ double sqrt64(double x) {
  if (!(x > 0.0)) return sqrt(x);
  const double y0 = cvt::widen(rsqrtf(cvt::narrow(x)));
  const double y1 = y0 * fma(-0.5 * x * y0, y0, 1.5);
  const double s = x * y1;
  return fma(0.5 * y1, fma(-s, s, x), s);
}

// Fold the species of one node: C[0..5] of rho e(T) and rho R_mix, from the partial densities
// rhoY[0..ns).
__device__ __forceinline__ void fold(const GasParams& g, const double* rhoY, double C[6], double& rhoR) {
#pragma unroll
  for (int j = 0; j < 6; ++j) C[j] = 0.0;
  rhoR = 0.0;
#pragma unroll
  for (int k = 0; k < DG_MAX_SPECIES; ++k) {
    if (k >= g.ns) break;
    const double r = rhoY[k];
    rhoR = fma(r, g.Rk[k], rhoR);
#pragma unroll
    for (int j = 0; j < 6; ++j) C[j] = fma(r, g.fc[k][j], C[j]);
  }
}

// Float-pair arithmetic on the FP32 pipe (a value is hi + lo, about 48 significant bits): the
// error-free sum of two floats (Knuth's TwoSum) and the product-accumulate acc += x y, whose
// partial products are formed exactly with FMA and then renormalised (Dekker / Knuth).  The
// _rn intrinsics keep the compiler from contracting a product into a later sum, which would break
// the error-free transformations.
struct FP2 {
  float hi, lo;
};
__device__ __forceinline__ FP2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return FP2{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ void fp2_fma(FP2& acc, float2 x, float2 y) {
  const float p = __fmul_rn(x.x, y.x);
  const float e = fmaf(x.x, y.y, fmaf(x.y, y.x, fmaf(x.x, y.x, -p)));  // the product's rounding + cross terms
  const FP2 s = two_sum(acc.hi, p);
  const float lo = __fadd_rn(s.lo, __fadd_rn(e, acc.lo));
  const float hi = __fadd_rn(s.hi, lo);  // renormalise (|s.hi| >= |lo|)
  acc = FP2{hi, __fsub_rn(lo, __fsub_rn(hi, s.hi))};
}

// The fold of the mixed-precision form: the same sums as fold() in float-pair arithmetic on the
// FP32 pipe (the FP64 pipe, 1/64 of the FP32 rate here, then only adds the two halves), from the
// partial densities split into float pairs.  The coefficients carry ~48 bits (relative error a few
// 1e-15 of the summed magnitudes), which moves the converged temperature by ~1e-11 K, well below
// the Newton tolerance; the Newton iteration itself stays FP64.
__device__ __forceinline__ void fold_fp2(const GasParams& g, const double* rhoY, double C[6], double& rhoR) {
  FP2 a[7];
#pragma unroll
  for (int j = 0; j < 7; ++j) a[j] = FP2{0.0f, 0.0f};
#pragma unroll
  for (int k = 0; k < DG_MAX_SPECIES; ++k) {
    if (k >= g.ns) break;
    const float2 r = cvt::split(rhoY[k]);
#pragma unroll
    for (int j = 0; j < 7; ++j) fp2_fma(a[j], r, g.fc2[k][j]);
  }
#pragma unroll
  for (int j = 0; j < 6; ++j) C[j] = cvt::widen(a[j].hi) + cvt::widen(a[j].lo);
  rhoR = cvt::widen(a[6].hi) + cvt::widen(a[6].lo);
}

// rho cv(T) = d(rho e)/dT.
__device__ __forceinline__ double heat_capacity(const double C[6], double t) {
  return fma(t, fma(t, fma(t, fma(t, 5.0 * C[5], 4.0 * C[4]), 3.0 * C[3]), 2.0 * C[2]), C[1]);
}

// Block-level solve state for NB nodes (slot = thread index).  D holds the derivative
// coefficients 2 C2, 3 C3, 4 C4, 5 C5 so that an update reloads them instead of recomputing.
template <int NB>
struct Rounds {
  double C[6][NB];
  double D[4][NB];
  double e[NB];  // rho e of the node
  double t[NB];  // current iterate
  int it[NB];    // updates taken
  int list[2][NB];
  int count[3];
};

// All 32 lanes of the warp call this: lanes with flag append value to list (length *cnt).
__device__ __forceinline__ void append(int* list, int* cnt, bool flag, int value) {
  const unsigned mask = __ballot_sync(0xffffffffu, flag);
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == 0 && mask) base = atomicAdd(cnt, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (flag) list[base + __popc(mask & ((1u << lane) - 1u))] = value;
}

// Barriers of the block solve: the whole block (__syncthreads), or a named barrier among the
// `count` threads of a group of warps (a warp-specialised kernel whose other warps run other work).
struct BlockSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
template <int ID, int COUNT>  // barrier 1..15, threads (a multiple of 32)
struct GroupSync {
  __device__ __forceinline__ void operator()() const {
    asm volatile("bar.sync %0, %1;\n" ::"n"(ID), "n"(COUNT) : "memory");
  }
};

// Every thread of the group (NB threads, index tid in 0..NB-1) stages its node (valid or not):
// coefficients, rho e and the seed; the valid slots form the first active list.  Begins with a
// barrier so that the previous use of R is over.
template <int NB, class Sync>
__device__ __forceinline__ void stage(Rounds<NB>& R, bool valid, const double C[6], double rho_e, double seed,
                                      int tid, Sync sync) {
  sync();
  if (tid == 0) R.count[0] = R.count[1] = R.count[2] = 0;
#pragma unroll
  for (int j = 0; j < 6; ++j) R.C[j][tid] = C[j];
#pragma unroll
  for (int j = 0; j < 4; ++j) R.D[j][tid] = (double)(j + 2) * C[j + 2];
  R.e[tid] = rho_e;
  R.t[tid] = seed;
  R.it[tid] = 0;
  sync();
  append(R.list[0], &R.count[0], valid, tid);
  sync();
}
template <int NB>
__device__ __forceinline__ void stage(Rounds<NB>& R, bool valid, const double C[6], double rho_e, double seed) {
  stage<NB>(R, valid, C, rho_e, seed, (int)threadIdx.x, BlockSync());
}

// Newton rounds over the staged nodes; returns true when some node had not converged after
// max_it updates (uniform over the group).  On return R.t and R.it hold every slot's result.
template <int NB, class Sync>
__device__ __forceinline__ bool rounds(Rounds<NB>& R, int max_it, double tol, int tid, Sync sync) {
  int m = R.count[0];
  for (int r = 0; m > 0 && r < max_it; ++r) {
    bool again = false;
    int slot = 0;
    if (tid < m) {
      slot = R.list[r & 1][tid];
      const double t = R.t[slot];
      const double eT = fma(t, fma(t, fma(t, fma(t, fma(t, R.C[5][slot], R.C[4][slot]), R.C[3][slot]),
                                             R.C[2][slot]), R.C[1][slot]), R.C[0][slot]);
      const double cv = fma(t, fma(t, fma(t, fma(t, R.D[3][slot], R.D[2][slot]), R.D[1][slot]), R.D[0][slot]),
                            R.C[1][slot]);
      const double dT = (eT - R.e[slot]) * rcp64(cv);
      R.t[slot] = t - dT;
      R.it[slot] = r + 1;
      again = !(fabs(dT) < tol);
    }
    if (tid == 0) R.count[(r + 2) % 3] = 0;  // the list before last: nobody reads its count again
    append(R.list[(r + 1) & 1], &R.count[(r + 1) % 3], again, slot);
    sync();
    m = R.count[(r + 1) % 3];
  }
  return m > 0;
}
template <int NB>
__device__ __forceinline__ bool rounds(Rounds<NB>& R, int max_it, double tol) {
  return rounds<NB>(R, max_it, tol, (int)threadIdx.x, BlockSync());
}

// The mixed-precision form's node record from the converged temperature t: the float state,
// p = rho R_mix t as a float pair, and the sound speed from c^2 = R_mix t (cv + R_mix) / cv formed
// in FP64 and rounded once (rhoR = rho R_mix, rhocv = rho cv: their ratio is R_mix / cv).
__device__ __forceinline__ void store_prims(const MixturePrims& mp, const GasParams& g, const double* __restrict__ q,
                                            int64_t n, int64_t node, double rho, double ir, double rhoR, double t,
                                            double rhocv) {
  const int nvar = 5 + g.ns;
  float v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = 0.0f;
  const float2 rho2 = cvt::split(rho);
  const double p = rhoR * t;
  const float2 p2 = cvt::split(p);
  if (!(rho2.x > 0.0f) || !(p2.x > 0.0f)) atomicOr(mp.status, DG_STATUS_NONPHYSICAL);
  v[0] = rho2.x;
  float lo[4];
#pragma unroll
  for (int j = 1; j < 5; ++j) {
    const float2 s = cvt::split(q[j * n + node]);
    v[j] = s.x;
    lo[j - 1] = s.y;
  }
  mp.lo[node] = make_float4(lo[0], lo[1], lo[2], lo[3]);
  v[5] = p2.x;
  v[6] = p2.y;
  const double c2 = p * ir * fma(rhoR, rcp64(rhocv), 1.0);
  v[7] = sqrtf(cvt::narrow(c2));
  for (int k = 0; k < nvar - 5; ++k) v[8 + k] = cvt::narrow(q[(5 + k) * n + node]);
  float4* r = mp.rec + 4 * node;
  r[0] = make_float4(v[0], v[1], v[2], v[3]);
  r[1] = make_float4(v[4], v[5], v[6], v[7]);
  r[2] = make_float4(v[8], v[9], v[10], v[11]);
  r[3] = make_float4(v[12], v[13], v[14], v[15]);
}

// The FP64 form's primitives at the converged temperature t: 1/rho, p = rho R_mix t and
// c = sqrt(c^2), c^2 = (p / rho) (1 + R_mix / cv).
__device__ __forceinline__ void store_prims64(const MixturePrims& mp, int64_t n, int64_t node, double rho, double ir,
                                              double rhoR, double t, double rhocv) {
  const double p = rhoR * t;
  if (!(rho > 0.0) || !(p > 0.0)) atomicOr(mp.status, DG_STATUS_NONPHYSICAL);
  mp.prim[node] = ir;
  mp.prim[n + node] = p;
  mp.prim[2 * n + node] = sqrt64(p * ir * fma(rhoR, rcp64(rhocv), 1.0));
}

// Loads node i of q [5 + ns][n]: rho, its reciprocal, rho e = rho E - |rho u|^2 / (2 rho) and the
// fold of the partial densities.
template <bool FP2FOLD = false>
__device__ __forceinline__ void load_node(const GasParams& g, const double* __restrict__ q, int64_t n, int64_t i,
                                          double& rho, double& ir, double& rho_e, double C[6], double& rhoR,
                                          double* rhoY) {
  rho = q[i];
  ir = rcp64(rho);
  const double mx = q[n + i], my = q[2 * n + i], mz = q[3 * n + i];
  rho_e = fma(-0.5 * ir, fma(mx, mx, fma(my, my, mz * mz)), q[4 * n + i]);
#pragma unroll
  for (int k = 0; k < DG_MAX_SPECIES; ++k) rhoY[k] = k < g.ns ? q[(5 + k) * n + i] : 0.0;
  if (FP2FOLD)
    fold_fp2(g, rhoY, C, rhoR);
  else
    fold(g, rhoY, C, rhoR);
}

}  // namespace newton
}  // namespace dg
