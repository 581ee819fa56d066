// Mixed-precision form of the DG right-hand side: shared pieces of its kernels.
//
// The D and LIFT contractions run on the tensor cores as split-BF16 products (x = hi + mid
// + lo, each bf16, so 24 significant bits in FP32's exponent range; the six products with
// term orders adding up to at most 2, FP32 accumulation; dg_tc.cuh), the pointwise fluxes
// run in FP32, and the pressure, the differences that would cancel (pressure minus an
// element reference, p- - p+, rho and T relative to a reference and their jumps) and the RK
// accumulation stay in FP64.
//
// Why the differences: D annihilates constants, so the large, nearly constant part of a flux
// (the pressure in the momentum flux) carries no information but would dominate the
// rounding error of an FP32 operand.  Subtracting an element reference value in FP64 before
// rounding keeps the operands small.
//
// This header holds the per-node primitives pass, the case descriptor the kernels share, and
// the FP32 pointwise flux arithmetic.
#pragma once

#include <cuda_bf16.h>

#include "dg_cvt.cuh"
#include "dg_kernels.cuh"

namespace dg {
namespace mixk {

using kern::GS;

// FP64 reciprocal from an FP32 seed plus one Newton step (relative error ~1e-14); the seed's
// conversions run on the integer pipe.
__device__ __forceinline__ double recip64(double x, float& r32) {
  r32 = 1.0f / cvt::narrow(x);
  const double r = cvt::widen(r32);
  return r * fma(-x, r, 2.0);
}

// Per-node tables of the mixed form for a perfect gas, in the mesh's scratch (76 of its 80 bytes
// per node), as records so that a node's values come in a few wide loads:
//   node [KNp][2] float4: {rho_hi, rho u, rho v, rho w}, {rho E, p_hi, p_lo, rho_lo}
//   fv4  [KNp][2] float4: {tau_xx, tau_yy, tau_zz, tau_xy}, {tau_xz, tau_yz, Q_x, Q_y};  fvz [KNp]: Q_z
//   temp [KNp] float2: {T_hi, T_lo}
// rho, p and T are float pairs hi + lo (hi = the FP64 value rounded to FP32, lo = the rounded rest:
// about 48 significant bits), so the differences that would cancel (p against the element's first
// node, p- - p+, rho and T against a reference and their jumps) are formed as (hi - hi') + (lo - lo')
// in FP32, whose hi part is exact for values within a factor of two of each other.
struct NodeTables {
  float4* node;
  float4* fv4;
  float* fvz;
  float2* temp;
};

__host__ __device__ inline NodeTables node_tables(double* base, size_t KNp) {
  float* f = reinterpret_cast<float*>(base);
  NodeTables t;
  t.node = reinterpret_cast<float4*>(f);
  t.fv4 = reinterpret_cast<float4*>(f + 8 * KNp);
  t.temp = reinterpret_cast<float2*>(f + 16 * KNp);
  t.fvz = f + 18 * KNp;
  return t;
}

// x = hi + lo with hi = x rounded to FP32 and lo the rest rounded to FP32 (integer pipe, dg_cvt.cuh).
__device__ __forceinline__ float2 split2(double x) { return cvt::split(x); }

// One case of the mixed form: its state buffers (q[0] in, q[1] out for a single
// stage; the two alternate over the stages of a batched step), RK register,
// per-node tables, geometry, neighbour map, size, time step and gas.
struct MixedGas {
  double gamma, R, mu, kappa, inv_R;
};

struct MixedCase {
  double* q[2];
  double* k;
  // perfect gas: node records (see NodeTables)
  float4* node;
  float4* fv4;
  float* fvz;
  float2* temp;
  // mixture: node records and the low halves of momentum and energy (see mixture_records)
  float4* mrec;
  float4* mlo;
  const float* geo;
  const int32_t* vmapP;
  int K;
  int Np;
  int nvar;   // conserved variables: 5, or 5 + species for a mixture
  double dt;
  MixedGas gas;
  // DG_BC_INFLOW state as a node record and a temperature pair (perfect gas), or as a mixture
  // record and its low halves (p and c at the inflow temperature)
  float4 in_node[2];
  float2 in_temp;
  float4 in_mrec[4];
  float4 in_mlo;
  // artificial viscosity (perfect gas, FP64 passes): element viscosities [K] and the flux
  // sigma = eps grad_h q, [(5 d + v)][K][Np], stored only in elements with eps > 0
  const double* av_eps;
  const double* av_sig;
  int wait_polls;  // polls per bounded mbarrier wait of the tensor-core kernels; 0 = the default
};

// Exterior record of a boundary face node (code = -vmapP; r0, r1 hold the node's own record on
// entry): the ghost states of the FP64 path in record form: slip wall (momentum mirrored), no-slip
// wall (momentum reversed), inflow (the prescribed state), outflow (the node's own).
__device__ __forceinline__ void ghost_record(int code, const float n[3], const MixedCase& c, float4& r0, float4& r1) {
  if (code == DG_BC_SLIP_WALL) {
    const float mn2 = 2.0f * (r0.y * n[0] + r0.z * n[1] + r0.w * n[2]);
    r0.y -= mn2 * n[0];
    r0.z -= mn2 * n[1];
    r0.w -= mn2 * n[2];
  } else if (code == DG_BC_NOSLIP_WALL) {
    r0.y = -r0.y;
    r0.z = -r0.z;
    r0.w = -r0.w;
  } else if (code == DG_BC_INFLOW) {
    r0 = c.in_node[0];
    r1 = c.in_node[1];
  }
}

// The same ghost states for a mixture node: q[13] its float state, a = {rho E, p_hi, p_lo, c} and
// lo = the low halves of momentum and energy (the node's own on entry).  A wall ghost keeps rho,
// |m|, rho E and rho Y, hence the node's temperature, p and c: only the momentum (both halves)
// changes.  An inflow ghost is the inflow record.
__device__ __forceinline__ void ghost_mix_record(int code, const float n[3], const MixedCase& c, float* q, float4& a,
                                                 float4& lo) {
  if (code == DG_BC_SLIP_WALL) {
    const float mn2 = 2.0f * (q[1] * n[0] + q[2] * n[1] + q[3] * n[2]);
    const float ln2 = 2.0f * (lo.x * n[0] + lo.y * n[1] + lo.z * n[2]);
    q[1] -= mn2 * n[0];
    q[2] -= mn2 * n[1];
    q[3] -= mn2 * n[2];
    lo.x -= ln2 * n[0];
    lo.y -= ln2 * n[1];
    lo.z -= ln2 * n[2];
  } else if (code == DG_BC_NOSLIP_WALL) {
    q[1] = -q[1];
    q[2] = -q[2];
    q[3] = -q[3];
    lo.x = -lo.x;
    lo.y = -lo.y;
    lo.z = -lo.z;
  } else if (code == DG_BC_INFLOW) {
    const float4 r0 = c.in_mrec[0], r2 = c.in_mrec[2], r3 = c.in_mrec[3];
    a = c.in_mrec[1];
    lo = c.in_mlo;
    q[0] = r0.x; q[1] = r0.y; q[2] = r0.z; q[3] = r0.w; q[4] = a.x;
    q[5] = r2.x; q[6] = r2.y; q[7] = r2.z; q[8] = r2.w;
    q[9] = r3.x; q[10] = r3.y; q[11] = r3.z; q[12] = r3.w;
  }
}

// Exterior viscous flux {tau_xx, tau_yy, tau_zz, tau_xy, tau_xz, tau_yz, Q_x, Q_y, Q_z} of a
// boundary face node (fv holds the node's own on entry): walls are adiabatic (Q+ = -Q-); a slip
// wall is shear-free, tau+ = -tau- + 2 (n.tau- n) n n^T, so that tau+ n = 2 (n.tau- n) n - tau- n.
__device__ __forceinline__ void ghost_viscous(int code, const float n[3], float fv[9]) {
  if (code != DG_BC_SLIP_WALL && code != DG_BC_NOSLIP_WALL) return;
  fv[6] = -fv[6];
  fv[7] = -fv[7];
  fv[8] = -fv[8];
  if (code == DG_BC_SLIP_WALL) {
    float tn[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      tn[i] = 0.0f;
#pragma unroll
      for (int d = 0; d < 3; ++d) tn[i] = fmaf(n[d], fv[kern::tau_index(i, d)], tn[i]);
    }
    const float tnn2 = 2.0f * (tn[0] * n[0] + tn[1] * n[1] + tn[2] * n[2]);
    fv[0] = fmaf(tnn2, n[0] * n[0], -fv[0]);
    fv[1] = fmaf(tnn2, n[1] * n[1], -fv[1]);
    fv[2] = fmaf(tnn2, n[2] * n[2], -fv[2]);
    fv[3] = fmaf(tnn2, n[0] * n[1], -fv[3]);
    fv[4] = fmaf(tnn2, n[0] * n[2], -fv[4]);
    fv[5] = fmaf(tnn2, n[1] * n[2], -fv[5]);
  }
}

// Per-node record of the mixed form for a mixture (64 of the scratch's 80 bytes per node), written
// by the temperature Newton kernels at the converged temperature (dg_newton.cuh):
//   [KNp][4] float4: {rho_hi, rho u, rho v, rho w}, {rho E, p_hi, p_lo, c},
//                    {rho Y_1 .. rho Y_4}, {rho Y_5 .. rho Y_8}   (absent species 0)
// and, in the remaining 16 bytes, the low halves of the float pairs of momentum and energy:
//   [KNp] float4: {(rho u)_lo, (rho v)_lo, (rho w)_lo, (rho E)_lo}
// read only where a difference would cancel: the Lax-Friedrichs jumps q- - q+, multiplied by the
// wave speed (a sound speed of ~1e3 m/s against velocities of ~10 m/s here), whose FP32 rounding
// would otherwise dominate the momentum error.
constexpr int MIX_V = 5 + DG_MAX_SPECIES;
static_assert(MIX_V <= 13, "the mixture record holds up to 8 species");
__host__ __device__ inline float4* mixture_records(double* base) { return reinterpret_cast<float4*>(base); }
__host__ __device__ inline float4* mixture_lo(double* base, size_t KNp) {
  return reinterpret_cast<float4*>(base) + 4 * KNp;
}

// ---- pass 0: per node, FP64 pressure (and temperature) and the node record, so that the later
// kernels read traces without recomputing or converting them.
__device__ __forceinline__ void prims_node(const MixedCase& c, const double* __restrict__ qin, size_t KNp, size_t i,
                                           unsigned* status) {
  double qv[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) qv[v] = qin[v * KNp + i];
  float ir32;
  const double ir = recip64(qv[0], ir32);
  const double p = (c.gas.gamma - 1.0) * (qv[4] - 0.5 * ir * fma(qv[1], qv[1], fma(qv[2], qv[2], qv[3] * qv[3])));
  const float2 rho2 = split2(qv[0]), p2 = split2(p);
  if (!(rho2.x > 0.0f) || !(p2.x > 0.0f)) atomicOr(status, DG_STATUS_NONPHYSICAL);
  c.node[2 * i] = make_float4(rho2.x, cvt::narrow(qv[1]), cvt::narrow(qv[2]), cvt::narrow(qv[3]));
  c.node[2 * i + 1] = make_float4(cvt::narrow(qv[4]), p2.x, p2.y, rho2.y);
  if (c.gas.mu > 0.0) c.temp[i] = split2(p * ir * c.gas.inv_R);  // T = p / (rho R), no FP64 division
}

static __global__ void prims_kernel(const MixedCase c, const double* __restrict__ qin, const size_t KNp,
                             unsigned* __restrict__ status) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < KNp; i += (size_t)gridDim.x * blockDim.x)
    prims_node(c, qin, KNp, i, status);
}

constexpr int PRIMS_CHUNK = 1024;  // nodes per work item of the batched pass

// work item (case, first node of a PRIMS_CHUNK run); the stage's parity picks the input buffer
static __global__ void prims_batched(const MixedCase* __restrict__ cases, const int2* __restrict__ work, const int nwork,
                              const int stage, unsigned* __restrict__ status) {
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int2 it = work[w];
    const MixedCase& c = cases[it.x];
    const size_t KNp = (size_t)c.K * c.Np;
    const double* qin = c.q[stage & 1];
    for (int j = threadIdx.x; j < PRIMS_CHUNK; j += blockDim.x) {
      const size_t i = (size_t)it.y + j;
      if (i < KNp) prims_node(c, qin, KNp, i, status);
    }
  }
}

// ---- pointwise FP32 fluxes ---------------------------------------------------------------------
// Volume flux of one node, F[d][v] = (rho u_d, rho u u_d + dp e_d, u_d (rho E + p)) minus the
// viscous flux (NS); dp is the pressure relative to the element's first node (an FP64 difference
// rounded to FP32), pf the pressure itself.  Viscous flux layout: tau_xx, tau_yy, tau_zz, tau_xy,
// tau_xz, tau_yz, then (u . tau - q_heat)_d.
template <bool NS>
__device__ __forceinline__ void node_flux(const float q[5], float dp, float pf, const float fv[9], float F[3][5]) {
  const float ir = 1.0f / q[0];
  const float u[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    F[d][0] = q[1 + d];
    F[d][1] = q[1] * u[d];
    F[d][2] = q[2] * u[d];
    F[d][3] = q[3] * u[d];
    F[d][1 + d] += dp;
    F[d][4] = u[d] * (q[4] + pf);
    if (NS) {
#pragma unroll
      for (int ii = 0; ii < 3; ++ii) F[d][1 + ii] -= fv[kern::tau_index(ii, d)];
      F[d][4] -= fv[6 + d];
    }
  }
}

// Surface term of one face node before the Fscale factor: g = n.F(q-) - F*, with the local
// Lax-Friedrichs flux F* (pointwise lambda) and, for NS, the central viscous flux; dpn = p- - p+
// as an FP64 difference rounded to FP32.
template <bool NS>
__device__ __forceinline__ void face_term(const float qm[5], const float qp[5], float pm, float pp, float dpn,
                                          const float fvm[9], const float fvp[9], const float n[3], float gam,
                                          float g[5]) {
  const float irm = 1.0f / qm[0], irp = 1.0f / qp[0];
  const float unm = (qm[1] * n[0] + qm[2] * n[1] + qm[3] * n[2]) * irm;
  const float unp = (qp[1] * n[0] + qp[2] * n[1] + qp[3] * n[2]) * irp;
  const float cm = sqrtf(gam * pm * irm), cp = sqrtf(gam * pp * irp);
  const float lam = fmaxf(fabsf(unm) + cm, fabsf(unp) + cp);
  float dq[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) dq[v] = qm[v] - qp[v];
  float dF[5];
  dF[0] = dq[1] * n[0] + dq[2] * n[1] + dq[3] * n[2];
#pragma unroll
  for (int ii = 0; ii < 3; ++ii) dF[1 + ii] = qm[1 + ii] * unm - qp[1 + ii] * unp + dpn * n[ii];
  dF[4] = unm * (qm[4] + pm) - unp * (qp[4] + pp);
#pragma unroll
  for (int v = 0; v < 5; ++v) g[v] = 0.5f * (dF[v] - lam * dq[v]);
  if (NS) {
#pragma unroll
    for (int ii = 0; ii < 3; ++ii) {
      float dv = 0.0f;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int cc = kern::tau_index(ii, d);
        dv = fmaf(n[d], fvm[cc] - fvp[cc], dv);
      }
      g[1 + ii] -= 0.5f * dv;
    }
    float de = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) de = fmaf(n[d], fvm[6 + d] - fvp[6 + d], de);
    g[4] -= 0.5f * de;
  }
}

// Mixture volume flux of one node (nvar <= V variables): the Euler part as node_flux<false>,
// and the passive species rho Y_k u_d.
template <int V>
__device__ __forceinline__ void node_flux_mix(const float q[V], int nvar, float dp, float pf, float F[3][V]) {
  const float ir = 1.0f / q[0];
  const float u[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    F[d][0] = q[1 + d];
    F[d][1] = q[1] * u[d];
    F[d][2] = q[2] * u[d];
    F[d][3] = q[3] * u[d];
    F[d][1 + d] += dp;
    F[d][4] = u[d] * (q[4] + pf);
#pragma unroll
    for (int v = 5; v < V; ++v) F[d][v] = v < nvar ? q[v] * u[d] : 0.0f;
  }
}

// Mixture surface term of one face node before Fscale: local Lax-Friedrichs with the sound
// speeds of both traces (from the temperature solve).  dlo: the differences of the low halves of
// momentum and energy, added to the jumps q- - q+ of the dissipation term.
template <int V>
__device__ __forceinline__ void face_term_mix(const float qm[V], const float qp[V], int nvar, float pm, float pp,
                                              float dpn, float cm, float cp, const float n[3], const float dlo[4],
                                              float g[V]) {
  const float irm = 1.0f / qm[0], irp = 1.0f / qp[0];
  const float unm = (qm[1] * n[0] + qm[2] * n[1] + qm[3] * n[2]) * irm;
  const float unp = (qp[1] * n[0] + qp[2] * n[1] + qp[3] * n[2]) * irp;
  const float lam = fmaxf(fabsf(unm) + cm, fabsf(unp) + cp);
  float dq[V];
#pragma unroll
  for (int v = 0; v < V; ++v) dq[v] = qm[v] - qp[v];
#pragma unroll
  for (int v = 1; v < 5; ++v) dq[v] += dlo[v - 1];
  float dF[V];
  dF[0] = dq[1] * n[0] + dq[2] * n[1] + dq[3] * n[2];
#pragma unroll
  for (int ii = 0; ii < 3; ++ii) dF[1 + ii] = qm[1 + ii] * unm - qp[1 + ii] * unp + dpn * n[ii];
  dF[4] = unm * (qm[4] + pm) - unp * (qp[4] + pp);
#pragma unroll
  for (int v = 5; v < V; ++v) dF[v] = qm[v] * unm - qp[v] * unp;
#pragma unroll
  for (int v = 0; v < V; ++v) g[v] = v < nvar ? 0.5f * (dF[v] - lam * dq[v]) : 0.0f;
}

// Viscous flux of one node from the gradients grad[d][w] of w = (rho, rho u, rho v, rho w, T)
// (velocity gradient by the product rule), Stokes hypothesis: fv = (tau_xx, tau_yy, tau_zz,
// tau_xy, tau_xz, tau_yz, (u . tau + kappa grad T)_x, _y, _z).
__device__ __forceinline__ void viscous_flux_node(float rho, const float m[3], const float grad[3][5], float mu,
                                                  float kap, float fv[9]) {
  const float ir = 1.0f / rho;
  const float u[3] = {m[0] * ir, m[1] * ir, m[2] * ir};
  float du[3][3];
#pragma unroll
  for (int ii = 0; ii < 3; ++ii)
#pragma unroll
    for (int d = 0; d < 3; ++d) du[ii][d] = (grad[d][1 + ii] - u[ii] * grad[d][0]) * ir;
  const float divu = du[0][0] + du[1][1] + du[2][2];
  float tau[3][3];
#pragma unroll
  for (int ii = 0; ii < 3; ++ii)
#pragma unroll
    for (int jj = 0; jj < 3; ++jj) tau[ii][jj] = mu * (du[ii][jj] + du[jj][ii]);
#pragma unroll
  for (int ii = 0; ii < 3; ++ii) tau[ii][ii] -= (2.0f / 3.0f) * mu * divu;
  fv[0] = tau[0][0];
  fv[1] = tau[1][1];
  fv[2] = tau[2][2];
  fv[3] = tau[0][1];
  fv[4] = tau[0][2];
  fv[5] = tau[1][2];
#pragma unroll
  for (int d = 0; d < 3; ++d) fv[6 + d] = fmaf(u[0], tau[0][d], fmaf(u[1], tau[1][d], fmaf(u[2], tau[2][d], kap * grad[d][4])));
}

}  // namespace mixk

// The mixed-form view of one mesh and state (k_mixed.cu).
mixk::MixedCase make_mixed_case(const MeshDev& m, const GasParams& g, const double* qin, double* out, double* k,
                                double dt);

}  // namespace dg
