// Mixed-precision form of the DG right-hand side: the D and LIFT contractions run
// on the tensor cores as split-BF16 products (x = hi + mid + lo, each bf16, so
// 24 significant bits in FP32's exponent range; the six products with term orders
// adding up to at most 2, FP32 accumulation), the pointwise fluxes run in FP32,
// and the pressure, the differences that would cancel (pressure minus an element
// reference, p- - p+, rho and T relative to a reference and their jumps) and the
// RK accumulation stay in FP64.
//
// Why the differences: D annihilates constants, so the large, nearly constant
// part of a flux (the pressure in the momentum flux) carries no information but
// would dominate the rounding error of an FP32 operand.  Subtracting an element
// reference value in FP64 before rounding keeps the operands small.
//
// Contraction layout per block of EPB elements (rows r = element * 5 + variable):
//   C[r][i] = sum_k A[r][k] B[i][k],  A[r][:] = [F_r | F_s | F_t | Fscale g],
//   B[i][:] = [-Dr_i | -Ds_i | -Dt_i | LIFT_i]   =>   C = rhs.
// Every operand is stored as three bf16 arrays (hi, mid, lo) of 32-bit words,
// each word holding two consecutive k; the producing threads write the three
// terms directly, so no rescaling pass is needed.
#pragma once

#include <cuda_bf16.h>

#include "dg_kernels.cuh"

namespace dg {
namespace mixk {

using kern::GS;

constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }
// smallest stride >= w words with stride = 4 (mod 8): the 8 row groups x 4 lanes of an
// mma fragment load then hit 32 distinct banks
constexpr int frag_stride(int w) { return w % 8 <= 4 ? w - w % 8 + 4 : w - w % 8 + 12; }

template <int N>
struct MOrd {
  using O = kern::Ord<N>;
  static constexpr int Np = O::Np, Nfp = O::Nfp, NF = O::NF;
  static constexpr int NPAD = round_up(Np, 8);
  // right-hand side contraction
  static constexpr int KREAL = 3 * Np + NF;
  static constexpr int KR = round_up(KREAL, 16);
  static constexpr int EPB = N == 1 ? 32 : 16;  // default tile (rows EPB * 5, a multiple of 16)
  static constexpr int AS = frag_stride(KR / 2), BS = frag_stride(KR / 2);
  // BR1 pass: volume contraction over Np, one surface contraction per face over Nfp
  static constexpr int EPBV = N >= 3 ? 8 : (N == 2 ? 16 : 32);
  static constexpr int KW = round_up(Np, 16), KF = round_up(Nfp, 16), KJ = 4 * KF;
  static constexpr int ND = round_up(3 * Np, 8);
  static constexpr int AWS = frag_stride(KW / 2), AJS = frag_stride(KJ / 2);
  static constexpr int BDS = frag_stride(KW / 2), BLS = frag_stride(KF / 2);
};

// ---- split-BF16 tensor-core tile --------------------------------------------------------
__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// c (this lane's 4 accumulators of the 16x8 tile at rows m0.., cols n0..) += sum_k A[r][kA0 + k] B[n][k]
// over k < 16 ksteps (kwa0 = kA0 / 2 words into each A row; B rows start at k = 0).  A: three
// term arrays (stride AS words, term stride AT words); B: three term arrays (stride BS, term
// stride BT).  Products (A term, B term): (0,0) (0,1) (1,0) (0,2) (1,1) (2,0).
__device__ __forceinline__ void mma_tile3(const uint32_t* __restrict__ A, int AS, int AT,
                                          const uint32_t* __restrict__ B, int BS, int BT, int m0, int n0,
                                          int kwa0, int ksteps, float* c) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const uint32_t* a0 = A + (m0 + g) * AS + kwa0 + t;
  const uint32_t* a1 = A + (m0 + g + 8) * AS + kwa0 + t;
  const uint32_t* bb = B + (n0 + g) * BS + t;
  for (int ks = 0; ks < ksteps; ++ks) {
    const int kw = ks * 8;
    uint32_t a[3][4], b[3][2];
#pragma unroll
    for (int term = 0; term < 3; ++term) {
      a[term][0] = a0[term * AT + kw];
      a[term][1] = a1[term * AT + kw];
      a[term][2] = a0[term * AT + kw + 4];
      a[term][3] = a1[term * AT + kw + 4];
      b[term][0] = bb[term * BT + kw];
      b[term][1] = bb[term * BT + kw + 4];
    }
    mma_bf16(c, a[0], b[0][0], b[0][1]);
    mma_bf16(c, a[0], b[1][0], b[1][1]);
    mma_bf16(c, a[1], b[0][0], b[0][1]);
    mma_bf16(c, a[0], b[2][0], b[2][1]);
    mma_bf16(c, a[1], b[1][0], b[1][1]);
    mma_bf16(c, a[2], b[0][0], b[0][1]);
  }
}

// Write fp32 value v as three bf16 terms at entry (row, k) of a three-term operand
// (row stride AS words, term stride AT words).
__device__ __forceinline__ void put3(uint32_t* A, int AS, int AT, int row, int k, float v) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(h);
  const __nv_bfloat16 m = __float2bfloat16_rn(r1);
  const __nv_bfloat16 l = __float2bfloat16_rn(r1 - __bfloat162float(m));
  unsigned short* base = reinterpret_cast<unsigned short*>(A + row * AS) + k;
  base[0] = __bfloat16_as_ushort(h);
  base[2 * AT] = __bfloat16_as_ushort(m);
  base[4 * AT] = __bfloat16_as_ushort(l);
}

// All (m, n) tiles of C = A[:, kA0:] B^T over ksteps (A from word offset kwa0, B from its
// first column), written to C with row stride CS; rows >= rows_out and cols >= cols_out are dropped.
__device__ __forceinline__ void block_gemm3(const uint32_t* A, int AS, int AT, const uint32_t* B, int BS, int BT,
                                            int mtiles, int ntiles, int kwa0, int ksteps, float* C, int CS,
                                            int rows_out, int cols_out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  for (int tile = warp; tile < mtiles * ntiles; tile += nw) {
    const int mt = tile / ntiles, nt = tile - mt * ntiles;
    float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    mma_tile3(A, AS, AT, B, BS, BT, mt * 16, nt * 8, kwa0, ksteps, c);
    const int r0 = mt * 16 + g, r1 = r0 + 8, n = nt * 8 + 2 * t;
    if (r0 < rows_out) {
      if (n < cols_out) C[r0 * CS + n] = c[0];
      if (n + 1 < cols_out) C[r0 * CS + n + 1] = c[1];
    }
    if (r1 < rows_out) {
      if (n < cols_out) C[r1 * CS + n] = c[2];
      if (n + 1 < cols_out) C[r1 * CS + n + 1] = c[3];
    }
  }
}

// Copy a three-term table [3][rows][w] words from global into smem with row stride S.
__device__ __forceinline__ void load_table3(uint32_t* dst, int S, const uint32_t* __restrict__ src, int rows, int w) {
  for (int i = threadIdx.x; i < 3 * rows * w; i += blockDim.x) {
    const int term = i / (rows * w), rem = i - term * rows * w, r = rem / w, c = rem - r * w;
    dst[(term * rows + r) * S + c] = src[i];
  }
}

// FP64 reciprocal from an FP32 seed plus one Newton step (relative error ~1e-14).
__device__ __forceinline__ double recip64(double x, float& r32) {
  r32 = 1.0f / (float)x;
  double r = (double)r32;
  return r * fma(-x, r, 2.0);
}

// FP64 pressure of a perfect gas: p = (gamma-1)(rho E - |m|^2 / (2 rho)).
__device__ __forceinline__ double pressure64(const GasParams& g, const double* qv, double ir) {
  return (g.gamma - 1.0) * (qv[4] - 0.5 * ir * fma(qv[1], qv[1], fma(qv[2], qv[2], qv[3] * qv[3])));
}

// Per-node tables of the mixed form, in the mesh's scratch (72 bytes per node).
struct MixedScratch {
  float* fv;   // [9][KNp] viscous flux (BR1 output)
  float* qf;   // [5][KNp] float copy of the state
  double* p;   // [KNp] pressure (FP64)
  double* T;   // [KNp] temperature (FP64, viscous only)
};

__host__ __device__ inline MixedScratch mixed_scratch(double* base, size_t KNp) {
  float* f = reinterpret_cast<float*>(base);
  MixedScratch m;
  m.fv = f;
  m.qf = f + 9 * KNp;
  m.p = reinterpret_cast<double*>(f + 14 * KNp);
  m.T = m.p + KNp;
  return m;
}

// One case of the mixed form: its state buffers (q[0] in, q[1] out for a single
// stage; the two alternate over the stages of a batched step), RK register,
// per-node tables, geometry, neighbour map, size, time step and gas.
struct MixedGas {
  double gamma, R, mu, kappa;
};

struct MixedCase {
  double* q[2];
  double* k;
  float* qf;
  double* p;
  double* T;
  float* fv;
  const float* geo;
  const int32_t* vmapP;
  int K;
  int Np;
  double dt;
  MixedGas gas;
};

// ---- pass 0: per node, FP64 pressure (and temperature) and a float copy of the state,
// so that the later kernels read traces without recomputing or converting them.
__device__ __forceinline__ void prims_node(const MixedCase& c, const double* __restrict__ qin, size_t KNp, size_t i,
                                           unsigned* status) {
  double qv[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) qv[v] = qin[v * KNp + i];
  float ir32;
  const double ir = recip64(qv[0], ir32);
  const double p = (c.gas.gamma - 1.0) * (qv[4] - 0.5 * ir * fma(qv[1], qv[1], fma(qv[2], qv[2], qv[3] * qv[3])));
  if (!(qv[0] > 0.0) || !(p > 0.0)) atomicOr(status, DG_STATUS_NONPHYSICAL);
#pragma unroll
  for (int v = 0; v < 5; ++v) c.qf[v * KNp + i] = (float)qv[v];
  c.p[i] = p;
  if (c.gas.mu > 0.0) c.T[i] = p * ir / c.gas.R;
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

// ---- pointwise FP32 fluxes shared by the mma.sync and tcgen05 tiles ------------------------------
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

// ---- tile configurations -------------------------------------------------------------------
template <int N, int EPB_>
struct RT {  // right-hand side: EPB elements per block
  using M = MOrd<N>;
  static constexpr int Np = M::Np, Nfp = M::Nfp, NF = M::NF, NPAD = M::NPAD, KREAL = M::KREAL, KR = M::KR;
  static constexpr int EPB = EPB_, ROWS = EPB * 5, NODES = EPB * Np, NT = round_up(NODES, 32);
  static constexpr int AS = M::AS, BS = M::BS, AT = ROWS * AS, BT = NPAD * BS;
  static constexpr size_t smem(bool ns) {
    return sizeof(double) * NODES + sizeof(uint32_t) * (3 * AT + 3 * BT) +
           sizeof(float) * (ROWS * NPAD + 5 * NODES + EPB * GS + (ns ? 9 * NODES : 0)) + sizeof(int) * NF;
  }
};

template <int N, int EPB_>
struct VT {  // BR1 pass: EPB elements per block
  using M = MOrd<N>;
  static constexpr int Np = M::Np, Nfp = M::Nfp, NF = M::NF, NPAD = M::NPAD;
  static constexpr int KW = M::KW, KF = M::KF, KJ = M::KJ, ND = M::ND;
  static constexpr int AWS = M::AWS, AJS = M::AJS, BDS = M::BDS, BLS = M::BLS;
  static constexpr int EPB = EPB_, NODES = EPB * Np, NT = round_up(NODES, 32);
  static constexpr int RW = EPB * 5, RWP = round_up(RW, 16);  // rows (element, field)
  static constexpr int AWT = RWP * AWS, AJT = RWP * AJS, BDT = ND * BDS, BLT = 4 * NPAD * BLS;
  static constexpr size_t smem() {
    return sizeof(double) * 2 * NODES + sizeof(uint32_t) * 3 * (AWT + AJT + BDT + BLT) +
           sizeof(float) * (RW * ND + 4 * RW * NPAD + 3 * NODES + EPB * GS) + sizeof(int) * NF;
  }
};

// ---- right-hand side: shared-memory layout, block set-up and one tile --------------------------
template <class T, int PHYS>
struct RhsSmem {
  double* sP;
  uint32_t *sA, *sB;
  float *sC, *sQ, *sGeo, *sFv;
  int* sFm;
  __device__ explicit RhsSmem(unsigned char* raw) {
    sP = reinterpret_cast<double*>(raw);
    sA = reinterpret_cast<uint32_t*>(sP + T::NODES);
    sB = sA + 3 * T::AT;
    sC = reinterpret_cast<float*>(sB + 3 * T::BT);
    sQ = sC + T::ROWS * T::NPAD;
    sGeo = sQ + 5 * T::NODES;
    sFv = sGeo + T::EPB * GS;
    sFm = reinterpret_cast<int*>(sFv + (PHYS == kern::NAVIER_STOKES ? 9 * T::NODES : 0));
  }
};

// Operator table, face map, zeroed contraction operand (its padding stays zero).
template <class T, int PHYS>
__device__ __forceinline__ void rhs_block_setup(const RhsSmem<T, PHYS>& S, const uint32_t* __restrict__ b_g,
                                                const int32_t* __restrict__ fmask_g) {
  const int tid = threadIdx.x;
  for (int i = tid; i < 3 * T::AT; i += blockDim.x) S.sA[i] = 0u;
  load_table3(S.sB, T::BS, b_g, T::NPAD, T::KR / 2);
  for (int i = tid; i < T::NF; i += blockDim.x) S.sFm[i] = fmask_g[i];
  __syncthreads();
}

// Elements [e0, e0 + EPB) of case c: right-hand side and (RK) the stage update.
template <class T, int PHYS, bool RK>
__device__ __forceinline__ void rhs_tile(const RhsSmem<T, PHYS>& S, const MixedCase& c,
                                         const double* __restrict__ qin, double* __restrict__ out, const int e0,
                                         const double a, const double b) {
  constexpr int Np = T::Np, Nfp = T::Nfp, NF = T::NF, EPB = T::EPB, NODES = T::NODES, ROWS = T::ROWS;
  constexpr int AS = T::AS, AT = T::AT, BS = T::BS, BT = T::BT, KR = T::KR, NPAD = T::NPAD;
  constexpr bool NS = PHYS == kern::NAVIER_STOKES;
  const int tid = threadIdx.x;
  const int K = c.K;
  const int nel = min(EPB, K - e0);
  const int nn = nel * Np;
  const size_t KNp = (size_t)K * Np;
  const size_t base = (size_t)e0 * Np;
  const float* __restrict__ qf_g = c.qf;
  const double* __restrict__ p_g = c.p;
  const float* __restrict__ fv_g = c.fv;
  const int32_t* __restrict__ vmapP = c.vmapP;

  if (nel < EPB)  // rows of absent elements: clear what an earlier tile left there
    for (int i = tid; i < 3 * (ROWS - nel * 5) * AS; i += blockDim.x) {
      const int term = i / ((ROWS - nel * 5) * AS), rem = i - term * (ROWS - nel * 5) * AS;
      S.sA[term * AT + nel * 5 * AS + rem] = 0u;
    }
  for (int i = tid; i < nel * GS; i += blockDim.x) S.sGeo[i] = c.geo[(size_t)e0 * GS + i];
  for (int i = tid; i < nn; i += blockDim.x) S.sP[i] = p_g[base + i];
#pragma unroll
  for (int v = 0; v < 5; ++v)
    for (int i = tid; i < nn; i += blockDim.x) S.sQ[v * NODES + i] = qf_g[v * KNp + base + i];
  if (NS)
    for (int cc = 0; cc < 9; ++cc)
      for (int i = tid; i < nn; i += blockDim.x) S.sFv[cc * NODES + i] = fv_g[cc * KNp + base + i];
  __syncthreads();

  // the RK inputs of this thread's node, loaded now so that their latency hides behind the fluxes
  double k_old[5], q_old[5];
  if (RK && tid < nn) {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const size_t gi = v * KNp + base + tid;
      k_old[v] = a != 0.0 ? c.k[gi] : 0.0;
      q_old[v] = qin[gi];
    }
  }

  // volume fluxes (FP32; pressure relative to the element's first node, in FP64)
  if (tid < nn) {
    const int e = tid / Np, i = tid - e * Np;
    const float* G = S.sGeo + e * GS;
    float qv[5], fv[9], F[3][5];
#pragma unroll
    for (int v = 0; v < 5; ++v) qv[v] = S.sQ[v * NODES + tid];
#pragma unroll
    for (int cc = 0; cc < 9; ++cc) fv[cc] = NS ? S.sFv[cc * NODES + tid] : 0.0f;
    node_flux<NS>(qv, (float)(S.sP[tid] - S.sP[e * Np]), (float)S.sP[tid], fv, F);
#pragma unroll
    for (int ra = 0; ra < 3; ++ra) {
      const float gx = G[3 * ra], gy = G[3 * ra + 1], gz = G[3 * ra + 2];
#pragma unroll
      for (int v = 0; v < 5; ++v)
        put3(S.sA, AS, AT, e * 5 + v, ra * Np + i, fmaf(gx, F[0][v], fmaf(gy, F[1][v], gz * F[2][v])));
    }
  }

  // surface terms (FP32; the pressure jump in FP64)
  const float gam = (float)c.gas.gamma;
  for (int j = tid; j < nel * NF; j += blockDim.x) {
    const int e = j / NF, mm = j - e * NF, f = mm / Nfp;
    const float* G = S.sGeo + e * GS;
    const float n3[3] = {G[9 + 4 * f], G[10 + 4 * f], G[11 + 4 * f]};
    const float fs = G[12 + 4 * f];
    const int own = e * Np + S.sFm[mm];
    const int P = vmapP[(size_t)(e0 + e) * NF + mm];
    float qm[5], qp[5], fvm[9], fvp[9];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      qm[v] = S.sQ[v * NODES + own];
      qp[v] = qf_g[v * KNp + P];
    }
#pragma unroll
    for (int cc = 0; cc < 9; ++cc) {
      fvm[cc] = NS ? S.sFv[cc * NODES + own] : 0.0f;
      fvp[cc] = NS ? fv_g[cc * KNp + P] : 0.0f;
    }
    const double pp64 = p_g[P];
    float g[5];
    face_term<NS>(qm, qp, (float)S.sP[own], (float)pp64, (float)(S.sP[own] - pp64), fvm, fvp, n3, gam, g);
#pragma unroll
    for (int v = 0; v < 5; ++v) put3(S.sA, AS, AT, e * 5 + v, 3 * Np + mm, fs * g[v]);
  }
  __syncthreads();

  block_gemm3(S.sA, AS, AT, S.sB, BS, BT, ROWS / 16, NPAD / 8, 0, KR / 16, S.sC, NPAD, ROWS, NPAD);
  __syncthreads();

  // output / RK update (FP64 accumulation)
  if (tid < nn) {
    const float dtf = (float)c.dt;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const int e = tid / Np, i = tid - e * Np;
      const float r = S.sC[(e * 5 + v) * NPAD + i];
      const size_t gi = v * KNp + base + tid;
      if (RK) {
        const double kk = fma(a, k_old[v], (double)(dtf * r));
        c.k[gi] = kk;
        out[gi] = fma(b, kk, q_old[v]);
      } else {
        out[gi] = (double)r;
      }
    }
  }
  __syncthreads();
}

// ---- BR1 pass: shared-memory layout, block set-up and one tile ----------------------------------
template <class T>
struct VisSmem {
  double *sRho, *sT;
  uint32_t *sAw, *sAj, *sD, *sL;
  float *sC1, *sC2, *sM, *sGeo;
  int* sFm;
  __device__ explicit VisSmem(unsigned char* raw) {
    sRho = reinterpret_cast<double*>(raw);
    sT = sRho + T::NODES;
    sAw = reinterpret_cast<uint32_t*>(sT + T::NODES);
    sAj = sAw + 3 * T::AWT;
    sD = sAj + 3 * T::AJT;
    sL = sD + 3 * T::BDT;
    sC1 = reinterpret_cast<float*>(sL + 3 * T::BLT);
    sC2 = sC1 + T::RW * T::ND;
    sM = sC2 + 4 * T::RW * T::NPAD;
    sGeo = sM + 3 * T::NODES;
    sFm = reinterpret_cast<int*>(sGeo + T::EPB * GS);
  }
};

template <class T>
__device__ __forceinline__ void vis_block_setup(const VisSmem<T>& S, const uint32_t* __restrict__ d_g,
                                                const uint32_t* __restrict__ l_g,
                                                const int32_t* __restrict__ fmask_g) {
  const int tid = threadIdx.x;
  for (int i = tid; i < 3 * (T::AWT + T::AJT); i += blockDim.x) S.sAw[i] = 0u;
  load_table3(S.sD, T::BDS, d_g, T::ND, T::KW / 2);
  load_table3(S.sL, T::BLS, l_g, 4 * T::NPAD, T::KF / 2);
  for (int i = tid; i < T::NF; i += blockDim.x) S.sFm[i] = fmask_g[i];
  __syncthreads();
}

// Gradients of (rho, rho u, T):
//   C1[(e,f)][(a,i)]   = sum_j w[e,f,j] D_a[i][j]                             (volume)
//   C2_s[(e,f)][i]     = sum_m (Fscale (w+ - w-)/2)[e,f,s,m] LIFT_s[i][m]      (face s)
// grad_d w = sum_a (dr_a/dx_d) C1 + sum_s n_d,s C2_s; stress and heat flux in FP32 -> fv[9][K][Np].
// rho and T enter relative to the element's first node and their jumps are FP64
// differences; the momentum comes from the float state copy.
template <class T>
__device__ __forceinline__ void vis_tile(const VisSmem<T>& S, const MixedCase& c, const double* __restrict__ qin,
                                         const int e0) {
  constexpr int Np = T::Np, Nfp = T::Nfp, NF = T::NF, EPB = T::EPB, NODES = T::NODES;
  constexpr int RW = T::RW, RWP = T::RWP, KW = T::KW, KF = T::KF, ND = T::ND, NPAD = T::NPAD;
  constexpr int AWS = T::AWS, AJS = T::AJS, BDS = T::BDS, BLS = T::BLS;
  constexpr int AWT = T::AWT, AJT = T::AJT, BDT = T::BDT, BLT = T::BLT;
  const int tid = threadIdx.x;
  const int K = c.K;
  const int nel = min(EPB, K - e0);
  const int nn = nel * Np;
  const size_t KNp = (size_t)K * Np;
  const size_t base = (size_t)e0 * Np;
  const float* __restrict__ qf_g = c.qf;
  const double* __restrict__ T_g = c.T;
  const int32_t* __restrict__ vmapP = c.vmapP;

  if (nel < EPB) {
    const int r0 = nel * 5, nr = RWP - r0;
    for (int i = tid; i < 3 * nr * AWS; i += blockDim.x) {
      const int term = i / (nr * AWS), rem = i - term * nr * AWS;
      S.sAw[term * AWT + r0 * AWS + rem] = 0u;
    }
    for (int i = tid; i < 3 * nr * AJS; i += blockDim.x) {
      const int term = i / (nr * AJS), rem = i - term * nr * AJS;
      S.sAj[term * AJT + r0 * AJS + rem] = 0u;
    }
  }
  for (int i = tid; i < nel * GS; i += blockDim.x) S.sGeo[i] = c.geo[(size_t)e0 * GS + i];
  for (int i = tid; i < nn; i += blockDim.x) {
    S.sRho[i] = qin[base + i];
    S.sT[i] = T_g[base + i];
  }
#pragma unroll
  for (int v = 0; v < 3; ++v)
    for (int i = tid; i < nn; i += blockDim.x) S.sM[v * NODES + i] = qf_g[(1 + v) * KNp + base + i];
  __syncthreads();

  if (tid < nn) {
    const int e = tid / Np, i = tid - e * Np;
    const int r0 = e * Np;
    put3(S.sAw, AWS, AWT, e * 5 + 0, i, (float)(S.sRho[tid] - S.sRho[r0]));
#pragma unroll
    for (int v = 0; v < 3; ++v) put3(S.sAw, AWS, AWT, e * 5 + 1 + v, i, S.sM[v * NODES + tid]);
    put3(S.sAw, AWS, AWT, e * 5 + 4, i, (float)(S.sT[tid] - S.sT[r0]));
  }
  for (int j = tid; j < nel * NF; j += blockDim.x) {
    const int e = j / NF, mm = j - e * NF, f = mm / Nfp, jj = mm - f * Nfp;
    const float hfs = 0.5f * S.sGeo[e * GS + 12 + 4 * f];
    const int own = e * Np + S.sFm[mm];
    const int P = vmapP[(size_t)(e0 + e) * NF + mm];
    const int col = f * KF + jj;  // each face's jumps start a fresh 16-wide k block
    put3(S.sAj, AJS, AJT, e * 5 + 0, col, hfs * (float)(qin[P] - S.sRho[own]));
#pragma unroll
    for (int v = 0; v < 3; ++v)
      put3(S.sAj, AJS, AJT, e * 5 + 1 + v, col, hfs * (qf_g[(1 + v) * KNp + P] - S.sM[v * NODES + own]));
    put3(S.sAj, AJS, AJT, e * 5 + 4, col, hfs * (float)(T_g[P] - S.sT[own]));
  }
  __syncthreads();

  block_gemm3(S.sAw, AWS, AWT, S.sD, BDS, BDT, RWP / 16, ND / 8, 0, KW / 16, S.sC1, ND, RW, ND);
#pragma unroll
  for (int f = 0; f < 4; ++f)
    block_gemm3(S.sAj, AJS, AJT, S.sL + f * NPAD * BLS, BLS, BLT, RWP / 16, NPAD / 8, f * KF / 2, KF / 16,
                S.sC2 + f * RW * NPAD, NPAD, RW, NPAD);
  __syncthreads();

  if (tid < nn) {
    const int e = tid / Np, i = tid - e * Np;
    const float* G = S.sGeo + e * GS;
    float grad[3][5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const float* c1 = S.sC1 + (e * 5 + v) * ND;
      const float dr = c1[i], ds = c1[Np + i], dtt = c1[2 * Np + i];
#pragma unroll
      for (int d = 0; d < 3; ++d) grad[d][v] = fmaf(G[d], dr, fmaf(G[3 + d], ds, G[6 + d] * dtt));
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const float l = S.sC2[(f * RW + e * 5 + v) * NPAD + i];
#pragma unroll
        for (int d = 0; d < 3; ++d) grad[d][v] = fmaf(G[9 + 4 * f + d], l, grad[d][v]);
      }
    }
    const float m3[3] = {S.sM[tid], S.sM[NODES + tid], S.sM[2 * NODES + tid]};
    float f9[9];
    viscous_flux_node((float)S.sRho[tid], m3, grad, (float)c.gas.mu, (float)c.gas.kappa, f9);
    const size_t gi = base + tid;
#pragma unroll
    for (int cc = 0; cc < 9; ++cc) c.fv[cc * KNp + gi] = f9[cc];
  }
  __syncthreads();
}

// ---- kernels: one case (dg_rhs / dg_rk_stage), persistent over its element tiles -----------------
template <int N, int PHYS, bool RK>
__global__ void __launch_bounds__(RT<N, MOrd<N>::EPB>::NT) rhs_mixed_kernel(
    const MixedCase c, const uint32_t* __restrict__ b_g, const int32_t* __restrict__ fmask_g, const double a,
    const double b) {
  using T = RT<N, MOrd<N>::EPB>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const RhsSmem<T, PHYS> S(smem_raw);
  rhs_block_setup<T, PHYS>(S, b_g, fmask_g);
  for (int e0 = blockIdx.x * T::EPB; e0 < c.K; e0 += gridDim.x * T::EPB)
    rhs_tile<T, PHYS, RK>(S, c, c.q[0], c.q[1], e0, a, b);
}

template <int N>
__global__ void __launch_bounds__(VT<N, MOrd<N>::EPBV>::NT) viscous_mixed_kernel(
    const MixedCase c, const uint32_t* __restrict__ d_g, const uint32_t* __restrict__ l_g,
    const int32_t* __restrict__ fmask_g) {
  using T = VT<N, MOrd<N>::EPBV>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const VisSmem<T> S(smem_raw);
  vis_block_setup<T>(S, d_g, l_g, fmask_g);
  for (int e0 = blockIdx.x * T::EPB; e0 < c.K; e0 += gridDim.x * T::EPB) vis_tile<T>(S, c, c.q[0], e0);
}

// ---- kernels: a batch of cases, persistent over a work list of (case, first element) ----------
// The stage's parity picks input and output among each case's two state buffers.
template <int N, int EPB, int PHYS>
__global__ void __launch_bounds__(RT<N, EPB>::NT) rhs_mixed_batched(
    const MixedCase* __restrict__ cases, const int2* __restrict__ work, const int nwork,
    const uint32_t* __restrict__ b_g, const int32_t* __restrict__ fmask_g, const int stage, const double a,
    const double b) {
  using T = RT<N, EPB>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const RhsSmem<T, PHYS> S(smem_raw);
  rhs_block_setup<T, PHYS>(S, b_g, fmask_g);
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int2 it = work[w];
    const MixedCase& c = cases[it.x];
    rhs_tile<T, PHYS, true>(S, c, c.q[stage & 1], c.q[(stage & 1) ^ 1], it.y, a, b);
  }
}

template <int N, int EPB>
__global__ void __launch_bounds__(VT<N, EPB>::NT) viscous_mixed_batched(
    const MixedCase* __restrict__ cases, const int2* __restrict__ work, const int nwork,
    const uint32_t* __restrict__ d_g, const uint32_t* __restrict__ l_g, const int32_t* __restrict__ fmask_g,
    const int stage) {
  using T = VT<N, EPB>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const VisSmem<T> S(smem_raw);
  vis_block_setup<T>(S, d_g, l_g, fmask_g);
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int2 it = work[w];
    const MixedCase& c = cases[it.x];
    vis_tile<T>(S, c, c.q[stage & 1], it.y);
  }
}

}  // namespace mixk

// The mixed-form view of one mesh and state (k_mixed.cu).
mixk::MixedCase make_mixed_case(const MeshDev& m, const GasParams& g, const double* qin, double* out, double* k,
                                double dt);

}  // namespace dg
