// Mixed-precision form of the DG right-hand side: the D and LIFT contractions run
// on the tensor cores as split-FP16 products (x = hi + lo, each fp16; three
// products hi*hi + hi*lo + lo*hi, FP32 accumulation, ~22-bit operands), the
// pointwise fluxes run in FP32, and the pressure, the differences that would
// cancel (pressure minus an element reference, trace jumps q- - q+, p- - p+) and
// the RK accumulation stay in FP64.
//
// Why the differences: D annihilates constants, so the large, nearly constant
// part of a flux (the pressure in the momentum flux) carries no information but
// would dominate the rounding error of an FP32/FP16 operand.  Subtracting an
// element reference value in FP64 before rounding keeps the operands small.
//
// Contraction layout per block of EPB elements (rows r = element * 5 + variable):
//   C[r][i] = sum_k A[r][k] B[i][k],  A[r][:] = [F_r | F_s | F_t | Fscale g],
//   B[i][:] = [-Dr_i | -Ds_i | -Dt_i | LIFT_i]   =>   C = rhs.
// Each A row is scaled by a power of two to max |.| < 1 before the split; the
// scale is undone on the FP32 result.
#pragma once

#include <cuda_fp16.h>

#include "dg_kernels.cuh"

namespace dg {
namespace mixk {

using kern::GS;

constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }

template <int N>
struct MOrd {
  using O = kern::Ord<N>;
  static constexpr int Np = O::Np, Nfp = O::Nfp, NF = O::NF;
  static constexpr int NPAD = round_up(Np, 8);
  // right-hand side GEMM
  static constexpr int KREAL = 3 * Np + NF;
  static constexpr int KR = round_up(KREAL, 16);
  static constexpr int EPB = N == 1 ? 32 : 16;
  static constexpr int ROWS = EPB * 5;  // multiple of 16
  static constexpr int NODES = EPB * Np;
  static constexpr int NT = round_up(NODES, 32);
  static constexpr int AS = round_up(KR, 32) + 8;        // A row stride (words), = 8 mod 32
  static constexpr int BS = round_up(KR / 2, 32) + 4;    // B row stride (words), = 4 mod 32
  // BR1 pass
  static constexpr int EPBV = N >= 3 ? 8 : (N == 2 ? 16 : 32);
  static constexpr int NODESV = EPBV * Np;
  static constexpr int NTV = round_up(NODESV, 32);
  static constexpr int RW = EPBV * 5, RWP = round_up(RW, 16);    // rows (element, field)
  static constexpr int RJ = EPBV * 15, RJP = round_up(RJ, 16);   // rows (element, field, direction)
  static constexpr int KW = round_up(Np, 16), KJ = round_up(NF, 16);
  static constexpr int ND = round_up(3 * Np, 8);
  static constexpr int AWS = round_up(KW, 32) + 8, AJS = round_up(KJ, 32) + 8;
  static constexpr int BDS = round_up(KW / 2, 32) + 4, BLS = round_up(KJ / 2, 32) + 4;
};

// ---- split-FP16 tensor-core tile --------------------------------------------------------
__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// c (this lane's 4 accumulators of the 16x8 tile at rows m0.., cols n0..) +=
// sum_k A[r][k] B[n][k], k < 16*ksteps.  A: words (hi | lo << 16) per entry, row
// stride AS; B: words of two consecutive k (k | k+1 << 16), row stride BS, hi and lo
// tables.  Products: Ahi*Bhi + Ahi*Blo + Alo*Bhi.
__device__ __forceinline__ void mma_tile(const uint32_t* __restrict__ A, int AS, const uint32_t* __restrict__ Bh,
                                         const uint32_t* __restrict__ Bl, int BS, int m0, int n0, int ksteps,
                                         float* c) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const uint32_t* a0 = A + (m0 + g) * AS + 2 * t;
  const uint32_t* a1 = A + (m0 + g + 8) * AS + 2 * t;
  const uint32_t* bh = Bh + (n0 + g) * BS + t;
  const uint32_t* bl = Bl + (n0 + g) * BS + t;
  for (int ks = 0; ks < ksteps; ++ks) {
    const int k0 = ks * 16;
    const uint2 x0 = *reinterpret_cast<const uint2*>(a0 + k0);
    const uint2 x1 = *reinterpret_cast<const uint2*>(a1 + k0);
    const uint2 x2 = *reinterpret_cast<const uint2*>(a0 + k0 + 8);
    const uint2 x3 = *reinterpret_cast<const uint2*>(a1 + k0 + 8);
    const uint32_t ah[4] = {__byte_perm(x0.x, x0.y, 0x5410), __byte_perm(x1.x, x1.y, 0x5410),
                            __byte_perm(x2.x, x2.y, 0x5410), __byte_perm(x3.x, x3.y, 0x5410)};
    const uint32_t al[4] = {__byte_perm(x0.x, x0.y, 0x7632), __byte_perm(x1.x, x1.y, 0x7632),
                            __byte_perm(x2.x, x2.y, 0x7632), __byte_perm(x3.x, x3.y, 0x7632)};
    const uint32_t bh0 = bh[k0 / 2], bh1 = bh[k0 / 2 + 4];
    const uint32_t bl0 = bl[k0 / 2], bl1 = bl[k0 / 2 + 4];
    mma16816(c, ah, bh0, bh1);
    mma16816(c, ah, bl0, bl1);
    mma16816(c, al, bh0, bh1);
  }
}

// fp32 value (already scaled) -> word (fp16 hi | fp16 lo << 16)
__device__ __forceinline__ uint32_t split_word(float xs) {
  const __half h = __float2half_rn(xs);
  const __half l = __float2half_rn(xs - __half2float(h));
  return (uint32_t)__half_as_ushort(h) | ((uint32_t)__half_as_ushort(l) << 16);
}

// In-place: rows [0, rows) of A hold fp32 bits in columns [0, kreal); each row is
// scaled by 2^-e (max |.| in [0.5, 1)) and split; inv_scale[r] = 2^e.  Columns
// beyond kreal must already be zero words.  One warp per row.
__device__ __forceinline__ void scale_split_rows(uint32_t* A, int AS, int rows, int kreal, float* inv_scale) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = warp; r < rows; r += nw) {
    uint32_t* row = A + r * AS;
    float mx = 0.0f;
    for (int k = lane; k < kreal; k += 32) mx = fmaxf(mx, fabsf(__uint_as_float(row[k])));
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int ex = 0;
    if (mx > 0.0f && isfinite(mx)) frexpf(mx, &ex);
    const float s = ldexpf(1.0f, -ex);
    for (int k = lane; k < kreal; k += 32) row[k] = split_word(__uint_as_float(row[k]) * s);
    if (lane == 0) inv_scale[r] = ldexpf(1.0f, ex);
  }
}

// All (m, n) tiles of C[rows][ncols] = A B^T over ksteps, written (times
// inv_scale[row]) to C with row stride CS; rows >= rows_out are dropped.
__device__ __forceinline__ void block_gemm(const uint32_t* A, int AS, const uint32_t* Bh, const uint32_t* Bl, int BS,
                                           int mtiles, int ntiles, int ksteps, const float* inv_scale, float* C,
                                           int CS, int rows_out, int cols_out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  for (int tile = warp; tile < mtiles * ntiles; tile += nw) {
    const int mt = tile / ntiles, nt = tile - mt * ntiles;
    float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    mma_tile(A, AS, Bh, Bl, BS, mt * 16, nt * 8, ksteps, c);
    const int r0 = mt * 16 + g, r1 = r0 + 8, n = nt * 8 + 2 * t;
    if (r0 < rows_out) {
      const float s = inv_scale[r0];
      if (n < cols_out) C[r0 * CS + n] = c[0] * s;
      if (n + 1 < cols_out) C[r0 * CS + n + 1] = c[1] * s;
    }
    if (r1 < rows_out) {
      const float s = inv_scale[r1];
      if (n < cols_out) C[r1 * CS + n] = c[2] * s;
      if (n + 1 < cols_out) C[r1 * CS + n + 1] = c[3] * s;
    }
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

// Pass 0: per node, FP64 pressure (and temperature) and a float copy of the state,
// so that the later kernels read traces without recomputing or converting them.
template <bool NS>
__global__ void prims_kernel(const double* __restrict__ q, float* __restrict__ qf, double* __restrict__ p_out,
                             double* __restrict__ T_out, unsigned* __restrict__ status, const GasParams gp,
                             const size_t KNp) {
  const double iR = 1.0 / gp.R;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < KNp; i += (size_t)gridDim.x * blockDim.x) {
    double qv[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) qv[v] = q[v * KNp + i];
    float ir32;
    const double ir = recip64(qv[0], ir32);
    const double p = pressure64(gp, qv, ir);
    if (!(qv[0] > 0.0) || !(p > 0.0)) atomicOr(status, DG_STATUS_NONPHYSICAL);
#pragma unroll
    for (int v = 0; v < 5; ++v) qf[v * KNp + i] = (float)qv[v];
    p_out[i] = p;
    if (NS) T_out[i] = p * ir * iR;
  }
}

// ---------------------------------------------------------------------------------------------
// Mixed right-hand side (perfect gas, Euler or Navier-Stokes), optionally fused
// with the LSRK4 stage update (FP64).  Reads the float state copy, the FP64
// pressures and (NS) the float viscous flux produced by the earlier passes.
// ---------------------------------------------------------------------------------------------
template <int N, int PHYS, bool RK>
__global__ void __launch_bounds__(MOrd<N>::NT) rhs_mixed_kernel(
    const double* __restrict__ q, double* __restrict__ out, double* __restrict__ kreg,
    const uint32_t* __restrict__ bh_g, const uint32_t* __restrict__ bl_g, const int32_t* __restrict__ fmask_g,
    const float* __restrict__ geo_g, const int32_t* __restrict__ vmapP, const float* __restrict__ qf_g,
    const double* __restrict__ p_g, const float* __restrict__ fv_g, const GasParams gp, const int K,
    const double a, const double b, const float dt) {
  using M = MOrd<N>;
  constexpr int Np = M::Np, Nfp = M::Nfp, NF = M::NF, EPB = M::EPB, NODES = M::NODES, ROWS = M::ROWS;
  constexpr int AS = M::AS, BS = M::BS, KR = M::KR, NPAD = M::NPAD;
  constexpr bool NS = PHYS == kern::NAVIER_STOKES;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sP = reinterpret_cast<double*>(smem_raw);          // NODES
  uint32_t* sA = reinterpret_cast<uint32_t*>(sP + NODES);    // ROWS * AS
  uint32_t* sBh = sA + ROWS * AS;
  uint32_t* sBl = sBh + NPAD * BS;
  float* sC = reinterpret_cast<float*>(sBl + NPAD * BS);     // ROWS * NPAD
  float* sSc = sC + ROWS * NPAD;                              // ROWS
  float* sQ = sSc + ROWS;                                     // 5 * NODES
  float* sGeo = sQ + 5 * NODES;                               // EPB * GS
  float* sFv = sGeo + EPB * GS;                               // 9 * NODES (NS)
  int* sFm = reinterpret_cast<int*>(sFv + (NS ? 9 * NODES : 0));

  const int tid = threadIdx.x;
  const int e0 = blockIdx.x * EPB;
  const int nel = min(EPB, K - e0);
  const int nn = nel * Np;
  const size_t KNp = (size_t)K * Np;
  const size_t base = (size_t)e0 * Np;

  for (int i = tid; i < ROWS * AS; i += blockDim.x) sA[i] = 0u;
  for (int i = tid; i < NPAD * (KR / 2); i += blockDim.x) {
    const int r = i / (KR / 2), c = i - r * (KR / 2);
    sBh[r * BS + c] = bh_g[i];
    sBl[r * BS + c] = bl_g[i];
  }
  for (int i = tid; i < NF; i += blockDim.x) sFm[i] = fmask_g[i];
  for (int i = tid; i < nel * GS; i += blockDim.x) sGeo[i] = geo_g[(size_t)e0 * GS + i];
  for (int i = tid; i < nn; i += blockDim.x) sP[i] = p_g[base + i];
#pragma unroll
  for (int v = 0; v < 5; ++v)
    for (int i = tid; i < nn; i += blockDim.x) sQ[v * NODES + i] = qf_g[v * KNp + base + i];
  if (NS)
    for (int c = 0; c < 9; ++c)
      for (int i = tid; i < nn; i += blockDim.x) sFv[c * NODES + i] = fv_g[c * KNp + base + i];
  __syncthreads();

  // ---- volume fluxes (FP32; pressure relative to the element's first node, in FP64) ----
  if (tid < nn) {
    const int e = tid / Np, i = tid - e * Np;
    const float* G = sGeo + e * GS;
    const float rho = sQ[tid];
    const float m[3] = {sQ[NODES + tid], sQ[2 * NODES + tid], sQ[3 * NODES + tid]};
    const float E = sQ[4 * NODES + tid];
    const float dp = (float)(sP[tid] - sP[e * Np]);
    const float pf = (float)sP[tid];
    const float ir = 1.0f / rho;
    const float u[3] = {m[0] * ir, m[1] * ir, m[2] * ir};
    float F[3][5];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      F[d][0] = m[d];
      F[d][1] = m[0] * u[d];
      F[d][2] = m[1] * u[d];
      F[d][3] = m[2] * u[d];
      F[d][1 + d] += dp;
      F[d][4] = u[d] * (E + pf);
      if (NS) {
#pragma unroll
        for (int ii = 0; ii < 3; ++ii) F[d][1 + ii] -= sFv[kern::tau_index(ii, d) * NODES + tid];
        F[d][4] -= sFv[(6 + d) * NODES + tid];
      }
    }
#pragma unroll
    for (int ra = 0; ra < 3; ++ra) {
      const float gx = G[3 * ra], gy = G[3 * ra + 1], gz = G[3 * ra + 2];
#pragma unroll
      for (int v = 0; v < 5; ++v)
        sA[(e * 5 + v) * AS + ra * Np + i] = __float_as_uint(fmaf(gx, F[0][v], fmaf(gy, F[1][v], gz * F[2][v])));
    }
  }

  // ---- surface terms (FP32; the pressure jump in FP64) ----
  for (int j = tid; j < nel * NF; j += blockDim.x) {
    const int e = j / NF, mm = j - e * NF, f = mm / Nfp;
    const float* G = sGeo + e * GS;
    const float nx = G[9 + 4 * f], ny = G[10 + 4 * f], nz = G[11 + 4 * f], fs = G[12 + 4 * f];
    const int own = e * Np + sFm[mm];
    const int P = vmapP[(size_t)(e0 + e) * NF + mm];
    float qm[5], qp[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      qm[v] = sQ[v * NODES + own];
      qp[v] = qf_g[v * KNp + P];
    }
    const double pp64 = p_g[P];
    const float dpn = (float)(sP[own] - pp64);
    const float pm = (float)sP[own], pp = (float)pp64;
    const float irm = 1.0f / qm[0], irp = 1.0f / qp[0];
    const float unm = (qm[1] * nx + qm[2] * ny + qm[3] * nz) * irm;
    const float unp = (qp[1] * nx + qp[2] * ny + qp[3] * nz) * irp;
    const float gam = (float)gp.gamma;
    const float cm = sqrtf(gam * pm * irm), cp = sqrtf(gam * pp * irp);
    const float lam = fmaxf(fabsf(unm) + cm, fabsf(unp) + cp);
    const float nn3[3] = {nx, ny, nz};
    float dq[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) dq[v] = qm[v] - qp[v];
    float dF[5];
    dF[0] = dq[1] * nx + dq[2] * ny + dq[3] * nz;
#pragma unroll
    for (int ii = 0; ii < 3; ++ii) dF[1 + ii] = qm[1 + ii] * unm - qp[1 + ii] * unp + dpn * nn3[ii];
    dF[4] = unm * (qm[4] + pm) - unp * (qp[4] + pp);
    float g[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) g[v] = 0.5f * (dF[v] - lam * dq[v]);
    if (NS) {
#pragma unroll
      for (int ii = 0; ii < 3; ++ii) {
        float dv = 0.0f;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const int c = kern::tau_index(ii, d);
          dv = fmaf(nn3[d], sFv[c * NODES + own] - fv_g[c * KNp + P], dv);
        }
        g[1 + ii] -= 0.5f * dv;
      }
      float de = 0.0f;
#pragma unroll
      for (int d = 0; d < 3; ++d) de = fmaf(nn3[d], sFv[(6 + d) * NODES + own] - fv_g[(6 + d) * KNp + P], de);
      g[4] -= 0.5f * de;
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) sA[(e * 5 + v) * AS + 3 * Np + mm] = __float_as_uint(fs * g[v]);
  }
  __syncthreads();

  scale_split_rows(sA, AS, ROWS, M::KREAL, sSc);
  __syncthreads();
  block_gemm(sA, AS, sBh, sBl, BS, ROWS / 16, NPAD / 8, KR / 16, sSc, sC, NPAD, ROWS, NPAD);
  __syncthreads();

  // ---- output / RK update (FP64 accumulation) ----
  if (tid < nn) {
    const int e = tid / Np, i = tid - e * Np;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const float r = sC[(e * 5 + v) * NPAD + i];
      const size_t gi = v * KNp + base + tid;
      if (RK) {
        const double kk = fma(a, a != 0.0 ? kreg[gi] : 0.0, (double)(dt * r));
        kreg[gi] = kk;
        out[gi] = fma(b, kk, q[gi]);
      } else {
        out[gi] = (double)r;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Mixed BR1 pass: gradients of (rho, rho u, T) by two tensor-core contractions
//   C1[(e,f)][(a,i)] = sum_j w[e,f,j] D_a[i][j]                 (volume)
//   C2[(e,f,d)][i]   = sum_m (Fscale n_d (w+ - w-)/2)[e,f,m] LIFT[i][m]   (surface)
// grad_d w = sum_a (dr_a/dx_d) C1 + C2; stress and heat flux in FP32 -> fv[9][K][Np].
// rho and T enter relative to the element's first node and their jumps are FP64
// differences; the momentum comes from the float state copy.
// ---------------------------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(MOrd<N>::NTV) viscous_mixed_kernel(
    const double* __restrict__ q, const float* __restrict__ qf_g, const double* __restrict__ T_g,
    float* __restrict__ fv_out, const uint32_t* __restrict__ dh_g, const uint32_t* __restrict__ dl_g,
    const uint32_t* __restrict__ lh_g, const uint32_t* __restrict__ ll_g, const int32_t* __restrict__ fmask_g,
    const float* __restrict__ geo_g, const int32_t* __restrict__ vmapP, const GasParams gp, const int K) {
  using M = MOrd<N>;
  constexpr int Np = M::Np, Nfp = M::Nfp, NF = M::NF, EPB = M::EPBV, NODES = M::NODESV;
  constexpr int RW = M::RW, RWP = M::RWP, RJ = M::RJ, RJP = M::RJP, KW = M::KW, KJ = M::KJ, ND = M::ND;
  constexpr int AWS = M::AWS, AJS = M::AJS, BDS = M::BDS, BLS = M::BLS, NPAD = M::NPAD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sRho = reinterpret_cast<double*>(smem_raw);        // NODES (FP64)
  double* sT = sRho + NODES;                                  // NODES (FP64)
  uint32_t* sAw = reinterpret_cast<uint32_t*>(sT + NODES);
  uint32_t* sAj = sAw + RWP * AWS;
  uint32_t* sDh = sAj + RJP * AJS;
  uint32_t* sDl = sDh + ND * BDS;
  uint32_t* sLh = sDl + ND * BDS;
  uint32_t* sLl = sLh + NPAD * BLS;
  float* sC1 = reinterpret_cast<float*>(sLl + NPAD * BLS);   // RW x ND
  float* sC2 = sC1 + RW * ND;                                 // RJ x NPAD
  float* sScW = sC2 + RJ * NPAD;
  float* sScJ = sScW + RWP;
  float* sM = sScJ + RJP;                                     // 3 * NODES momentum (float)
  float* sGeo = sM + 3 * NODES;                               // EPB * GS
  int* sFm = reinterpret_cast<int*>(sGeo + EPB * GS);

  const int tid = threadIdx.x;
  const int e0 = blockIdx.x * EPB;
  const int nel = min(EPB, K - e0);
  const int nn = nel * Np;
  const size_t KNp = (size_t)K * Np;
  const size_t base = (size_t)e0 * Np;

  for (int i = tid; i < RWP * AWS + RJP * AJS; i += blockDim.x) sAw[i] = 0u;
  for (int i = tid; i < ND * (KW / 2); i += blockDim.x) {
    const int r = i / (KW / 2), c = i - r * (KW / 2);
    sDh[r * BDS + c] = dh_g[i];
    sDl[r * BDS + c] = dl_g[i];
  }
  for (int i = tid; i < NPAD * (KJ / 2); i += blockDim.x) {
    const int r = i / (KJ / 2), c = i - r * (KJ / 2);
    sLh[r * BLS + c] = lh_g[i];
    sLl[r * BLS + c] = ll_g[i];
  }
  for (int i = tid; i < NF; i += blockDim.x) sFm[i] = fmask_g[i];
  for (int i = tid; i < nel * GS; i += blockDim.x) sGeo[i] = geo_g[(size_t)e0 * GS + i];
  for (int i = tid; i < nn; i += blockDim.x) {
    sRho[i] = q[base + i];
    sT[i] = T_g[base + i];
  }
#pragma unroll
  for (int v = 0; v < 3; ++v)
    for (int i = tid; i < nn; i += blockDim.x) sM[v * NODES + i] = qf_g[(1 + v) * KNp + base + i];
  __syncthreads();

  if (tid < nn) {
    const int e = tid / Np, i = tid - e * Np;
    const int r0 = e * Np;
    sAw[(e * 5 + 0) * AWS + i] = __float_as_uint((float)(sRho[tid] - sRho[r0]));
#pragma unroll
    for (int v = 0; v < 3; ++v) sAw[(e * 5 + 1 + v) * AWS + i] = __float_as_uint(sM[v * NODES + tid]);
    sAw[(e * 5 + 4) * AWS + i] = __float_as_uint((float)(sT[tid] - sT[r0]));
  }
  for (int j = tid; j < nel * NF; j += blockDim.x) {
    const int e = j / NF, mm = j - e * NF, f = mm / Nfp;
    const float* G = sGeo + e * GS;
    const float hfs = 0.5f * G[12 + 4 * f];
    const float nf[3] = {G[9 + 4 * f], G[10 + 4 * f], G[11 + 4 * f]};
    const int own = e * Np + sFm[mm];
    const int P = vmapP[(size_t)(e0 + e) * NF + mm];
    float jump[5];
    jump[0] = (float)(q[P] - sRho[own]);
#pragma unroll
    for (int v = 0; v < 3; ++v) jump[1 + v] = qf_g[(1 + v) * KNp + P] - sM[v * NODES + own];
    jump[4] = (float)(T_g[P] - sT[own]);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const float jf = hfs * jump[v];
#pragma unroll
      for (int d = 0; d < 3; ++d) sAj[(e * 15 + v * 3 + d) * AJS + mm] = __float_as_uint(nf[d] * jf);
    }
  }
  __syncthreads();

  scale_split_rows(sAw, AWS, RWP, Np, sScW);
  scale_split_rows(sAj, AJS, RJP, NF, sScJ);
  __syncthreads();
  block_gemm(sAw, AWS, sDh, sDl, BDS, RWP / 16, ND / 8, KW / 16, sScW, sC1, ND, RW, ND);
  block_gemm(sAj, AJS, sLh, sLl, BLS, RJP / 16, NPAD / 8, KJ / 16, sScJ, sC2, NPAD, RJ, NPAD);
  __syncthreads();

  if (tid < nn) {
    const int e = tid / Np, i = tid - e * Np;
    const float* G = sGeo + e * GS;
    float grad[3][5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const float* c1 = sC1 + (e * 5 + v) * ND;
      const float dr = c1[i], ds = c1[Np + i], dtt = c1[2 * Np + i];
#pragma unroll
      for (int d = 0; d < 3; ++d)
        grad[d][v] = fmaf(G[d], dr, fmaf(G[3 + d], ds, fmaf(G[6 + d], dtt, sC2[(e * 15 + v * 3 + d) * NPAD + i])));
    }
    const float rho = (float)sRho[tid], ir = 1.0f / rho;
    const float u[3] = {sM[tid] * ir, sM[NODES + tid] * ir, sM[2 * NODES + tid] * ir};
    float du[3][3];
#pragma unroll
    for (int ii = 0; ii < 3; ++ii)
#pragma unroll
      for (int d = 0; d < 3; ++d) du[ii][d] = (grad[d][1 + ii] - u[ii] * grad[d][0]) * ir;
    const float mu = (float)gp.mu, kap = (float)gp.kappa;
    const float divu = du[0][0] + du[1][1] + du[2][2];
    float tau[3][3];
#pragma unroll
    for (int ii = 0; ii < 3; ++ii)
#pragma unroll
      for (int jj = 0; jj < 3; ++jj) tau[ii][jj] = mu * (du[ii][jj] + du[jj][ii]);
#pragma unroll
    for (int ii = 0; ii < 3; ++ii) tau[ii][ii] -= (2.0f / 3.0f) * mu * divu;
    const size_t gi = base + tid;
    fv_out[0 * KNp + gi] = tau[0][0];
    fv_out[1 * KNp + gi] = tau[1][1];
    fv_out[2 * KNp + gi] = tau[2][2];
    fv_out[3 * KNp + gi] = tau[0][1];
    fv_out[4 * KNp + gi] = tau[0][2];
    fv_out[5 * KNp + gi] = tau[1][2];
#pragma unroll
    for (int d = 0; d < 3; ++d)
      fv_out[(6 + d) * KNp + gi] = fmaf(u[0], tau[0][d], fmaf(u[1], tau[1][d], fmaf(u[2], tau[2][d], kap * grad[d][4])));
  }
}

template <int N, int PHYS>
constexpr size_t rhs_mixed_smem() {
  using M = MOrd<N>;
  return sizeof(double) * M::NODES + sizeof(uint32_t) * (M::ROWS * M::AS + 2 * M::NPAD * M::BS) +
         sizeof(float) * (M::ROWS * M::NPAD + M::ROWS + 5 * M::NODES + M::EPB * GS +
                          (PHYS == kern::NAVIER_STOKES ? 9 * M::NODES : 0)) +
         sizeof(int) * M::NF;
}

template <int N>
constexpr size_t viscous_mixed_smem() {
  using M = MOrd<N>;
  return sizeof(double) * 2 * M::NODESV +
         sizeof(uint32_t) * (M::RWP * M::AWS + M::RJP * M::AJS + 2 * M::ND * M::BDS + 2 * M::NPAD * M::BLS) +
         sizeof(float) * (M::RW * M::ND + M::RJ * M::NPAD + M::RWP + M::RJP + 3 * M::NODESV + M::EPBV * GS) +
         sizeof(int) * M::NF;
}

}  // namespace mixk
}  // namespace dg
