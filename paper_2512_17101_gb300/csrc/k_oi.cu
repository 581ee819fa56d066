// Over-integrated Euler and Navier-Stokes right-hand sides on tetrahedra (Sec. 5.3 names
// over-integration among the stabilisations of its shock runs): the weak form
//   rhs = sum_a M^-1 (I D_a)^T W G_a - LIFT(Fscale n.G*),  G_a = sum_d (dr_a/dx_d) G_d,
// with I the nodal basis at the q^3 points of a Stroud conical-product rule and W its weights
// (tables from build_overint_ops).  Euler: G = F(I q), n.G* the pointwise Lax-Friedrichs flux of
// the face-node traces.  Navier-Stokes (VISC): G = F(I q) - I Fv with the nodal BR1 viscous flux Fv
// of the first pass, and n.G* gains minus the central viscous flux, with the walls' exterior
// viscous fluxes (adiabatic; shear-free at a slip wall).  Artificial viscosity (AV): G also loses the
// interpolant of the nodal flux sigma = eps grad_h q of the AV pass (nonzero only in elements with
// eps > 0), and n.G* the central flux n.(sigma- + sigma+)/2 (sigma+ = sigma- at boundary faces).
//
// Sum factorisation.  The rule is a tensor product in the collapsed coordinates (a_i, b_j, c_k)
// and the orthonormal modes factor there, psi_pqr = A_p(a) B_pq(b) C_pqr(c), so the state at the
// points is u = sum_p A_p sum_q B_pq sum_r C_pqr m_pqr with the modes m = V_o^-1 q, and the
// moments y_n = sum_g w_g psi_n(g) F(g) run the same sums backwards (the weights split over the
// three directions).  The weak-form operator on the moments is M^-1 D_a^T V_o^-T = V_o Dh_a^T,
// because I = Psi V_o^-1 and M^-1 = V_o V_o^T, with the modal derivative matrices
// Dh_a = V_o^-1 D_a V_o, most of whose entries vanish (a mode's derivative has lower degree); they
// are applied sparse, by column.  The geometric factors are constant per element (affine
// tetrahedra), so the moments are taken of the physical flux components and turned contravariant
// on the Np modes, not on the q^3 points.  The diffusive fluxes (VISC, AV) are degree-N nodal
// fields, whose products with the test-function gradients the rule integrates exactly when
// q >= N + 1: their part is the exact M^-1 D_a^T M = V_o Dh_a^T V_o^-1 on their nodal
// contravariant components, so their modes join the moments (the host refuses fewer points).
//
// One persistent block per group of E elements keeps every intermediate in shared memory:
//   A. the modes X = V_o^-1 q; the Lax-Friedrichs flux of the face traces (ghost states at
//      boundary faces), minus the central diffusive fluxes -> sG; the nodal contravariant
//      diffusive flux -> sD
//   B. T1[pq][k] = sum_r C_pqr(c_k) X_pqr                      C. T2[p][j][k] = sum_q B_pq(b_j) T1
//   D. per point: the state sum_p A_p(a_i) T2, its Euler flux F_d -> F (no weight, physical axes)
//   E. S1[p][j][k] = sum_i Aw_p(a_i) F[i][j][k] (folded by the Gauss-Legendre symmetry)
//   F. S2[pq][k] = sum_j Bw_pq(b_j) S1
//   G. y_d[n] = sum_k Cw_n(c_k) S2[pq(n)][k], then Y_a = sum_d (dr_a/dx_d) y_d - V_o^-1 D_a
//   G2. u = sum_a Dh_a^T Y_a (sparse)
//   H. rhs = V_o u - LIFT (Fscale f*), then the RK update -> HBM
// Buffers that are dead by then are reused: T2, S1 and u share R2, X|T1 and S2 share R3, F and Y R1.
// All arithmetic is FP64.
#include <algorithm>

#include "dg_kernels.cuh"

namespace dg {
namespace {

using kern::GS;
using kern::Ord;

// x > 0 and not NaN (+inf included), decided on the bits so that the check costs no FP64 issue:
// positive doubles order like their bit patterns, and NaNs lie above +inf.
__device__ __forceinline__ bool oi_positive(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b <= 0x7FF0000000000000LL;
}

// Shared-memory plan in doubles: the tables once per block, then per element.
struct OiLayout {
  int tA, tB, tC, tables;             // table lengths: A, B, C (each doubled with its weighted copy)
  int r1, r2, r3, per_elem, ints;
};

template <int N>
__host__ __device__ inline OiLayout oi_layout(int q, int nnz, bool diff) {
  using O = Ord<N>;
  constexpr int Np = O::Np, Nt2 = (N + 1) * (N + 2) / 2;
  OiLayout L;
  L.tA = (N + 1) * q;
  L.tB = Nt2 * q;
  L.tC = Np * q;
  L.tables = 2 * (L.tA + L.tB + L.tC) + 2 * Np * Np + nnz + O::NF * Np;
  const int q2 = q * q, q3 = q2 * q;
  L.r1 = 15 * (q3 > Np ? q3 : Np);
  L.r2 = 15 * (N + 1) * q2 > 5 * Np ? 15 * (N + 1) * q2 : 5 * Np;
  L.r3 = 5 * Np + 5 * Nt2 * q > 15 * Nt2 * q ? 5 * Np + 5 * Nt2 * q : 15 * Nt2 * q;
  L.per_elem = GS + 5 * Np + 5 * O::NF + L.r1 + L.r2 + L.r3 + (diff ? 15 * Np : 0);
  // fmask, pq -> (p, first mode, count), p -> first pq, mode -> pq, Dh column starts, rows, columns
  L.ints = O::NF + 3 * Nt2 + (N + 1) + Np + (Np + 1) + nnz + Np;
  return L;
}

template <int N>
inline size_t oi_smem(int q, int nnz, int E, bool diff) {
  const OiLayout L = oi_layout<N>(q, nnz, diff);
  return sizeof(double) * ((size_t)L.tables + (size_t)E * L.per_elem) + sizeof(int) * (size_t)L.ints;
}

template <int N, bool VISC, bool AV, bool RK>
__global__ void __launch_bounds__(512, 1) rhs_oi_kernel(const double* __restrict__ q, double* __restrict__ out,
                                                      double* __restrict__ kreg, const double* __restrict__ tab,
                                                      const double* __restrict__ fv_g,
                                                      const double* __restrict__ av_g,
                                                      const double* __restrict__ av_eps,
                                                      const double* __restrict__ ops_g,
                                                      const int32_t* __restrict__ fmask_g,
                                                      const double* __restrict__ geo_g,
                                                      const int32_t* __restrict__ vmapP, unsigned* __restrict__ status,
                                                      const GasParams gp, const BcParams bc, const int K,
                                                      const int nq, const int nnz, const int E, const double a,
                                                      const double b, const double dt) {
  using O = Ord<N>;
  constexpr int Np = O::Np, NF = O::NF, Nt2 = (N + 1) * (N + 2) / 2;
  constexpr bool DIFF = VISC || AV;
  const OiLayout L = oi_layout<N>(nq, nnz, DIFF);
  const int q2 = nq * nq, q3 = q2 * nq;
  const int lT1 = Nt2 * nq, lT2 = (N + 1) * q2;  // per-slab lengths of T1|S2 and T2|S1
  extern __shared__ double smem[];
  double* sA = smem;                   // [N+1][q], then Aw
  double* sAw = sA + L.tA;
  double* sB = sAw + L.tA;             // [Nt2][q], then Bw
  double* sBw = sB + L.tB;
  double* sC = sBw + L.tB;             // [Np][q], then Cw
  double* sCw = sC + L.tC;
  double* sVi = sCw + L.tC;            // [Np(j)][Np(n)]: (V_o^-1)[n][j]
  double* sVo = sVi + Np * Np;         // [Np(n)][Np(i)]: V_o[i][n]
  double* sDh = sVo + Np * Np;         // [nnz]: Dh_a[m][n] by column n
  double* sLT = sDh + nnz;             // [NF][Np]: LIFT[i][m] at [m][i]
  double* sGeo = sLT + NF * Np;        // [E][GS]
  double* sQ = sGeo + E * GS;          // [5][E][Np]
  double* sG = sQ + 5 * E * Np;        // [5][E][NF]: Fscale n.G*
  double* R1 = sG + 5 * E * NF;        // F [15][E][q3] (slab 5 d + v), then Y [15][E][Np] (slab 5 a + v)
  double* R2 = R1 + E * L.r1;          // T2 [5][E][lT2], then S1 [15][E][lT2], then u [5][E][Np]
  double* R3 = R2 + E * L.r2;          // X [5][E][Np] | T1 [5][E][lT1], then S2 [15][E][lT1]
  double* sD = R3 + E * L.r3;          // DIFF: [15][E][Np] contravariant diffusive flux (slab 5 a + v)
  int* sFm = reinterpret_cast<int*>(sD + (DIFF ? 15 * E * Np : 0));
  int* sPQp = sFm + NF;                // pq -> p
  int* sPQn = sPQp + Nt2;              // pq -> first mode
  int* sPQc = sPQn + Nt2;              // pq -> modes with this (p, q)
  int* sP0 = sPQc + Nt2;               // p -> first pq
  int* sNpq = sP0 + (N + 1);           // mode -> pq
  int* sDp = sNpq + Np;                // [Np + 1]: starts of the stored Dh columns
  int* sDi = sDp + (Np + 1);           // [nnz]: a Np + m of each Dh entry
  int* sDc = sDi + nnz;                // [Np]: the column n of each stored column, longest first
  double* sX = R3;
  double* sT1 = R3 + 5 * E * Np;
  const int tid = threadIdx.x, NT = blockDim.x;
  const size_t KNp = (size_t)K * Np;

  {
    const int ntab = 2 * (L.tA + L.tB + L.tC) + 2 * Np * Np + nnz;
    for (int i = tid; i < ntab; i += NT) smem[i] = tab[i];
    for (int i = tid; i < 2 * Np + 1 + nnz; i += NT) sDp[i] = (int)tab[ntab + i];  // Dh_ptr | Dh_idx | Dh_col
  }
  for (int i = tid; i < Np * NF; i += NT) {
    const int r = i / NF, m = i - r * NF;
    sLT[m * Np + r] = ops_g[3 * Np * Np + i];
  }
  for (int i = tid; i < NF; i += NT) sFm[i] = fmask_g[i];
  if (tid == 0) {
    for (int p = 0, pq = 0, n = 0; p <= N; ++p) {
      sP0[p] = pq;
      for (int qq = 0; p + qq <= N; ++qq, ++pq) {
        sPQp[pq] = p;
        sPQn[pq] = n;
        sPQc[pq] = N + 1 - p - qq;
        for (int r = 0; p + qq + r <= N; ++r) sNpq[n++] = pq;
      }
    }
  }

  const double gm1 = gp.gamma - 1.0;
  const int groups = (K + E - 1) / E;
  for (int grp = blockIdx.x; grp < groups; grp += gridDim.x) {
    const int e0 = grp * E, nel = min(E, K - e0), nn = nel * Np;
    const size_t base = (size_t)e0 * Np;
    __syncthreads();  // the tables are in, and the previous group's reads of sQ, sGeo and R1 are done
    for (int i = tid; i < nel * GS; i += NT) sGeo[i] = geo_g[(size_t)e0 * GS + i];
    for (int v = 0; v < 5; ++v)
      for (int i = tid; i < nn; i += NT) sQ[(v * E + i / Np) * Np + i % Np] = q[v * KNp + base + i];
    __syncthreads();

    // ---- A: modes; face fluxes; nodal contravariant diffusive fluxes ----
    for (int it = tid; it < 5 * nn; it += NT) {
      const int n = it % Np, rest = it / Np, e = rest % nel, v = rest / nel;
      const double* x = sQ + (v * E + e) * Np;
      double acc = 0.0;
#pragma unroll 4
      for (int j = 0; j < Np; ++j) acc = fma(sVi[j * Np + n], x[j], acc);
      sX[(v * E + e) * Np + n] = acc;
    }
    for (int j = tid; j < nel * NF; j += NT) {
      const int e = j / NF, m = j - e * NF, f = m / O::Nfp;
      const double* G = sGeo + e * GS;
      const double nx = G[9 + 4 * f], ny = G[10 + 4 * f], nz = G[11 + 4 * f], fs = G[12 + 4 * f];
      const size_t Mn = base + (size_t)(e * Np + sFm[m]);
      const int P = vmapP[(size_t)(e0 + e) * NF + m];  // < 0: boundary face node, -DG_BC_* code
      const size_t Pn = P >= 0 ? (size_t)P : Mn;
      double qm[5], qp[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        qm[v] = sQ[(v * E + e) * Np + sFm[m]];
        qp[v] = q[v * KNp + Pn];
      }
      if (P < 0) kern::ghost_state<5>(-P, qm, nx, ny, nz, bc, 5, qp);
      const double irm = 1.0 / qm[0], irp = 1.0 / qp[0];
      const double pm = gm1 * (qm[4] - 0.5 * irm * (qm[1] * qm[1] + qm[2] * qm[2] + qm[3] * qm[3]));
      const double pp = gm1 * (qp[4] - 0.5 * irp * (qp[1] * qp[1] + qp[2] * qp[2] + qp[3] * qp[3]));
      if (!oi_positive(qp[0]) || !oi_positive(pp) || !oi_positive(qm[0]) || !oi_positive(pm))
        atomicOr(status, DG_STATUS_NONPHYSICAL);
      const double cm = sqrt(gp.gamma * pm * irm), cp = sqrt(gp.gamma * pp * irp);
      const double unm = (qm[1] * nx + qm[2] * ny + qm[3] * nz) * irm;
      const double unp = (qp[1] * nx + qp[2] * ny + qp[3] * nz) * irp;
      const double lam = fmax(fabs(unm) + cm, fabs(unp) + cp);
      double fm[5], fp[5];
      kern::normal_flux<5>(qm, unm, pm, nx, ny, nz, 5, fm);
      kern::normal_flux<5>(qp, unp, pp, nx, ny, nz, 5, fp);
      double gs[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) gs[v] = 0.5 * ((fm[v] + fp[v]) + lam * (qm[v] - qp[v]));
      if (VISC) {
        // minus the central viscous flux (n.Fv- + n.Fv+)/2: traction t = tau n and energy flux e;
        // at a boundary node the exterior flux is the interior one (Pn is the node itself), except
        // that walls are adiabatic (e+ = -e-) and a slip wall is shear-free (t+ = 2 (n.t-) n - t-)
        const double nn3[3] = {nx, ny, nz};
        double tm[3], tp[3], em = 0.0, ep = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          tm[i] = 0.0;
          tp[i] = 0.0;
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const int c = kern::tau_index(i, d);
            tm[i] = fma(nn3[d], fv_g[c * KNp + Mn], tm[i]);
            tp[i] = fma(nn3[d], fv_g[c * KNp + Pn], tp[i]);
          }
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          em = fma(nn3[d], fv_g[(6 + d) * KNp + Mn], em);
          ep = fma(nn3[d], fv_g[(6 + d) * KNp + Pn], ep);
        }
        if (P == -DG_BC_SLIP_WALL || P == -DG_BC_NOSLIP_WALL) {
          ep = -em;
          if (P == -DG_BC_SLIP_WALL) {
            const double tn = tm[0] * nx + tm[1] * ny + tm[2] * nz;
#pragma unroll
            for (int i = 0; i < 3; ++i) tp[i] = 2.0 * tn * nn3[i] - tm[i];
          }
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) gs[1 + i] -= 0.5 * (tm[i] + tp[i]);
        gs[4] -= 0.5 * (em + ep);
      }
      if (AV) {
        // minus the central AV flux n.(sigma- + sigma+)/2; at a boundary node Pn is the node itself,
        // so sigma+ = sigma-
        const bool onM = av_eps[e0 + e] > 0.0, onP = av_eps[Pn / Np] > 0.0;
        if (onM || onP) {
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            double sm = 0.0, sp = 0.0;
            if (onM) sm = fma(nx, av_g[v * KNp + Mn], fma(ny, av_g[(5 + v) * KNp + Mn], nz * av_g[(10 + v) * KNp + Mn]));
            if (onP) sp = fma(nx, av_g[v * KNp + Pn], fma(ny, av_g[(5 + v) * KNp + Pn], nz * av_g[(10 + v) * KNp + Pn]));
            gs[v] -= 0.5 * (sm + sp);
          }
        }
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) sG[(v * E + e) * NF + m] = fs * gs[v];
    }
    if (DIFF) {
      // sD[5 a + v] = sum_d (dr_a/dx_d) Fd_d[v], Fd = Fv + sigma (Fv: rows 1-4, sigma only where
      // eps > 0); a row with nothing in it is left out of H and not written
      for (int it = tid; it < nn; it += NT) {
        const int e = it / Np, j = it - e * Np;
        const double* G = sGeo + e * GS;
        const size_t gn = base + it;
        const bool on = AV && av_eps[e0 + e] > 0.0;
        double fd[3][5];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
#pragma unroll
          for (int v = 0; v < 5; ++v) fd[d][v] = on ? av_g[(5 * d + v) * KNp + gn] : 0.0;
          if (VISC) {
#pragma unroll
            for (int i = 0; i < 3; ++i) fd[d][1 + i] += fv_g[kern::tau_index(i, d) * KNp + gn];
            fd[d][4] += fv_g[(6 + d) * KNp + gn];
          }
        }
#pragma unroll
        for (int ra = 0; ra < 3; ++ra)
#pragma unroll
          for (int v = 0; v < 5; ++v)
            sD[((5 * ra + v) * E + e) * Np + j] =
                fma(G[3 * ra], fd[0][v], fma(G[3 * ra + 1], fd[1][v], G[3 * ra + 2] * fd[2][v]));
      }
    }
    __syncthreads();

    // ---- B: T1[pq][k] = sum_r C_pqr(c_k) X_pqr ----
    for (int it = tid; it < 5 * nel * lT1; it += NT) {
      const int idx = it % lT1, rest = it / lT1, e = rest % nel, v = rest / nel;
      const int pq = idx / nq, k = idx - pq * nq;
      const int n0 = sPQn[pq], cnt = sPQc[pq];
      const double* x = sX + (v * E + e) * Np + n0;
      double acc = 0.0;
      for (int r = 0; r < cnt; ++r) acc = fma(sC[(n0 + r) * nq + k], x[r], acc);
      sT1[(v * E + e) * lT1 + idx] = acc;
    }
    __syncthreads();

    // ---- C: T2[p][j][k] = sum_q B_pq(b_j) T1[pq][k] (into R2) ----
    for (int it = tid; it < 5 * nel * lT2; it += NT) {
      const int idx = it % lT2, rest = it / lT2, e = rest % nel, v = rest / nel;
      const int p = idx / q2, jk = idx - p * q2, j = jk / nq, k = jk - j * nq;
      const int pq0 = sP0[p];
      const double* t1 = sT1 + (v * E + e) * lT1 + k;
      double acc = 0.0;
      for (int qq = 0; qq <= N - p; ++qq) acc = fma(sB[(pq0 + qq) * nq + j], t1[(pq0 + qq) * nq], acc);
      R2[(v * E + e) * lT2 + idx] = acc;
    }
    __syncthreads();

    // ---- D: state and Euler flux at every point (g = (k q + j) q + i) -> F (R1) ----
    for (int it = tid; it < nel * q3; it += NT) {
      const int e = it / q3, g = it - e * q3;
      const int i = g % nq, jk = g / nq;  // jk = k q + j
      const int j = jk % nq, k = jk / nq;
      double qg[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double* t2 = R2 + (v * E + e) * lT2 + j * nq + k;
        double acc = 0.0;
#pragma unroll
        for (int p = 0; p <= N; ++p) acc = fma(sA[p * nq + i], t2[p * q2], acc);
        qg[v] = acc;
      }
      const double ir = 1.0 / qg[0];
      const double u[3] = {qg[1] * ir, qg[2] * ir, qg[3] * ir};
      // rho u_c u_d, each product once: the flux's momentum block is symmetric
      const double mxx = qg[1] * u[0], myy = qg[2] * u[1], mzz = qg[3] * u[2];
      const double mxy = qg[1] * u[1], mxz = qg[1] * u[2], myz = qg[2] * u[2];
      const double p = gm1 * fma(-0.5, mxx + myy + mzz, qg[4]);
      if (!oi_positive(qg[0]) || !oi_positive(p)) atomicOr(status, DG_STATUS_NONPHYSICAL);
      const double H = qg[4] + p;
      double* F = R1 + e * q3 + g;
      const int sl = E * q3;  // slab stride
      F[0 * sl] = qg[1];
      F[1 * sl] = mxx + p;
      F[2 * sl] = mxy;
      F[3 * sl] = mxz;
      F[4 * sl] = u[0] * H;
      F[5 * sl] = qg[2];
      F[6 * sl] = mxy;
      F[7 * sl] = myy + p;
      F[8 * sl] = myz;
      F[9 * sl] = u[1] * H;
      F[10 * sl] = qg[3];
      F[11 * sl] = mxz;
      F[12 * sl] = myz;
      F[13 * sl] = mzz + p;
      F[14 * sl] = u[2] * H;
    }
    __syncthreads();

    // ---- E: S1[p][j][k] = sum_i Aw_p(a_i) F[(k q + j) q + i] (into R2), one thread per line
    //      (s, e, j, k) for every p, folded by the rule's symmetry Aw_p(a_(q-1-i)) = (-1)^p Aw_p(a_i):
    //      even p take F_i + F_(q-1-i), odd p the difference, and odd p skip the middle point ----
    {
      const int h = nq >> 1;
      for (int it = tid; it < 15 * nel * q2; it += NT) {
        const int jk = it % q2, rest = it / q2, e = rest % nel, s = rest / nel;
        const int j = jk / nq, k = jk - j * nq;
        const double* f = R1 + (s * E + e) * q3 + (k * nq + j) * nq;
        double acc[N + 1];
#pragma unroll
        for (int p = 0; p <= N; ++p) acc[p] = 0.0;
        for (int i = 0; i < h; ++i) {
          const double x = f[i], y = f[nq - 1 - i];
          const double ev = x + y, od = x - y;
#pragma unroll
          for (int p = 0; p <= N; ++p) acc[p] = fma(sAw[p * nq + i], (p & 1) ? od : ev, acc[p]);
        }
        if (nq & 1) {
          const double mid = f[h];
#pragma unroll
          for (int p = 0; p <= N; p += 2) acc[p] = fma(sAw[p * nq + h], mid, acc[p]);
        }
        double* o = R2 + (s * E + e) * lT2 + jk;  // S1 index (p q + j) q + k = p q^2 + jk
#pragma unroll
        for (int p = 0; p <= N; ++p) o[p * q2] = acc[p];
      }
    }
    __syncthreads();

    // ---- F: S2[pq][k] = sum_j Bw_pq(b_j) S1[p][j][k] (into R3) ----
    for (int it = tid; it < 15 * nel * lT1; it += NT) {
      const int idx = it % lT1, rest = it / lT1, e = rest % nel, s = rest / nel;
      const int pq = idx / nq, k = idx - pq * nq;
      const double* s1 = R2 + (s * E + e) * lT2 + sPQp[pq] * q2 + k;
      const double* w = sBw + pq * nq;
      double acc = 0.0;
      for (int j = 0; j < nq; ++j) acc = fma(w[j], s1[j * nq], acc);
      R3[(s * E + e) * lT1 + idx] = acc;
    }
    __syncthreads();

    // ---- G: moments y_d[n] = sum_k Cw_n(c_k) S2[pq(n)][k], contravariant Y_a, less the modes of
    //      the nodal contravariant diffusive flux (into R1) ----
    for (int it = tid; it < 5 * nn; it += NT) {
      const int n = it % Np, rest = it / Np, e = rest % nel, v = rest / nel;
      const double* w = sCw + n * nq;
      const int off = sNpq[n] * nq;
      double y[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double* s2 = R3 + ((5 * d + v) * E + e) * lT1 + off;
        double acc = 0.0;
        for (int k = 0; k < nq; ++k) acc = fma(w[k], s2[k], acc);
        y[d] = acc;
      }
      const double* G = sGeo + e * GS;
      const bool dif = DIFF && ((AV && av_eps[e0 + e] > 0.0) || (VISC && v > 0));
#pragma unroll
      for (int ra = 0; ra < 3; ++ra) {
        double ya = fma(G[3 * ra], y[0], fma(G[3 * ra + 1], y[1], G[3 * ra + 2] * y[2]));
        if (dif) {
          // the diffusive part, M^-1 D_a^T M D_a = V_o Dh_a^T (V_o^-1 D_a): its modes join the moments
          const double* dd = sD + ((5 * ra + v) * E + e) * Np;
          double acc = 0.0;
#pragma unroll 4
          for (int j = 0; j < Np; ++j) acc = fma(sVi[j * Np + n], dd[j], acc);
          ya -= acc;
        }
        R1[((5 * ra + v) * E + e) * Np + n] = ya;
      }
    }
    __syncthreads();

    // ---- G2: modal divergence u[n] = sum_a sum_m Dh_a[m][n] Y_a[m] (into R2) ----
    // stored column c, then field and element, so that a warp's threads walk columns of similar
    // length (the columns are stored longest first)
    for (int it = tid; it < 5 * nn; it += NT) {
      const int c = it / (5 * nel), r = it - c * 5 * nel, v = r / nel, e = r - v * nel;
      const int n = sDc[c];
      const double* Y = R1 + (v * E + e) * Np;  // Y_a at Y[a 5 E Np + m]
      double acc = 0.0;
      for (int x = sDp[c]; x < sDp[c + 1]; ++x) {
        const int am = sDi[x], ra = am / Np, m = am - ra * Np;
        acc = fma(sDh[x], Y[ra * 5 * E * Np + m], acc);
      }
      R2[(v * E + e) * Np + n] = acc;
    }
    __syncthreads();

    // ---- H: rhs = V_o u - LIFT (Fscale f*), then the output or RK update ----
    for (int it = tid; it < 5 * nn; it += NT) {
      const int i = it % Np, rest = it / Np, e = rest % nel, v = rest / nel;
      const double* u = R2 + (v * E + e) * Np;
      double acc = 0.0, acl = 0.0;
#pragma unroll 4
      for (int n = 0; n < Np; ++n) acc = fma(sVo[n * Np + i], u[n], acc);
      const double* gq = sG + (v * E + e) * NF;
#pragma unroll 4
      for (int m = 0; m < NF; ++m) acl = fma(sLT[m * Np + i], gq[m], acl);
      acc -= acl;
      const size_t gi = v * KNp + base + e * Np + i;
      if (RK) {
        const double kk = (a != 0.0 ? a * kreg[gi] : 0.0) + dt * acc;
        kreg[gi] = kk;
        out[gi] = fma(b, kk, sQ[(v * E + e) * Np + i]);
      } else {
        out[gi] = acc;
      }
    }
  }
}

// Elements per block and blocks per SM: two blocks of at least two elements each if they fit in
// an SM's shared memory, else one block with as many elements as fit; false when one element does
// not.
template <int N>
bool oi_config(int nq, int nnz, bool diff, int& E, int& bps, size_t& smem) {
  int dev = 0, per_sm = 0, per_block = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const OiLayout L = oi_layout<N>(nq, nnz, diff);
  for (bps = 2; bps >= 1; --bps) {
    const size_t budget = std::min((size_t)per_block, (size_t)per_sm / bps - 1024);
    const size_t fixed = sizeof(double) * L.tables + sizeof(int) * L.ints;
    if (budget <= fixed) continue;
    E = (int)((budget - fixed) / (sizeof(double) * L.per_elem));
    E = std::min(E, 64);
    if (E >= (bps == 2 ? 2 : 1)) {
      smem = oi_smem<N>(nq, nnz, E, diff);
      return true;
    }
  }
  return false;
}

template <int N, bool VISC, bool AV, bool RK>
cudaError_t launch_oi_t(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k, double a,
                        double b, double dt, cudaStream_t s) {
  int E = 0, bps = 0;
  size_t smem = 0;
  if (!oi_config<N>(m.oi_q, m.oi_nnz, VISC || AV, E, bps, smem)) return cudaErrorInvalidConfiguration;
  cudaError_t e =
      cudaFuncSetAttribute(rhs_oi_kernel<N, VISC, AV, RK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int NT = bps == 2 ? 256 : 512;
  const int groups = (m.K + E - 1) / E;
  const int blocks = std::min(groups, sms * bps);
  rhs_oi_kernel<N, VISC, AV, RK><<<blocks, NT, smem, s>>>(q, out, k, m.oi_tab, m.scratch, m.av_sig, m.av_eps, m.ops,
                                                            m.fmask, m.geo, m.vmapP, m.status, g, m.bc, m.K, m.oi_q, m.oi_nnz,
                                                            E, a, b, dt);
  return cudaGetLastError();
}

}  // namespace

bool overint_fits(int N, int q, int nnz, bool visc, bool av) {
  int E = 0, bps = 0;
  size_t smem = 0;
  const bool diff = visc || av;
  switch (N) {
    case 1: return oi_config<1>(q, nnz, diff, E, bps, smem);
    case 2: return oi_config<2>(q, nnz, diff, E, bps, smem);
    case 3: return oi_config<3>(q, nnz, diff, E, bps, smem);
    case 4: return oi_config<4>(q, nnz, diff, E, bps, smem);
    default: return false;
  }
}

cudaError_t launch_rhs_overint(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k,
                               bool rk, double a, double b, double dt, cudaStream_t s) {
  const bool av = m.av.eps0 > 0;
  switch (m.N) {
#define DG_PICK(NN, VI, AVV)                                                          \
  return rk ? launch_oi_t<NN, VI, AVV, true>(m, g, q, out, k, a, b, dt, s)            \
            : launch_oi_t<NN, VI, AVV, false>(m, g, q, out, k, a, b, dt, s);
#define DG_CASE(NN)                    \
  case NN:                             \
    if (g.mu > 0) {                    \
      if (av) { DG_PICK(NN, true, true) } \
      DG_PICK(NN, true, false)         \
    }                                  \
    if (av) { DG_PICK(NN, false, true) } \
    DG_PICK(NN, false, false)
    DG_CASE(1)
    DG_CASE(2)
    DG_CASE(3)
    DG_CASE(4)
#undef DG_CASE
#undef DG_PICK
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace dg
