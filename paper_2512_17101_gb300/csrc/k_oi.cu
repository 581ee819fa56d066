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
// Both fluxes are degree-N fields, so their parts of the integral are exact.
//
// One persistent block per group of E elements keeps every intermediate in shared memory:
//   1. point-parallel : the state (and viscous flux) at the points, the flux there, its
//                       contravariant components times the weight -> sF[a][v][e][g]
//   2. face-node-par. : the Lax-Friedrichs flux of the traces (ghost states at boundary faces) -> sG
//   3. (a, v, e, i)   : y_a = I^T (W F_a), one sum over the points per output
//   4. (v, e, i)      : rhs = sum_a (M^-1 D_a^T) y_a - LIFT (Fscale f*), then the RK update -> HBM
// The tables (I^T with an odd row stride, the weights, (M^-1 D_a^T)^T, LIFT^T) are loaded once per
// block, laid out so that consecutive threads read consecutive words.  All arithmetic is FP64.
#include <algorithm>

#include "dg_kernels.cuh"

namespace dg {
namespace {

using kern::GS;
using kern::Ord;

// Row stride of I^T in shared memory: the point count, made odd so that threads reading one
// point of consecutive rows hit distinct banks.
__host__ __device__ inline int oi_ldq(int Ng) { return Ng | 1; }

struct OiLayout {
  int ldq, tables, per_elem;  // doubles: tables, and the per-element work
};

template <int N>
__host__ __device__ inline OiLayout oi_layout(int Ng, bool visc, bool av) {
  using O = Ord<N>;
  OiLayout L;
  L.ldq = oi_ldq(Ng);
  L.tables = O::Np * L.ldq + Ng + 3 * O::Np * O::Np + O::NF * O::Np;
  L.per_elem = GS + 5 * O::Np + 15 * Ng + 15 * O::Np + 5 * O::NF + (visc ? 9 * O::Np : 0) + (av ? 15 * O::Np : 0);
  return L;
}

template <int N>
inline size_t oi_smem(int Ng, int E, bool visc, bool av) {
  const OiLayout L = oi_layout<N>(Ng, visc, av);
  return sizeof(double) * ((size_t)L.tables + (size_t)E * L.per_elem) + sizeof(int) * Ord<N>::NF;
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
                                                      const int Ng, const int E, const double a, const double b,
                                                      const double dt) {
  using O = Ord<N>;
  constexpr int Np = O::Np, NF = O::NF;
  const OiLayout L = oi_layout<N>(Ng, VISC, AV);
  const int ldq = L.ldq;
  extern __shared__ double smem[];
  double* sIT = smem;                  // [Np][ldq]: l_j at point g
  double* sW = sIT + Np * ldq;         // [Ng]
  double* sWt = sW + Ng;               // [3][Np(j)][Np(i)]: (M^-1 D_a^T)[i][j]
  double* sLT = sWt + 3 * Np * Np;     // [NF][Np]: LIFT[i][m] at [m][i]
  double* sGeo = sLT + NF * Np;        // [E][GS]
  double* sQ = sGeo + E * GS;          // [5][E][Np]
  double* sF = sQ + 5 * E * Np;        // [3][5][E][Ng]: w_g F_a at the points
  double* sY = sF + 15 * E * Ng;       // [3][5][E][Np]
  double* sG = sY + 15 * E * Np;       // [5][E][NF]: Fscale n.G*
  double* sFv = sG + 5 * E * NF;       // VISC: [9][E][Np] nodal viscous flux (tau xx yy zz xy xz yz, Q)
  double* sS = sFv + (VISC ? 9 * E * Np : 0);  // AV: [15][E][Np] sigma[(5 d + v)], 0 where eps = 0
  int* sFm = reinterpret_cast<int*>(sS + (AV ? 15 * E * Np : 0));
  const int tid = threadIdx.x, NT = blockDim.x;
  const size_t KNp = (size_t)K * Np;

  for (int i = tid; i < Np * Ng; i += NT) {
    const int j = i / Ng, g = i - j * Ng;
    sIT[j * ldq + g] = tab[i];
  }
  for (int i = tid; i < Ng; i += NT) sW[i] = tab[Np * Ng + i];
  for (int i = tid; i < 3 * Np * Np; i += NT) sWt[i] = tab[Np * Ng + Ng + i];
  for (int i = tid; i < Np * NF; i += NT) {
    const int r = i / NF, m = i - r * NF;
    sLT[m * Np + r] = ops_g[3 * Np * Np + i];
  }
  for (int i = tid; i < NF; i += NT) sFm[i] = fmask_g[i];

  const double gm1 = gp.gamma - 1.0;
  const int groups = (K + E - 1) / E;
  for (int grp = blockIdx.x; grp < groups; grp += gridDim.x) {
    const int e0 = grp * E, nel = min(E, K - e0), nn = nel * Np;
    const size_t base = (size_t)e0 * Np;
    __syncthreads();  // the tables are in, and the previous group's reads of sQ/sGeo are done
    for (int i = tid; i < nel * GS; i += NT) sGeo[i] = geo_g[(size_t)e0 * GS + i];
    for (int v = 0; v < 5; ++v)
      for (int i = tid; i < nn; i += NT) sQ[(v * E + i / Np) * Np + i % Np] = q[v * KNp + base + i];
    if (VISC)
      for (int c = 0; c < 9; ++c)
        for (int i = tid; i < nn; i += NT) sFv[(c * E + i / Np) * Np + i % Np] = fv_g[c * KNp + base + i];
    if (AV)  // the AV flux is stored only in elements with eps > 0
      for (int c = 0; c < 15; ++c)
        for (int i = tid; i < nn; i += NT)
          sS[(c * E + i / Np) * Np + i % Np] = av_eps[e0 + i / Np] > 0.0 ? av_g[c * KNp + base + i] : 0.0;
    __syncthreads();

    // ---- 1: state, flux and weighted contravariant flux at every point ----
    for (int it = tid; it < nel * Ng; it += NT) {
      const int e = it / Ng, g = it - e * Ng;
      double qg[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, fvg[9], sg[15];
#pragma unroll
      for (int c = 0; c < 9; ++c) fvg[c] = 0.0;
#pragma unroll
      for (int c = 0; c < 15; ++c) sg[c] = 0.0;
      const bool on = AV && av_eps[e0 + e] > 0.0;
      for (int j = 0; j < Np; ++j) {
        const double l = sIT[j * ldq + g];
#pragma unroll
        for (int v = 0; v < 5; ++v) qg[v] = fma(l, sQ[(v * E + e) * Np + j], qg[v]);
        if (VISC) {
#pragma unroll
          for (int c = 0; c < 9; ++c) fvg[c] = fma(l, sFv[(c * E + e) * Np + j], fvg[c]);
        }
        if (AV && on) {
#pragma unroll
          for (int c = 0; c < 15; ++c) sg[c] = fma(l, sS[(c * E + e) * Np + j], sg[c]);
        }
      }
      const double ir = 1.0 / qg[0];
      const double u[3] = {qg[1] * ir, qg[2] * ir, qg[3] * ir};
      const double p = gm1 * (qg[4] - 0.5 * (qg[1] * u[0] + qg[2] * u[1] + qg[3] * u[2]));
      if (!(qg[0] > 0.0) || !(p > 0.0)) atomicOr(status, DG_STATUS_NONPHYSICAL);
      double F[3][5];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        F[d][0] = qg[1 + d];
        F[d][1] = qg[1] * u[d];
        F[d][2] = qg[2] * u[d];
        F[d][3] = qg[3] * u[d];
        F[d][1 + d] += p;
        F[d][4] = u[d] * (qg[4] + p);
        if (VISC) {
#pragma unroll
          for (int i = 0; i < 3; ++i) F[d][1 + i] -= fvg[kern::tau_index(i, d)];
          F[d][4] -= fvg[6 + d];
        }
        if (AV) {
#pragma unroll
          for (int v = 0; v < 5; ++v) F[d][v] -= sg[5 * d + v];
        }
      }
      const double* G = sGeo + e * GS;
      const double w = sW[g];
#pragma unroll
      for (int ra = 0; ra < 3; ++ra) {
        const double gx = w * G[3 * ra], gy = w * G[3 * ra + 1], gz = w * G[3 * ra + 2];
#pragma unroll
        for (int v = 0; v < 5; ++v)
          sF[((ra * 5 + v) * E + e) * Ng + g] = fma(gx, F[0][v], fma(gy, F[1][v], gz * F[2][v]));
      }
    }

    // ---- 2: Fscale f* at the face nodes (weak form), ghost states at boundary faces ----
    for (int j = tid; j < nel * NF; j += NT) {
      const int e = j / NF, m = j - e * NF, f = m / O::Nfp;
      const double* G = sGeo + e * GS;
      const double nx = G[9 + 4 * f], ny = G[10 + 4 * f], nz = G[11 + 4 * f], fs = G[12 + 4 * f];
      const int own = e * Np + sFm[m];
      const int P = vmapP[(size_t)(e0 + e) * NF + m];  // < 0: boundary face node, -DG_BC_* code
      const size_t Pn = P >= 0 ? (size_t)P : base + own;
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
      if (!(qp[0] > 0.0) || !(pp > 0.0) || !(qm[0] > 0.0) || !(pm > 0.0)) atomicOr(status, DG_STATUS_NONPHYSICAL);
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
            tm[i] = fma(nn3[d], sFv[(c * E + e) * Np + sFm[m]], tm[i]);
            tp[i] = fma(nn3[d], fv_g[c * KNp + Pn], tp[i]);
          }
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          em = fma(nn3[d], sFv[((6 + d) * E + e) * Np + sFm[m]], em);
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
          const int own_n = sFm[m];
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            double sm = 0.0, sp = 0.0;
            if (onM)
              sm = fma(nx, sS[(v * E + e) * Np + own_n],
                       fma(ny, sS[((5 + v) * E + e) * Np + own_n], nz * sS[((10 + v) * E + e) * Np + own_n]));
            if (onP)
              sp = fma(nx, av_g[v * KNp + Pn], fma(ny, av_g[(5 + v) * KNp + Pn], nz * av_g[(10 + v) * KNp + Pn]));
            gs[v] -= 0.5 * (sm + sp);
          }
        }
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) sG[(v * E + e) * NF + m] = fs * gs[v];
    }
    __syncthreads();

    // ---- 3: y_a = I^T (W F_a), one output per thread ----
    for (int it = tid; it < 15 * nel * Np; it += NT) {
      const int i = it % Np, rest = it / Np, e = rest % nel, av = rest / nel;
      const double* F = sF + (av * E + e) * Ng;
      const double* l = sIT + i * ldq;
      double y0 = 0.0, y1 = 0.0;
      int g = 0;
      for (; g + 1 < Ng; g += 2) {
        y0 = fma(l[g], F[g], y0);
        y1 = fma(l[g + 1], F[g + 1], y1);
      }
      if (g < Ng) y0 = fma(l[g], F[g], y0);
      sY[(av * E + e) * Np + i] = y0 + y1;
    }
    __syncthreads();

    // ---- 4: rhs = sum_a (M^-1 D_a^T) y_a - LIFT (Fscale f*), then the output or RK update ----
    for (int it = tid; it < 5 * nel * Np; it += NT) {
      const int i = it % Np, rest = it / Np, e = rest % nel, v = rest / nel;
      double acc = 0.0;
#pragma unroll
      for (int ra = 0; ra < 3; ++ra) {
        const double* y = sY + ((ra * 5 + v) * E + e) * Np;
        const double* W = sWt + ra * Np * Np + i;
#pragma unroll 4
        for (int j = 0; j < Np; ++j) acc = fma(W[j * Np], y[j], acc);
      }
      const double* gq = sG + (v * E + e) * NF;
#pragma unroll 4
      for (int m = 0; m < NF; ++m) acc = fma(-sLT[m * Np + i], gq[m], acc);
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
// an SM's shared memory, else one block with as many elements as fit; 0 when one element does not.
template <int N>
bool oi_config(int Ng, bool visc, bool av, int& E, int& bps, size_t& smem) {
  int dev = 0, per_sm = 0, per_block = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const OiLayout L = oi_layout<N>(Ng, visc, av);
  for (bps = 2; bps >= 1; --bps) {
    const size_t budget = std::min((size_t)per_block, (size_t)per_sm / bps - 1024);
    const size_t fixed = sizeof(double) * L.tables + sizeof(int) * Ord<N>::NF;
    if (budget <= fixed) continue;
    E = (int)((budget - fixed) / (sizeof(double) * L.per_elem));
    E = std::min(E, 64);
    if (E >= (bps == 2 ? 2 : 1)) {
      smem = oi_smem<N>(Ng, E, visc, av);
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
  if (!oi_config<N>(m.oi_ng, VISC, AV, E, bps, smem)) return cudaErrorInvalidConfiguration;
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
                                                            m.fmask, m.geo, m.vmapP, m.status, g, m.bc, m.K, m.oi_ng,
                                                            E, a, b, dt);
  return cudaGetLastError();
}

}  // namespace

bool overint_fits(int N, int Ng, bool visc, bool av) {
  int E = 0, bps = 0;
  size_t smem = 0;
  switch (N) {
    case 1: return oi_config<1>(Ng, visc, av, E, bps, smem);
    case 2: return oi_config<2>(Ng, visc, av, E, bps, smem);
    case 3: return oi_config<3>(Ng, visc, av, E, bps, smem);
    case 4: return oi_config<4>(Ng, visc, av, E, bps, smem);
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
