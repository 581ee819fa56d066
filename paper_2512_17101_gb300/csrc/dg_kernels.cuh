// FP64 nodal-DG kernels for sm_103a: fused volume flux + Lax-Friedrichs surface
// flux + LIFT (+ optional low-storage RK4 stage update), and the BR1 gradient /
// viscous-flux pass.
//
// Data layout (element-major nodal arrays, Sec. 1 Fig. 1): state [V][K][Np],
// node index fastest, so the Np*EPB nodes of a block's EPB consecutive
// elements are one contiguous, coalesced run per variable.  Each block owns EPB
// elements: it stages the reference operators (Dr|Ds|Dt|LIFT), the elements'
// geometric factors and their state in shared memory, then runs three phases
//   1. node-parallel   : pointwise fluxes, contravariant components -> smem
//   2. face-node-par.  : neighbour gather q+ = q[vmapP], numerical flux -> smem
//   3. node-parallel   : -sum_a D_a F_a + LIFT g, then the RK update, -> HBM
// so that no intermediate ever goes to HBM.  On GB300 FP64 runs at 1/64 of the
// FP32 rate, so these kernels are bound by the FP64 pipe, not by HBM.
#pragma once

#include "dg_internal.h"

namespace dg {
namespace kern {

constexpr int GS = DG_GEO_STRIDE;

template <int N>
struct Ord {
  static constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int Nfp = (N + 1) * (N + 2) / 2;
  static constexpr int NF = 4 * Nfp;
  static constexpr int EPB = N == 1 ? 32 : N == 2 ? 16 : 8;  // elements per block
  static constexpr int NODES = EPB * Np;                     // node slots per block
  static constexpr int NT = (NODES + 31) / 32 * 32;          // threads per block
  static constexpr int OPS = 3 * Np * Np + Np * NF;          // doubles in Dr|Ds|Dt|LIFT
};

// EULER_AV / NS_AV: the perfect-gas right-hand sides with the artificial-viscosity flux added.
// MIXTURE_NS: the NASA-7 mixture with viscosity, heat conduction and species diffusion (its
// viscous flux, [9 + 3 ns][K][Np], read from global memory).
enum Phys { EULER = 0, NAVIER_STOKES = 1, MIXTURE = 2, EULER_AV = 3, NS_AV = 4, MIXTURE_NS = 5 };
__host__ __device__ constexpr bool is_mix(int PHYS) { return PHYS == MIXTURE || PHYS == MIXTURE_NS; }
__host__ __device__ constexpr bool has_visc(int PHYS) { return PHYS == NAVIER_STOKES || PHYS == NS_AV; }
__host__ __device__ constexpr bool has_av(int PHYS) { return PHYS == EULER_AV || PHYS == NS_AV; }

// index of tau_ij in the stored symmetric viscous stress (xx yy zz xy xz yz)
__device__ __forceinline__ int tau_index(int i, int j) {
  return i == j ? i : (i + j == 1 ? 3 : (i + j == 2 ? 4 : 5));
}

// Mixture: R_mix and cp_mix at temperature T from mass fractions Y (nasa-7).
__device__ __forceinline__ void mixture_cp_R(const GasParams& g, const double* Y, double T, double& cp,
                                             double& Rmix) {
  cp = 0.0;
  Rmix = 0.0;
#pragma unroll
  for (int k = 0; k < DG_MAX_SPECIES; ++k) {
    if (k >= g.ns) break;
    const double* a = g.a[k];
    const double cpk = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
    cp = fma(Y[k] * g.Rk[k], cpk, cp);
    Rmix = fma(Y[k], g.Rk[k], Rmix);
  }
}

// Pressure and sound speed of state qv (V values) at temperature T (mixture only).
template <int PHYS, int V>
__device__ __forceinline__ void thermo(const GasParams& g, const double* qv, double ir, double T, double& p,
                                       double& c) {
  const double ke = 0.5 * ir * (qv[1] * qv[1] + qv[2] * qv[2] + qv[3] * qv[3]);
  if (!is_mix(PHYS)) {
    p = (g.gamma - 1.0) * (qv[4] - ke);
    c = sqrt(g.gamma * p * ir);
  } else {
    double Y[DG_MAX_SPECIES];
#pragma unroll
    for (int k = 0; k < DG_MAX_SPECIES; ++k) Y[k] = (5 + k < V && k < g.ns) ? qv[5 + k] * ir : 0.0;
    double cp, Rmix;
    mixture_cp_R(g, Y, T, cp, Rmix);
    p = qv[0] * Rmix * T;
    c = sqrt(cp / (cp - Rmix) * p * ir);
  }
}

// Normal Euler flux n.F(q) for velocity normal component un = u.n.
template <int V>
__device__ __forceinline__ void normal_flux(const double* qv, double un, double p, double nx, double ny, double nz,
                                            int nvar, double* fn) {
  fn[0] = qv[0] * un;
  fn[1] = fma(qv[1], un, p * nx);
  fn[2] = fma(qv[2], un, p * ny);
  fn[3] = fma(qv[3], un, p * nz);
  fn[4] = (qv[4] + p) * un;
#pragma unroll
  for (int v = 5; v < V; ++v)
    if (v < nvar) fn[v] = qv[v] * un;
}

// Exterior trace q+ at a boundary face node with code = -vmapP (DG_BC_*): the ghost states of the
// slip wall (mirror state), the no-slip wall (momentum reversed), supersonic inflow (the mesh's
// prescribed state) and supersonic outflow (the interior state).
template <int V>
__device__ __forceinline__ void ghost_state(int code, const double* qm, double nx, double ny, double nz,
                                            const BcParams& bc, int nvar, double* qp) {
#pragma unroll
  for (int v = 0; v < V; ++v) qp[v] = qm[v];
  if (code == DG_BC_SLIP_WALL) {
    const double mn2 = 2.0 * (qm[1] * nx + qm[2] * ny + qm[3] * nz);
    qp[1] = qm[1] - mn2 * nx;
    qp[2] = qm[2] - mn2 * ny;
    qp[3] = qm[3] - mn2 * nz;
  } else if (code == DG_BC_NOSLIP_WALL) {
    qp[1] = -qm[1];
    qp[2] = -qm[2];
    qp[3] = -qm[3];
  } else if (code == DG_BC_INFLOW) {
#pragma unroll
    for (int v = 0; v < V; ++v)
      if (v < nvar) qp[v] = bc.q_in[v];
  }
}

// ---------------------------------------------------------------------------------------------
// Right-hand side, optionally fused with the LSRK4 stage update.
//   RK == false: out = rhs
//   RK == true : k <- a k + dt rhs (k read only if a != 0), out = q + b k
// V is the compile-time maximum of variables; nvar (runtime) <= V are used.
// prim (may be null): [3][K][Np] = (1/rho, p, c) of q per node, evaluated once (a perfect gas by
// prims_fp64_kernel, a mixture by the temperature solve at its converged T) instead of at every
// node and at both traces of every face node here; null: evaluated here.
// ---------------------------------------------------------------------------------------------
template <int N, int V, int PHYS, bool RK>
__global__ void __launch_bounds__(Ord<N>::NT) rhs_kernel(
    const double* __restrict__ q, double* __restrict__ out, double* __restrict__ kreg,
    const double* __restrict__ Tg, const double* __restrict__ prim, const double* __restrict__ ops_g,
    const int32_t* __restrict__ fmask_g,
    const double* __restrict__ geo_g, const int32_t* __restrict__ vmapP, const double* __restrict__ fv_g,
    const double* __restrict__ av_g, const double* __restrict__ av_eps, unsigned* __restrict__ status,
    const GasParams gp, const BcParams bc, const int K, const int nvar, const double a, const double b,
    const double dt, const int kb, const int ke) {
  using O = Ord<N>;
  constexpr int Np = O::Np, Nfp = O::Nfp, NF = O::NF, EPB = O::EPB, NODES = O::NODES;
  extern __shared__ double smem[];
  double* sOps = smem;
  double* sGeo = sOps + O::OPS;
  double* sQ = sGeo + EPB * GS;
  double* sF = sQ + V * NODES;
  double* sG = sF + 3 * V * NODES;
  double* sFv = sG + V * EPB * NF;
  constexpr bool VISC = has_visc(PHYS), AV = has_av(PHYS);
  double* sT = sFv + (VISC ? 9 * NODES : 0);
  int* sFm = reinterpret_cast<int*>(sT + (is_mix(PHYS) ? NODES : 0));

  const int tid = threadIdx.x;
  const int e0 = kb + blockIdx.x * EPB;  // the launch covers elements [kb, ke) of the K
  const int nel = min(EPB, ke - e0);
  const int nn = nel * Np;
  const size_t KNp = (size_t)K * Np;
  const size_t base = (size_t)e0 * Np;

  for (int i = tid; i < O::OPS; i += blockDim.x) sOps[i] = ops_g[i];
  for (int i = tid; i < NF; i += blockDim.x) sFm[i] = fmask_g[i];
  for (int i = tid; i < nel * GS; i += blockDim.x) sGeo[i] = geo_g[(size_t)e0 * GS + i];
#pragma unroll
  for (int v = 0; v < V; ++v)
    if (v < nvar)
      for (int i = tid; i < nn; i += blockDim.x) sQ[v * NODES + i] = q[v * KNp + base + i];
  if (VISC)
    for (int c = 0; c < 9; ++c)
      for (int i = tid; i < nn; i += blockDim.x) sFv[c * NODES + i] = fv_g[c * KNp + base + i];
  if (is_mix(PHYS))
    for (int i = tid; i < nn; i += blockDim.x) sT[i] = Tg[base + i];
  __syncthreads();

  // ---- phase 1: pointwise fluxes, contravariant components ----
  if (tid < nn) {
    const int e = tid / Np;
    const double* G = sGeo + e * GS;
    double qv[V];
#pragma unroll
    for (int v = 0; v < V; ++v) qv[v] = v < nvar ? sQ[v * NODES + tid] : 0.0;
    double ir, p;
    if (is_mix(PHYS) || prim) {  // the pass that wrote them has checked rho and p (a mixture always has them)
      ir = prim[base + tid];
      p = prim[KNp + base + tid];
    } else {
      double c;
      ir = 1.0 / qv[0];
      thermo<PHYS, V>(gp, qv, ir, is_mix(PHYS) ? sT[tid] : 0.0, p, c);
      if (!(qv[0] > 0.0) || !(p > 0.0)) atomicOr(status, DG_STATUS_NONPHYSICAL);
    }
    const double vel[3] = {qv[1] * ir, qv[2] * ir, qv[3] * ir};
    double F[3][V];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      F[d][0] = qv[1 + d];
      F[d][1] = qv[1] * vel[d];
      F[d][2] = qv[2] * vel[d];
      F[d][3] = qv[3] * vel[d];
      F[d][1 + d] += p;
      F[d][4] = vel[d] * (qv[4] + p);
#pragma unroll
      for (int v = 5; v < V; ++v) F[d][v] = qv[v] * vel[d];
      if (VISC) {
#pragma unroll
        for (int i = 0; i < 3; ++i) F[d][1 + i] -= sFv[tau_index(i, d) * NODES + tid];
        F[d][4] -= sFv[(6 + d) * NODES + tid];
      }
      if (PHYS == MIXTURE_NS) {  // viscous flux of the mixture, [9 + 3 ns][K][Np]
        const size_t gi = base + tid;
#pragma unroll
        for (int i = 0; i < 3; ++i) F[d][1 + i] -= fv_g[tau_index(i, d) * KNp + gi];
        F[d][4] -= fv_g[(6 + d) * KNp + gi];
#pragma unroll
        for (int v = 5; v < V; ++v)
          if (v < nvar) F[d][v] -= fv_g[(9 + 3 * (v - 5) + d) * KNp + gi];
      }
      // artificial-viscosity flux eps grad q_v along x_d at av_g[(5 d + v)][K][Np]: zero, and not
      // stored, in elements with eps = 0 (most of them), so it is read from HBM only where eps > 0
      if (AV && av_eps[e0 + e] > 0.0) {
#pragma unroll
        for (int v = 0; v < 5; ++v) F[d][v] -= av_g[(5 * d + v) * KNp + base + tid];
      }
    }
#pragma unroll
    for (int ra = 0; ra < 3; ++ra) {
      const double gx = G[3 * ra], gy = G[3 * ra + 1], gz = G[3 * ra + 2];
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (v < nvar) sF[(ra * V + v) * NODES + tid] = fma(gx, F[0][v], fma(gy, F[1][v], gz * F[2][v]));
    }
  }

  // ---- phase 2: surface terms g = Fscale (n.G- - G*) at the block's face nodes ----
  for (int j = tid; j < nel * NF; j += blockDim.x) {
    const int e = j / NF, m = j - e * NF, f = m / Nfp;
    const double* G = sGeo + e * GS;
    const double nx = G[9 + 4 * f], ny = G[10 + 4 * f], nz = G[11 + 4 * f], fs = G[12 + 4 * f];
    const int own = e * Np + sFm[m];
    const int P = vmapP[(size_t)(e0 + e) * NF + m];  // < 0: boundary face node, -DG_BC_* code
    // a boundary node gathers its own trace, so that interior and boundary nodes run the same
    // code; the ghost state and the exterior viscous fluxes of its condition are applied in the
    // branch below, which interior faces never take
    const size_t Pn = P >= 0 ? (size_t)P : base + own;
    double qm[V], qp[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      qm[v] = v < nvar ? sQ[v * NODES + own] : 0.0;
      qp[v] = v < nvar ? q[v * KNp + Pn] : 0.0;
    }
    if (P < 0) ghost_state<V>(-P, qm, nx, ny, nz, bc, nvar, qp);
    double irm, irp, pm, cm, pp, cp;
    if (is_mix(PHYS) || prim) {
      const size_t gM = base + own;
      irm = prim[gM];
      pm = prim[KNp + gM];
      cm = prim[2 * KNp + gM];
      if (P >= 0 || (is_mix(PHYS) && P != -DG_BC_INFLOW)) {
        // a neighbour node, or a mixture's wall or outflow ghost: that keeps the node's rho, |m|,
        // rho E and rho Y, hence its temperature, p and c (Pn is then the node itself)
        irp = prim[Pn];
        pp = prim[KNp + Pn];
        cp = prim[2 * KNp + Pn];
      } else if (is_mix(PHYS)) {  // a mixture's inflow ghost: q_in at its own temperature
        irp = bc.prim_in[0];
        pp = bc.prim_in[1];
        cp = bc.prim_in[2];
      } else {  // a ghost state of the perfect gas
        irp = 1.0 / qp[0];
        thermo<PHYS, V>(gp, qp, irp, 0.0, pp, cp);
      }
    } else {
      irm = 1.0 / qm[0];
      irp = 1.0 / qp[0];
      thermo<PHYS, V>(gp, qm, irm, is_mix(PHYS) ? sT[own] : 0.0, pm, cm);
      thermo<PHYS, V>(gp, qp, irp, is_mix(PHYS) ? Tg[Pn] : 0.0, pp, cp);
    }
    if (P < 0 && (!(qp[0] > 0.0) || !(pp > 0.0))) atomicOr(status, DG_STATUS_NONPHYSICAL);
    const double unm = (qm[1] * nx + qm[2] * ny + qm[3] * nz) * irm;
    const double unp = (qp[1] * nx + qp[2] * ny + qp[3] * nz) * irp;
    const double lam = fmax(fabs(unm) + cm, fabs(unp) + cp);
    double fm[V], fp[V];
    normal_flux<V>(qm, unm, pm, nx, ny, nz, nvar, fm);
    normal_flux<V>(qp, unp, pp, nx, ny, nz, nvar, fp);
    double g[V];
#pragma unroll
    for (int v = 0; v < V; ++v) g[v] = 0.5 * ((fm[v] - fp[v]) - lam * (qm[v] - qp[v]));
    if (AV) {
      // central artificial-viscosity flux: n.(G- - G*) gains -(n.s- - n.s+)/2; at a boundary node
      // the exterior flux is the interior one (Pn is the node itself)
      const size_t gM = base + own;
      const bool onM = av_eps[e0 + e] > 0.0, onP = av_eps[Pn / Np] > 0.0;
      if (onM || onP) {
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          double sm = 0.0, sp = 0.0;
          if (onM)
            sm = fma(nx, av_g[(0 + v) * KNp + gM], fma(ny, av_g[(5 + v) * KNp + gM], nz * av_g[(10 + v) * KNp + gM]));
          if (onP)
            sp = fma(nx, av_g[(0 + v) * KNp + Pn], fma(ny, av_g[(5 + v) * KNp + Pn], nz * av_g[(10 + v) * KNp + Pn]));
          g[v] -= 0.5 * (sm - sp);
        }
      }
    }
    if (PHYS == MIXTURE_NS) {  // central viscous flux of the mixture
      const size_t gM = base + own;
      const double nn3[3] = {nx, ny, nz};
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        double dm = 0.0, dp = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const int c = tau_index(i, d);
          dm = fma(nn3[d], fv_g[c * KNp + gM], dm);
          dp = fma(nn3[d], fv_g[c * KNp + Pn], dp);
        }
        g[1 + i] -= 0.5 * (dm - dp);
      }
#pragma unroll
      for (int v = 4; v < V; ++v) {
        if (v >= nvar) break;
        const int c0 = v == 4 ? 6 : 9 + 3 * (v - 5);
        double dm = 0.0, dp = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          dm = fma(nn3[d], fv_g[(c0 + d) * KNp + gM], dm);
          dp = fma(nn3[d], fv_g[(c0 + d) * KNp + Pn], dp);
        }
        g[v] -= 0.5 * (dm - dp);
      }
      // at a boundary node the terms above cancel (exterior = interior flux); walls are adiabatic
      // and impermeable (the energy and species rows' exterior normal fluxes are minus the interior
      // ones: g gains minus the interior flux) and a slip wall is shear-free (t+ = 2 (n.t-) n - t-:
      // g gains -(t- - (n.t-) n))
      if (P == -DG_BC_SLIP_WALL || P == -DG_BC_NOSLIP_WALL) {
#pragma unroll
        for (int v = 4; v < V; ++v) {
          if (v >= nvar) break;
          const int c0 = v == 4 ? 6 : 9 + 3 * (v - 5);
          double dm = 0.0;
#pragma unroll
          for (int d = 0; d < 3; ++d) dm = fma(nn3[d], fv_g[(c0 + d) * KNp + gM], dm);
          g[v] -= dm;
        }
        if (P == -DG_BC_SLIP_WALL) {
          double tm[3];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            tm[i] = 0.0;
#pragma unroll
            for (int d = 0; d < 3; ++d) tm[i] = fma(nn3[d], fv_g[tau_index(i, d) * KNp + gM], tm[i]);
          }
          const double tn = tm[0] * nx + tm[1] * ny + tm[2] * nz;
#pragma unroll
          for (int i = 0; i < 3; ++i) g[1 + i] -= tm[i] - tn * nn3[i];
        }
      }
    }
    if (VISC) {
      // central viscous flux: n.(G- - G*) gains -(n.Fv- - n.Fv+)/2
      const double nn3[3] = {nx, ny, nz};
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        double dm = 0.0, dp = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const int c = tau_index(i, d);
          dm = fma(nn3[d], sFv[c * NODES + own], dm);
          dp = fma(nn3[d], fv_g[c * KNp + Pn], dp);
        }
        g[1 + i] -= 0.5 * (dm - dp);
      }
      double em = 0.0, ep = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        em = fma(nn3[d], sFv[(6 + d) * NODES + own], em);
        ep = fma(nn3[d], fv_g[(6 + d) * KNp + Pn], ep);
      }
      g[4] -= 0.5 * (em - ep);
      // at a boundary node the terms above cancel (exterior = interior flux); walls are adiabatic
      // (e+ = -e-: g gains -e-) and a slip wall is shear-free (t+ = 2 (n.t-) n - t-: g gains
      // -(t- - (n.t-) n))
      if (P == -DG_BC_SLIP_WALL || P == -DG_BC_NOSLIP_WALL) {
        g[4] -= em;
        if (P == -DG_BC_SLIP_WALL) {
          double tm[3];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            tm[i] = 0.0;
#pragma unroll
            for (int d = 0; d < 3; ++d) tm[i] = fma(nn3[d], sFv[tau_index(i, d) * NODES + own], tm[i]);
          }
          const double tn = tm[0] * nx + tm[1] * ny + tm[2] * nz;
#pragma unroll
          for (int i = 0; i < 3; ++i) g[1 + i] -= tm[i] - tn * nn3[i];
        }
      }
    }
#pragma unroll
    for (int v = 0; v < V; ++v)
      if (v < nvar) sG[v * EPB * NF + j] = fs * g[v];
  }
  __syncthreads();

  // ---- phase 3: rhs = -sum_a D_a F_a + LIFT g, then output / RK update ----
  if (tid < nn) {
    const int e = tid / Np, i = tid - e * Np;
    const double* Dr = sOps + i * Np;
    const double* Ds = sOps + Np * Np + i * Np;
    const double* Dt = sOps + 2 * Np * Np + i * Np;
    const double* L = sOps + 3 * Np * Np + i * NF;
    double acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0.0;
#pragma unroll 4
    for (int jn = 0; jn < Np; ++jn) {
      const double dr = Dr[jn], ds = Ds[jn], dtt = Dt[jn];
      const int col = e * Np + jn;
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (v < nvar)
          acc[v] = fma(dr, sF[(0 * V + v) * NODES + col],
                       fma(ds, sF[(1 * V + v) * NODES + col], fma(dtt, sF[(2 * V + v) * NODES + col], acc[v])));
    }
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = -acc[v];
#pragma unroll 4
    for (int mm = 0; mm < NF; ++mm) {
      const double l = L[mm];
      const int col = e * NF + mm;
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (v < nvar) acc[v] = fma(l, sG[v * EPB * NF + col], acc[v]);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      if (v >= nvar) break;
      const size_t gi = v * KNp + base + tid;
      if (RK) {
        const double kk = (a != 0.0 ? a * kreg[gi] : 0.0) + dt * acc[v];
        kreg[gi] = kk;
        out[gi] = fma(b, kk, sQ[v * NODES + tid]);
      } else {
        out[gi] = acc[v];
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// BR1 pass 1 for a perfect gas: gradients of w = (rho, rho u, rho v, rho w, T) with
// the central flux, then the viscous stress and energy flux per node:
//   grad_d w = sum_a (dr_a/dx_d) D_a w + sum_f n_d,f LIFT_f (Fscale (w+ - w-)/2)
//   out[9][K][Np] = (tau_xx, tau_yy, tau_zz, tau_xy, tau_xz, tau_yz, Q_x, Q_y, Q_z),
//   Q_d = sum_i u_i tau_id + kappa dT/dx_d.
// prim (may be null): the per-node (1/rho, p, c) of q, as for rhs_kernel.
// ---------------------------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(Ord<N>::NT) viscous_kernel(
    const double* __restrict__ q, double* __restrict__ fv_out, const double* __restrict__ prim,
    const double* __restrict__ ops_g, const int32_t* __restrict__ fmask_g, const double* __restrict__ geo_g,
    const int32_t* __restrict__ vmapP, unsigned* __restrict__ status, const GasParams gp, const BcParams bc,
    const int K, const int kb, const int ke) {
  using O = Ord<N>;
  constexpr int Np = O::Np, Nfp = O::Nfp, NF = O::NF, EPB = O::EPB, NODES = O::NODES;
  constexpr int W = 5;
  extern __shared__ double smem[];
  double* sOps = smem;
  double* sGeo = sOps + O::OPS;
  double* sW = sGeo + EPB * GS;
  double* sJ = sW + W * NODES;
  int* sFm = reinterpret_cast<int*>(sJ + W * EPB * NF);

  const int tid = threadIdx.x;
  const int e0 = kb + blockIdx.x * EPB;  // the launch covers elements [kb, ke) of the K
  const int nel = min(EPB, ke - e0);
  const int nn = nel * Np;
  const size_t KNp = (size_t)K * Np;
  const size_t base = (size_t)e0 * Np;

  for (int i = tid; i < O::OPS; i += blockDim.x) sOps[i] = ops_g[i];
  for (int i = tid; i < NF; i += blockDim.x) sFm[i] = fmask_g[i];
  for (int i = tid; i < nel * GS; i += blockDim.x) sGeo[i] = geo_g[(size_t)e0 * GS + i];
  const double gm1 = gp.gamma - 1.0, iR = 1.0 / gp.R;
  if (tid < nn) {
    double qv[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) qv[v] = q[v * KNp + base + tid];
    double ir, p;
    if (prim) {
      ir = prim[base + tid];
      p = prim[KNp + base + tid];
    } else {
      const double E = q[4 * KNp + base + tid];
      ir = 1.0 / qv[0];
      p = gm1 * (E - 0.5 * ir * (qv[1] * qv[1] + qv[2] * qv[2] + qv[3] * qv[3]));
      if (!(qv[0] > 0.0) || !(p > 0.0)) atomicOr(status, DG_STATUS_NONPHYSICAL);
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) sW[v * NODES + tid] = qv[v];
    sW[4 * NODES + tid] = p * ir * iR;
  }
  __syncthreads();

  for (int j = tid; j < nel * NF; j += blockDim.x) {
    const int e = j / NF, m = j - e * NF, f = m / Nfp;
    const double* G = sGeo + e * GS;
    const double fs = G[12 + 4 * f];
    const int own = e * Np + sFm[m];
    const int P = vmapP[(size_t)(e0 + e) * NF + m];  // < 0: boundary face node, -DG_BC_* code
    const size_t Pn = P >= 0 ? (size_t)P : base + own;  // a boundary node gathers its own trace
    double qp[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) qp[v] = q[v * KNp + Pn];
    if (P < 0) {  // exterior values w(q+) of the face's ghost state
      double qm[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) qm[v] = qp[v];
      ghost_state<5>(-P, qm, G[9 + 4 * f], G[10 + 4 * f], G[11 + 4 * f], bc, 5, qp);
    }
    double irp, pp;
    if (prim && P >= 0) {
      irp = prim[Pn];
      pp = prim[KNp + Pn];
    } else {
      irp = 1.0 / qp[0];
      pp = gm1 * (qp[4] - 0.5 * irp * (qp[1] * qp[1] + qp[2] * qp[2] + qp[3] * qp[3]));
    }
    const double wp[5] = {qp[0], qp[1], qp[2], qp[3], pp * irp * iR};
    const double hf = 0.5 * fs;
#pragma unroll
    for (int v = 0; v < W; ++v) sJ[v * EPB * NF + j] = hf * (wp[v] - sW[v * NODES + own]);
  }
  __syncthreads();

  if (tid < nn) {
    const int e = tid / Np, i = tid - e * Np;
    const double* G = sGeo + e * GS;
    const double* Dr = sOps + i * Np;
    const double* Ds = sOps + Np * Np + i * Np;
    const double* Dt = sOps + 2 * Np * Np + i * Np;
    const double* L = sOps + 3 * Np * Np + i * NF;
    double dref[3][W];
#pragma unroll
    for (int v = 0; v < W; ++v) dref[0][v] = dref[1][v] = dref[2][v] = 0.0;
#pragma unroll 4
    for (int jn = 0; jn < Np; ++jn) {
      const double dr = Dr[jn], ds = Ds[jn], dtt = Dt[jn];
#pragma unroll
      for (int v = 0; v < W; ++v) {
        const double w = sW[v * NODES + e * Np + jn];
        dref[0][v] = fma(dr, w, dref[0][v]);
        dref[1][v] = fma(ds, w, dref[1][v]);
        dref[2][v] = fma(dtt, w, dref[2][v]);
      }
    }
    double grad[3][W];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int v = 0; v < W; ++v)
        grad[d][v] = fma(G[d], dref[0][v], fma(G[3 + d], dref[1][v], G[6 + d] * dref[2][v]));
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      double lf[W];
#pragma unroll
      for (int v = 0; v < W; ++v) lf[v] = 0.0;
#pragma unroll 5
      for (int jj = 0; jj < Nfp; ++jj) {
        const double l = L[f * Nfp + jj];
        const int col = e * NF + f * Nfp + jj;
#pragma unroll
        for (int v = 0; v < W; ++v) lf[v] = fma(l, sJ[v * EPB * NF + col], lf[v]);
      }
      const double nf[3] = {G[9 + 4 * f], G[10 + 4 * f], G[11 + 4 * f]};
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < W; ++v) grad[d][v] = fma(nf[d], lf[v], grad[d][v]);
    }
    const double ir = prim ? prim[base + tid] : 1.0 / sW[tid];  // reloaded: not held across the passes
    const double u[3] = {sW[NODES + tid] * ir, sW[2 * NODES + tid] * ir, sW[3 * NODES + tid] * ir};
    double du[3][3];  // du[i][d] = d u_i / d x_d
#pragma unroll
    for (int ii = 0; ii < 3; ++ii)
#pragma unroll
      for (int d = 0; d < 3; ++d) du[ii][d] = (grad[d][1 + ii] - u[ii] * grad[d][0]) * ir;
    const double mu = gp.mu;
    const double divu = du[0][0] + du[1][1] + du[2][2];
    double tau[3][3];
#pragma unroll
    for (int ii = 0; ii < 3; ++ii)
#pragma unroll
      for (int jj = 0; jj < 3; ++jj) tau[ii][jj] = mu * (du[ii][jj] + du[jj][ii]);
#pragma unroll
    for (int ii = 0; ii < 3; ++ii) tau[ii][ii] -= (2.0 / 3.0) * mu * divu;
    const size_t gi = base + tid;
    fv_out[0 * KNp + gi] = tau[0][0];
    fv_out[1 * KNp + gi] = tau[1][1];
    fv_out[2 * KNp + gi] = tau[2][2];
    fv_out[3 * KNp + gi] = tau[0][1];
    fv_out[4 * KNp + gi] = tau[0][2];
    fv_out[5 * KNp + gi] = tau[1][2];
#pragma unroll
    for (int d = 0; d < 3; ++d)
      fv_out[(6 + d) * KNp + gi] =
          fma(u[0], tau[0][d], fma(u[1], tau[1][d], fma(u[2], tau[2][d], gp.kappa * grad[d][4])));
  }
}

// Dynamic shared memory of rhs_kernel / viscous_kernel, in bytes.
template <int N, int V, int PHYS>
constexpr size_t rhs_smem() {
  using O = Ord<N>;
  return sizeof(double) * (O::OPS + O::EPB * GS + V * O::NODES + 3 * V * O::NODES + V * O::EPB * O::NF +
                           (has_visc(PHYS) ? 9 * O::NODES : 0) + (is_mix(PHYS) ? O::NODES : 0)) +
         sizeof(int) * O::NF;
}

template <int N>
constexpr size_t viscous_smem() {
  using O = Ord<N>;
  return sizeof(double) * (O::OPS + O::EPB * GS + 5 * O::NODES + 5 * O::EPB * O::NF) + sizeof(int) * O::NF;
}

template <int N, int V, int PHYS, bool RK>
cudaError_t launch_rhs_t(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k,
                         const double* T, int nvar, double a, double b, double dt, cudaStream_t s,
                         ElemRange r = ElemRange()) {
  using O = Ord<N>;
  constexpr size_t smem = rhs_smem<N, V, PHYS>();
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(rhs_kernel<N, V, PHYS, RK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int kb = r.begin, ke = r.end < 0 ? m.K : r.end;
  if (ke <= kb) return cudaSuccess;
  const int blocks = (ke - kb + O::EPB - 1) / O::EPB;
  rhs_kernel<N, V, PHYS, RK><<<blocks, O::NT, smem, s>>>(q, out, k, T, m.prim, m.ops,
                                                           m.fmask, m.geo, m.vmapP,
                                                           PHYS == MIXTURE_NS ? m.mix_fv : m.scratch,
                                                           m.av_sig, m.av_eps, m.status, g, m.bc, m.K, nvar, a, b,
                                                           dt, kb, ke);
  return cudaGetLastError();
}

template <int V, int PHYS>
cudaError_t dispatch_rhs(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k,
                         const double* T, bool rk, double a, double b, double dt, cudaStream_t s,
                         ElemRange r = ElemRange()) {
  const int nvar = 5 + g.ns;
  switch (m.N) {
#define DG_CASE(NN)                                                                         \
  case NN:                                                                                  \
    return rk ? launch_rhs_t<NN, V, PHYS, true>(m, g, q, out, k, T, nvar, a, b, dt, s, r)   \
              : launch_rhs_t<NN, V, PHYS, false>(m, g, q, out, k, T, nvar, a, b, dt, s, r);
    DG_CASE(1)
    DG_CASE(2)
    DG_CASE(3)
    DG_CASE(4)
#undef DG_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace kern
}  // namespace dg
