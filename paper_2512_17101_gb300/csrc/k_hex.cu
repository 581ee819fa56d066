// Nodal DG on tensor-product hexahedra (the element type of the paper's timed runs, Sec. 5.2-5.4):
// Euler and Navier-Stokes (BR1) equations of a perfect gas, and scalar advection, on a box of
// axis-aligned hexahedra, FP64, fused with the low-storage RK4 stage like the tetrahedral path.
//
// Discretisation (collocated nodal spectral-element DG): tensor-product nodes from a 1-D node
// set x_0 = -1 < ... < x_N = 1 (Gauss-Lobatto-Legendre in the workloads), quadrature weights
// w_i = integral of the Lagrange basis l_i, D[i][j] = l_j'(x_i); diagonal collocated mass;
//   rhs = - sum_d (2/h_d) D_d F_d + sum over the faces f a node lies on (2/h_d(f)) / w_end (n.F- - n.F*),
// local Lax-Friedrichs n.F*.  Sum factorisation: the derivative along d at node (i, j, k) reads the
// N+1 fluxes on the line through the node, 3 (N+1) products per variable instead of (N+1)^3.
//
// Kernel layout: EPB whole elements per block (so that the lines are in the block's shared
// memory).  Node-parallel: fluxes, 1/rho, p and c into shared memory, then the line derivatives.
// Face-node-parallel: the Lax-Friedrichs terms, one axis at a time so that no two face nodes of a
// pass add into the same node (no warp of consecutive nodes steps through faces only some of its
// lanes lie on); the neighbour's face node (same position on the shared face, mirrored index along
// the face normal) read from global memory.  Neighbours come from the box structure: no geometry
// or map arrays.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "dg_cvt.cuh"
#include "dg_internal.h"

struct dg_hex_mesh_s {
  int n[3] = {0, 0, 0};
  int bc[6] = {0, 0, 0, 0, 0, 0};
  double q_in[5] = {0, 0, 0, 0, 0};
  bool has_inflow = false;
  double L[3] = {0, 0, 0};
  int N = 0, M = 0, Np = 0;
  int64_t K = 0;
  std::vector<double> nodes, w, D;  // host copies
  double* D_dev = nullptr;          // [M][M]
  double* fv_dev = nullptr;         // Navier-Stokes viscous flux [9][K][Np] (on first use)
  double* prim = nullptr;           // [3][K][Np] 1/rho, p, c of the state (on first use)
  // artificial viscosity (dg_hex_set_av): parameters, element viscosity [K], flux [15][K][Np]
  double av_eps0 = 0.0, av_s0 = 0.0, av_kappa = 1.0;
  double* av_eps = nullptr;
  double* av_sig = nullptr;
  bool overint = false;             // dg_hex_set_overintegration
  std::vector<double> oi_I, oi_A, oi_B;  // [Q][M], [M][Q], [M][Q]
  std::vector<double> oi_An, oi_Bn;      // [M][M]: A I and B I, the same contractions of a nodal field
  std::vector<double> modal;        // [M][M]: nodal values -> Legendre coefficients (GLL-weighted)
  std::vector<double> modal_norm;   // [M]: discrete norms of the Legendre polynomials
  unsigned* status = nullptr;
};

namespace dg {
namespace hexk {

template <int N>
struct HexCfg {
  static constexpr int M = N + 1, Np = M * M * M;
  static constexpr int EPB = N == 1 ? 32 : (N == 2 ? 8 : (N == 3 ? 4 : 2));
  static constexpr int NODES = EPB * Np, NT = (NODES + 31) / 32 * 32;
};

// Coefficients with the stage's dt folded in (s = dt in an RK stage, 1 for the right-hand side), so
// that the kernel accumulates dt * rhs directly: the volume term uses D_d = -(2/h_d) s D.
struct HexGeo {
  int n[3];
  int bc[6];        // DG_BC_* code of the box faces x-, x+, y-, y+, z-, z+ (0: periodic)
  double q_in[5];   // DG_BC_INFLOW state
  double dsc[3];    // -(2/h_d) s
  double lf[3][2];  // (2/h_d) / w_end s / 2
};

// FP64 reciprocal and square root from FP32 seeds (conversions on the integer pipe) and one
// Newton step each, relative error a few 1e-14: the IEEE FP64 division and square root are long
// instruction sequences on the FP64 pipe, which bounds this kernel, and every face incidence
// needs a trace's 1/rho and sound speed.
__device__ __forceinline__ double rcp_nr(double x) {
  const double r = cvt::widen(1.0f / cvt::narrow(x));
  return r * fma(-x, r, 2.0);
}
__device__ __forceinline__ double sqrt_nr(double x) {
  const double y = cvt::widen(rsqrtf(cvt::narrow(x)));  // ~ x^-1/2
  const double s = x * y;                                // ~ x^1/2
  return fma(0.5 * y, fma(-s, s, x), s);                 // s + (x - s^2) / (2 sqrt x)
}

// 1/rho, pressure and sound speed of a perfect gas.
__device__ __forceinline__ void pc(double gamma, const double* q, double& ir, double& p, double& c) {
  ir = rcp_nr(q[0]);
  p = (gamma - 1.0) * (q[4] - 0.5 * ir * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]));
  c = sqrt_nr(gamma * p * ir);
}

// 1/rho, p and c of every node into prim [3][K][Np], once per node: the right-hand-side and
// viscous kernels read them at their own nodes and at the neighbour trace of every face node
// instead of evaluating them there.  rho <= 0 or p <= 0 at a node sets DG_STATUS_NONPHYSICAL.
__global__ void __launch_bounds__(256) hex_prims_kernel(const double* __restrict__ q, double* __restrict__ prim,
                                                        const int64_t n, const double gamma,
                                                        unsigned* __restrict__ status) {
  bool bad = false;
  for (int64_t t = blockIdx.x * 256LL + threadIdx.x; t < n; t += (int64_t)gridDim.x * 256) {
    const double qv[5] = {q[t], q[n + t], q[2 * n + t], q[3 * n + t], q[4 * n + t]};
    double ir, p, c;
    pc(gamma, qv, ir, p, c);
    if (!(qv[0] > 0.0) || !(p > 0.0)) bad = true;
    prim[t] = ir;
    prim[n + t] = p;
    prim[2 * n + t] = c;
  }
  if (bad) atomicOr(status, (unsigned)DG_STATUS_NONPHYSICAL);
}

// The six neighbours of element e, slot 2d + end (end 0: the -x_d side), in 32-bit
// arithmetic (K < 2^31 is checked on the host): the 64-bit integer division is a long sequence
// whose conversions compete for the FP64 pipe that bounds these kernels.  Computed once per
// element, not per face node.
__device__ __forceinline__ void hex_neighbours(unsigned e, const int n[3], int* nb, const int* bc = nullptr) {
  const unsigned nx = n[0], ny = n[1], nz = n[2], nxy = nx * ny;
  const unsigned t = e / nx, ex = e - t * nx, ez = t / ny, ey = t - ez * ny;
  nb[0] = (int)(ex == 0 ? e + (nx - 1) : e - 1);
  nb[1] = (int)(ex == nx - 1 ? e - (nx - 1) : e + 1);
  nb[2] = (int)(ey == 0 ? e + (ny - 1) * nx : e - nx);
  nb[3] = (int)(ey == ny - 1 ? e - (ny - 1) * nx : e + nx);
  nb[4] = (int)(ez == 0 ? e + (nz - 1) * nxy : e - nxy);
  nb[5] = (int)(ez == nz - 1 ? e - (nz - 1) * nxy : e + nxy);
  if (bc) {  // faces on a non-periodic box boundary: -code
    if (ex == 0 && bc[0]) nb[0] = -bc[0];
    if (ex == nx - 1 && bc[1]) nb[1] = -bc[1];
    if (ey == 0 && bc[2]) nb[2] = -bc[2];
    if (ey == ny - 1 && bc[3]) nb[3] = -bc[3];
    if (ez == 0 && bc[4]) nb[4] = -bc[4];
    if (ez == nz - 1 && bc[5]) nb[5] = -bc[5];
  }
}

// Viscous flux storage of the Navier-Stokes form: [9][K][Np] = tau_xx, tau_yy, tau_zz, tau_xy,
// tau_xz, tau_yz, E_x, E_y, E_z (E_d = sum_i u_i tau_id + kappa dT/dx_d).
__host__ __device__ constexpr int hex_tau(int i, int d) { return i == d ? i : (i + d == 1 ? 3 : (i + d == 2 ? 4 : 5)); }

// Ghost state of a box-face node (n = -e_d or +e_d; q holds the node's own state on entry): slip
// wall (normal momentum mirrored), no-slip wall (momentum reversed), inflow (the prescribed state),
// outflow (the node's own).
__device__ __forceinline__ void hex_ghost(int code, int d, const HexGeo& geo, double* q) {
  if (code == DG_BC_SLIP_WALL) {
    q[1 + d] = -q[1 + d];
  } else if (code == DG_BC_NOSLIP_WALL) {
    q[1] = -q[1];
    q[2] = -q[2];
    q[3] = -q[3];
  } else if (code == DG_BC_INFLOW) {
#pragma unroll
    for (int v = 0; v < 5; ++v) q[v] = geo.q_in[v];
  }
}

// VISC: Navier-Stokes; fv holds the viscous flux of every node (hex_vis_kernel), subtracted from
// the volume fluxes and from the face traces' normal fluxes (central viscous flux).
// AV: the artificial-viscosity flux sig [(5 d + v)][K][Np] (eps grad q_v, stored only for elements
// with eps > 0) is subtracted like the viscous flux.
template <int N, bool RK, bool VISC, bool AV>
__global__ void __launch_bounds__(HexCfg<N>::NT) hex_rhs_kernel(const double* __restrict__ q, double* __restrict__ out,
                                                                 double* __restrict__ kreg,
                                                                 const double* __restrict__ D_g, const HexGeo geo,
                                                                 const int64_t K, const double gamma, const double a,
                                                                 const double b, const int accumulate,
                                                                 unsigned* __restrict__ status,
                                                                 const double* __restrict__ fv,
                                                                 const double* __restrict__ sig,
                                                                 const double* __restrict__ eps,
                                                                 const double* __restrict__ prim) {
  using C = HexCfg<N>;
  constexpr int M = C::M, Np = C::Np, EPB = C::EPB, NODES = C::NODES, NT = C::NT;
  __shared__ double sD[3][M * M];     // -(2/h_d) s D per axis
  __shared__ double sF[3][5][NODES];  // volume fluxes
  __shared__ double sS[5][NODES];     // lifted surface terms
  __shared__ double sPC[3][NODES];    // 1/rho, p, c of the block's nodes
  __shared__ int sNb[EPB][6];
  const int tid = threadIdx.x;
#pragma unroll
  for (int d = 0; d < 3; ++d)
    for (int i = tid; i < M * M; i += NT) sD[d][i] = geo.dsc[d] * D_g[i];
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  const int nel = (int)min((int64_t)EPB, K - e0);
  const int nn = nel * Np;
  const size_t KNp = (size_t)K * Np;
  const size_t base = (size_t)e0 * Np;
  double qv[5] = {0, 0, 0, 0, 0};
  if (tid < nel) hex_neighbours((unsigned)(e0 + tid), geo.n, sNb[tid], geo.bc);
  if (tid < nn) {
#pragma unroll
    for (int v = 0; v < 5; ++v) qv[v] = q[v * KNp + base + tid];
    const double ir = prim[base + tid], p = prim[KNp + base + tid];  // checked by the primitives pass
    sPC[0][tid] = ir;
    sPC[1][tid] = p;
    sPC[2][tid] = prim[2 * KNp + base + tid];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double ud = qv[1 + d] * ir;
      sF[d][0][tid] = qv[1 + d];
      sF[d][1][tid] = qv[1] * ud;
      sF[d][2][tid] = qv[2] * ud;
      sF[d][3][tid] = qv[3] * ud;
      sF[d][1 + d][tid] += p;
      sF[d][4][tid] = ud * (qv[4] + p);
      if (VISC) {
#pragma unroll
        for (int i = 0; i < 3; ++i) sF[d][1 + i][tid] -= fv[hex_tau(i, d) * KNp + base + tid];
        sF[d][4][tid] -= fv[(6 + d) * KNp + base + tid];
      }
      if (AV && eps[e0 + tid / Np] > 0.0) {
#pragma unroll
        for (int v = 0; v < 5; ++v) sF[d][v][tid] -= sig[(5 * d + v) * KNp + base + tid];
      }
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) sS[v][tid] = 0.0;
  }
  __syncthreads();

  // surface: face-node-parallel, one axis at a time (a node lies on at most one face of an axis,
  // so within a pass no two face nodes add into the same node)
  constexpr int FPA = 2 * M * M;  // face nodes of one element on the two faces of an axis
  constexpr int stride[3] = {1, M, M * M};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int s1 = stride[(d + 1) % 3], s2 = stride[(d + 2) % 3];
    for (int w = tid; w < nel * FPA; w += NT) {
      const int el = w / FPA, rem = w - el * FPA, end = rem / (M * M), ab = rem - end * M * M;
      const int ia = ab % M, ib = ab / M;
      const int node = (end ? N : 0) * stride[d] + ia * s1 + ib * s2;
      const int loc = el * Np + node;
      const int nnode = node + (end ? -N : N) * stride[d];  // mirrored index along d
      const int enb = sNb[el][2 * d + end];                 // < 0: box boundary, -DG_BC_* code
      const size_t gM = base + loc, gP = enb >= 0 ? (size_t)enb * Np + nnode : gM;
      double qm[5], qp[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        qm[v] = q[v * KNp + gM];
        qp[v] = q[v * KNp + gP];
      }
      const double irm = sPC[0][loc], pm = sPC[1][loc], cm = sPC[2][loc];
      double irp, pp, cp;
      if (enb >= 0) {
        irp = prim[gP];
        pp = prim[KNp + gP];
        cp = prim[2 * KNp + gP];
      } else {  // the ghost state
        hex_ghost(-enb, d, geo, qp);
        pc(gamma, qp, irp, pp, cp);
        if (!(qp[0] > 0.0) || !(pp > 0.0)) atomicOr(status, DG_STATUS_NONPHYSICAL);
      }
      // n = +-e_d: n.F(q) = +-(F_d(q)); the sign folded into the lifted term
      const double um = qm[1 + d] * irm, up = qp[1 + d] * irp;
      const double lam = fmax(fabs(um) + cm, fabs(up) + cp);
      double fm[5], fp[5];
      fm[0] = qm[1 + d];
      fp[0] = qp[1 + d];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        fm[1 + i] = qm[1 + i] * um;
        fp[1 + i] = qp[1 + i] * up;
      }
      fm[1 + d] += pm;
      fp[1 + d] += pp;
      fm[4] = um * (qm[4] + pm);
      fp[4] = up * (qp[4] + pp);
      if (VISC) {  // G_d = F_d - Fv_d on both traces: the central viscous flux
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          fm[1 + i] -= fv[hex_tau(i, d) * KNp + gM];
          fp[1 + i] -= fv[hex_tau(i, d) * KNp + gP];
        }
        fm[4] -= fv[(6 + d) * KNp + gM];
        fp[4] -= fv[(6 + d) * KNp + gP];
        // at a box boundary gP is the node itself: walls are adiabatic (E_d+ = -E_d-) and a slip
        // wall is shear-free (tau_id+ = -tau_id- for i != d)
        if (enb == -DG_BC_SLIP_WALL || enb == -DG_BC_NOSLIP_WALL) {
          fp[4] += 2.0 * fv[(6 + d) * KNp + gM];
          if (enb == -DG_BC_SLIP_WALL)
#pragma unroll
            for (int i = 0; i < 3; ++i)
              if (i != d) fp[1 + i] += 2.0 * fv[hex_tau(i, d) * KNp + gM];
        }
      }
      if (AV) {  // central artificial-viscosity flux; at a box boundary the exterior flux is the interior one
        const bool onM = eps[e0 + el] > 0.0, onP = enb >= 0 ? eps[enb] > 0.0 : onM;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          if (onM) fm[v] -= sig[(5 * d + v) * KNp + gM];
          if (onP) fp[v] -= sig[(5 * d + v) * KNp + gP];
        }
      }
      // n.G- - n.G* = (sgn (G_d- - G_d+) - lam (q- - q+)) / 2, lifted by (2/h_d) / w_end (times s)
      const double lf = end ? geo.lf[d][1] : geo.lf[d][0];
      const double sgnlf = end ? lf : -lf;
#pragma unroll
      for (int v = 0; v < 5; ++v) sS[v][loc] += fma(sgnlf, fm[v] - fp[v], -lf * lam * (qm[v] - qp[v]));
    }
    __syncthreads();
  }
  if (tid >= nn) return;

  const int el = tid / Np, node = tid - el * Np;
  const int idx[3] = {node % M, (node / M) % M, node / (M * M)};
  double acc[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) acc[v] = sS[v][tid];
  // volume: - sum_d (2/h_d) s sum_l D[idx_d][l] F_d(line node l)
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int line0 = el * Np + node - idx[d] * stride[d];
    const double* Drow = sD[d] + idx[d] * M;
#pragma unroll
    for (int l = 0; l < M; ++l) {
      const double dl = Drow[l];
      const int src = line0 + l * stride[d];
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v] = fma(dl, sF[d][v][src], acc[v]);
    }
  }

#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const size_t gi = v * KNp + base + tid;
    if (RK) {
      const double kk = accumulate ? fma(a, kreg[gi], acc[v]) : acc[v];  // acc = dt rhs
      kreg[gi] = kk;
      out[gi] = fma(b, kk, qv[v]);
    } else {
      out[gi] = acc[v];
    }
  }
}

// BR1 gradient pass of the Navier-Stokes form: w = (rho, rho u, rho v, rho w, T), exterior values
// w(q+) of the ghost state at box-boundary faces,
//   grad_d w = (2/h_d) D_d w + (at a node of a d-face) (2/h_d)/w_end n_d (w+ - w-)/2,
// then the viscous flux per node (Stokes hypothesis, kappa = mu cp / Pr) into fv [9][K][Np].
// geo carries the unscaled coefficients: dsc[d] = -(2/h_d), lf[d][end] = (2/h_d)/w_end / 2.
template <int N>
__global__ void __launch_bounds__(HexCfg<N>::NT) hex_vis_kernel(const double* __restrict__ q, double* __restrict__ fv,
                                                                 const double* __restrict__ D_g, const HexGeo geo,
                                                                 const int64_t K, const double gamma, const double R,
                                                                 const double mu, const double kappa,
                                                                 const double* __restrict__ prim) {
  using C = HexCfg<N>;
  constexpr int M = C::M, Np = C::Np, EPB = C::EPB, NODES = C::NODES, NT = C::NT;
  __shared__ double sD[3][M * M];     // (2/h_d) D per axis
  __shared__ double sW[5][NODES];     // w of the block's nodes
  __shared__ double sJ[3][5][NODES];  // lifted jump terms per axis
  __shared__ int sNb[EPB][6];
  const int tid = threadIdx.x;
#pragma unroll
  for (int d = 0; d < 3; ++d)
    for (int i = tid; i < M * M; i += NT) sD[d][i] = -geo.dsc[d] * D_g[i];
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  const int nel = (int)min((int64_t)EPB, K - e0);
  const int nn = nel * Np;
  const size_t KNp = (size_t)K * Np;
  const size_t base = (size_t)e0 * Np;
  const double gm1 = gamma - 1.0, iR = 1.0 / R;
  if (tid < nel) hex_neighbours((unsigned)(e0 + tid), geo.n, sNb[tid], geo.bc);
  if (tid < nn) {
    double qv[5];
#pragma unroll
    for (int v = 0; v < 4; ++v) qv[v] = q[v * KNp + base + tid];
    const double ir = prim[base + tid], p = prim[KNp + base + tid];
#pragma unroll
    for (int v = 0; v < 4; ++v) sW[v][tid] = qv[v];
    sW[4][tid] = p * ir * iR;
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int v = 0; v < 5; ++v) sJ[d][v][tid] = 0.0;
  }
  __syncthreads();
  constexpr int FPA = 2 * M * M;
  constexpr int stride[3] = {1, M, M * M};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int s1 = stride[(d + 1) % 3], s2 = stride[(d + 2) % 3];
    for (int w = tid; w < nel * FPA; w += NT) {
      const int el = w / FPA, rem = w - el * FPA, end = rem / (M * M), ab = rem - end * M * M;
      const int node = (end ? N : 0) * stride[d] + (ab % M) * s1 + (ab / M) * s2;
      const int loc = el * Np + node;
      const int nnode = node + (end ? -N : N) * stride[d];
      const int enb = sNb[el][2 * d + end];  // < 0: box boundary, -DG_BC_* code
      const size_t gP = enb >= 0 ? (size_t)enb * Np + nnode : base + loc;
      double qp[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) qp[v] = q[v * KNp + gP];
      double irp, pp;
      if (enb >= 0) {
        irp = prim[gP];
        pp = prim[KNp + gP];
      } else {  // exterior values w(q+) of the ghost state
        hex_ghost(-enb, d, geo, qp);
        irp = rcp_nr(qp[0]);
        pp = gm1 * (qp[4] - 0.5 * irp * (qp[1] * qp[1] + qp[2] * qp[2] + qp[3] * qp[3]));
      }
      const double wp[5] = {qp[0], qp[1], qp[2], qp[3], pp * irp * iR};
      const double lf = end ? geo.lf[d][1] : geo.lf[d][0];
      const double sgnlf = end ? lf : -lf;
#pragma unroll
      for (int v = 0; v < 5; ++v) sJ[d][v][loc] = sgnlf * (wp[v] - sW[v][loc]);
    }
  }
  __syncthreads();
  if (tid >= nn) return;
  const int el = tid / Np, node = tid - el * Np;
  const int idx[3] = {node % M, (node / M) % M, node / (M * M)};
  double g[3][5];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int line0 = el * Np + node - idx[d] * stride[d];
    const double* Drow = sD[d] + idx[d] * M;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      double acc = sJ[d][v][tid];
#pragma unroll
      for (int l = 0; l < M; ++l) acc = fma(Drow[l], sW[v][line0 + l * stride[d]], acc);
      g[d][v] = acc;
    }
  }
  const double ir = prim[base + tid];
  const double u[3] = {sW[1][tid] * ir, sW[2][tid] * ir, sW[3][tid] * ir};
  double du[3][3];  // du[i][d] = d u_i / d x_d
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int d = 0; d < 3; ++d) du[i][d] = (g[d][1 + i] - u[i] * g[d][0]) * ir;
  const double divu = du[0][0] + du[1][1] + du[2][2];
  double tau[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) tau[i][j] = mu * (du[i][j] + du[j][i]);
#pragma unroll
  for (int i = 0; i < 3; ++i) tau[i][i] -= (2.0 / 3.0) * mu * divu;
  const size_t gi = base + tid;
  fv[0 * KNp + gi] = tau[0][0];
  fv[1 * KNp + gi] = tau[1][1];
  fv[2 * KNp + gi] = tau[2][2];
  fv[3 * KNp + gi] = tau[0][1];
  fv[4 * KNp + gi] = tau[0][2];
  fv[5 * KNp + gi] = tau[1][2];
#pragma unroll
  for (int d = 0; d < 3; ++d)
    fv[(6 + d) * KNp + gi] = fma(u[0], tau[0][d], fma(u[1], tau[1][d], fma(u[2], tau[2][d], kappa * g[d][4])));
}

// Artificial viscosity on hexahedra (the reading of the tetrahedral path on tensor-product
// elements).  Indicator of the density per element: the GLL-weighted energy of its Legendre
// modes with an index equal to N over its total energy; the transform to the coefficients is the
// 1-D matrix T[a][i] = w_i L_a(x_i) / |L_a|^2 along each axis (sum factorisation).
struct HexAv {
  double T[25];    // [M][M], row a
  double nrm[5];   // |L_a|^2 in the GLL-weighted inner product
  double eps0, s0, kappa;
};

template <int N>
__global__ void __launch_bounds__(HexCfg<N>::NT) hex_av_sensor_kernel(const double* __restrict__ q,
                                                                       const HexAv av, const int64_t K,
                                                                       double* __restrict__ eps) {
  using C = HexCfg<N>;
  constexpr int M = C::M, Np = C::Np, EPB = C::EPB, NODES = C::NODES;
  __shared__ double sA[NODES], sB[NODES];
  const int tid = threadIdx.x;
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  const int nel = (int)min((int64_t)EPB, K - e0);
  const int nn = nel * Np;
  const size_t base = (size_t)e0 * Np;
  if (tid < nn) sA[tid] = q[base + tid];  // density
  __syncthreads();
  // three passes: index i (x) -> a, j (y) -> b, k (z) -> c; node index i + M (j + M k)
  constexpr int stride[3] = {1, M, M * M};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double* src = (d & 1) ? sB : sA;
    double* dst = (d & 1) ? sA : sB;
    if (tid < nn) {
      const int el = tid / Np, node = tid - el * Np;
      const int id = (node / stride[d]) % M;
      const int line0 = el * Np + node - id * stride[d];
      double c = 0.0;
#pragma unroll
      for (int l = 0; l < M; ++l) c = fma(av.T[id * M + l], src[line0 + l * stride[d]], c);
      dst[tid] = c;
    }
    __syncthreads();
  }
  // coefficients are in sB (three passes: A -> B -> A -> B)
  if (tid < nel) {
    double num = 0.0, den = 0.0;
    for (int m = 0; m < Np; ++m) {
      const int ia = m % M, ib = (m / M) % M, ic = m / (M * M);
      const double c = sB[tid * Np + m];
      const double en = c * c * av.nrm[ia] * av.nrm[ib] * av.nrm[ic];
      den += en;
      if (ia == N || ib == N || ic == N) num += en;
    }
    double e = 0.0;
    if (num > 0.0 && den > 0.0) {
      const double sv = log10(num / den);
      if (sv > av.s0 + av.kappa)
        e = av.eps0;
      else if (sv >= av.s0 - av.kappa)
        e = 0.5 * av.eps0 * (1.0 + sin(3.141592653589793 * (sv - av.s0) / (2.0 * av.kappa)));
    }
    eps[e0 + tid] = e;
  }
}

// BR1 gradient of the conserved variables (exterior values: the ghost state at box-boundary
// faces) times the element viscosity, into sig [(5 d + v)][K][Np]; blocks whose elements all have
// eps = 0 return at once (the right-hand side reads sig only where eps > 0).
template <int N>
__global__ void __launch_bounds__(HexCfg<N>::NT) hex_av_flux_kernel(const double* __restrict__ q,
                                                                     const double* __restrict__ eps,
                                                                     double* __restrict__ sig,
                                                                     const double* __restrict__ D_g,
                                                                     const HexGeo geo, const int64_t K) {
  using C = HexCfg<N>;
  constexpr int M = C::M, Np = C::Np, EPB = C::EPB, NODES = C::NODES, NT = C::NT;
  __shared__ double sD[3][M * M];
  __shared__ double sW[5][NODES];
  __shared__ double sJ[3][5][NODES];
  __shared__ int sNb[EPB][6];
  const int tid = threadIdx.x;
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  const int nel = (int)min((int64_t)EPB, K - e0);
  if (!__syncthreads_or(tid < nel && eps[e0 + tid] > 0.0)) return;
#pragma unroll
  for (int d = 0; d < 3; ++d)
    for (int i = tid; i < M * M; i += NT) sD[d][i] = -geo.dsc[d] * D_g[i];
  const int nn = nel * Np;
  const size_t KNp = (size_t)K * Np;
  const size_t base = (size_t)e0 * Np;
  if (tid < nel) hex_neighbours((unsigned)(e0 + tid), geo.n, sNb[tid], geo.bc);
  if (tid < nn) {
#pragma unroll
    for (int v = 0; v < 5; ++v) sW[v][tid] = q[v * KNp + base + tid];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int v = 0; v < 5; ++v) sJ[d][v][tid] = 0.0;
  }
  __syncthreads();
  constexpr int FPA = 2 * M * M;
  constexpr int stride[3] = {1, M, M * M};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int s1 = stride[(d + 1) % 3], s2 = stride[(d + 2) % 3];
    for (int w = tid; w < nel * FPA; w += NT) {
      const int el = w / FPA, rem = w - el * FPA, end = rem / (M * M), ab = rem - end * M * M;
      const int node = (end ? N : 0) * stride[d] + (ab % M) * s1 + (ab / M) * s2;
      const int loc = el * Np + node;
      const int nnode = node + (end ? -N : N) * stride[d];
      const int enb = sNb[el][2 * d + end];
      const size_t gP = enb >= 0 ? (size_t)enb * Np + nnode : base + loc;
      double qp[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) qp[v] = q[v * KNp + gP];
      if (enb < 0) hex_ghost(-enb, d, geo, qp);
      const double lf = end ? geo.lf[d][1] : geo.lf[d][0];
      const double sgnlf = end ? lf : -lf;
#pragma unroll
      for (int v = 0; v < 5; ++v) sJ[d][v][loc] = sgnlf * (qp[v] - sW[v][loc]);
    }
  }
  __syncthreads();
  if (tid >= nn) return;
  const int el = tid / Np, node = tid - el * Np;
  const double ee = eps[e0 + el];
  if (!(ee > 0.0)) return;
  const int idx[3] = {node % M, (node / M) % M, node / (M * M)};
  const size_t gi = base + tid;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int line0 = el * Np + node - idx[d] * stride[d];
    const double* Drow = sD[d] + idx[d] * M;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      double acc = sJ[d][v][tid];
#pragma unroll
      for (int l = 0; l < M; ++l) acc = fma(Drow[l], sW[v][line0 + l * stride[d]], acc);
      sig[(5 * d + v) * KNp + gi] = ee * acc;
    }
  }
}

// Over-integration (weak form; the paper names it among the stabilisations of its shock cases,
// Sec. 5.3): the volume integral of grad(phi_i) . F(q_h) with Q = ceil(3 (N+1) / 2) Gauss-Legendre
// points per axis,
//   rhs_vol = sum_d (2/h_d) (A_d (x) B (x) B) F_d(I q),
// I [Q][M] the interpolation from the nodes to the Gauss points, A = W^-1 (I D)^T W_Q along d,
// B = W^-1 I^T W_Q along the other axes; the face terms are the collocated weak-form ones,
// -(2/h_d)/w_end n.F*.  Everything per element stays in shared memory: the interpolated state
// (three passes), each direction's fluxes at the Gauss points and their three contractions.
template <int N, bool VISC = false, bool AV = false>
struct OiCfg {
  static constexpr int M = N + 1, Q = (3 * (N + 1) + 1) / 2, Np = M * M * M;
  static constexpr int EPB = N == 1 ? 16 : (N == 2 ? 4 : (N == 3 ? 2 : 1));
  static constexpr int NT = 256;
  // doubles per element: nodal state, x-, y- and z-interpolated state, fluxes, volume and face terms;
  // VISC or AV: the nodal diffusive flux (viscous and artificial) of one direction, five rows
  static constexpr int PER = 5 * (Np + M * M * Q + M * Q * Q + 2 * Q * Q * Q + 2 * Np) + (VISC || AV ? 5 * Np : 0);
  static constexpr size_t SMEM = sizeof(double) * PER * EPB + sizeof(int) * 6 * EPB;
};

struct HexOI {
  double I[40];   // [Q][M]
  double A[40];   // [M][Q]
  double B[40];   // [M][Q]
  double An[25];  // [M][M]: A I = W^-1 D^T M_e, exact for a degree-N nodal field (Q >= N + 1)
  double Bn[25];  // [M][M]: B I = W^-1 M_e
};

template <int N, bool RK, bool VISC, bool AV>
__global__ void __launch_bounds__(OiCfg<N, VISC, AV>::NT) hex_oi_kernel(const double* __restrict__ q, double* __restrict__ out,
                                                               double* __restrict__ kreg, const HexGeo geo,
                                                               const HexOI op, const int64_t K, const double gamma,
                                                               const double a, const double b, const int accumulate,
                                                               unsigned* __restrict__ status, const double* __restrict__ fv,
                                                               const double* __restrict__ sig, const double* __restrict__ eps) {
  using C = OiCfg<N, VISC, AV>;
  constexpr bool DIF = VISC || AV;  // a diffusive flux (viscous, artificial or both) joins F
  constexpr int M = C::M, Q = C::Q, Np = C::Np, EPB = C::EPB, NT = C::NT;
  constexpr int M2 = M * M, Q2 = Q * Q, Q3 = Q * Q * Q;
  extern __shared__ double sm[];
  double* sq = sm;                      // [5][EPB][Np]
  double* sA = sq + 5 * EPB * Np;       // [5][EPB][M][M][Q]  (x interpolated)   / [5][EPB][Q][M][M] later
  double* sB = sA + 5 * EPB * M2 * Q;   // [5][EPB][M][Q][Q]  (x, y interpolated)/ [5][EPB][Q][Q][M] later
  double* sC = sB + 5 * EPB * M * Q2;   // [5][EPB][Q][Q][Q]  state at the Gauss points
  double* sF = sC + 5 * EPB * Q3;       // [5][EPB][Q][Q][Q]  flux along d at the Gauss points
  double* acc = sF + 5 * EPB * Q3;      // [5][EPB][Np]       volume term
  double* sS = acc + 5 * EPB * Np;      // [5][EPB][Np]       face terms
  double* sFvN = sS + 5 * EPB * Np;     // DIF: [5][EPB][Np] the nodal diffusive flux along d, row by row
  int(*sNb)[6] = reinterpret_cast<int(*)[6]>(sFvN + (DIF ? 5 * EPB * Np : 0));
  const int tid = threadIdx.x;
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  const int nel = (int)min((int64_t)EPB, K - e0);
  const int nn = nel * Np;
  const size_t KNp = (size_t)K * Np;
  const size_t base = (size_t)e0 * Np;
  if (tid < nel) hex_neighbours((unsigned)(e0 + tid), geo.n, sNb[tid], geo.bc);
  for (int t = tid; t < 5 * nn; t += NT) {
    const int v = t / nn, i = t - v * nn;
    sq[v * EPB * Np + i] = q[v * KNp + base + i];
    acc[v * EPB * Np + i] = 0.0;
    sS[v * EPB * Np + i] = 0.0;
  }
  __syncthreads();
  // interpolation to the Gauss points: along x, then y, then z
  for (int t = tid; t < 5 * nel * M2 * Q; t += NT) {
    const int v = t / (nel * M2 * Q), r = t - v * nel * M2 * Q, el = r / (M2 * Q), s2 = r - el * M2 * Q;
    const int kj = s2 / Q, qa = s2 - kj * Q;  // kj = k M + j
    const double* src = sq + v * EPB * Np + el * Np + kj * M;
    double c = 0.0;
#pragma unroll
    for (int i = 0; i < M; ++i) c = fma(op.I[qa * M + i], src[i], c);
    sA[v * EPB * M2 * Q + el * M2 * Q + s2] = c;
  }
  __syncthreads();
  for (int t = tid; t < 5 * nel * M * Q2; t += NT) {
    const int v = t / (nel * M * Q2), r = t - v * nel * M * Q2, el = r / (M * Q2), s2 = r - el * M * Q2;
    const int k = s2 / Q2, qb = (s2 / Q) % Q, qa = s2 % Q;
    const double* src = sA + v * EPB * M2 * Q + el * M2 * Q + k * M * Q + qa;
    double c = 0.0;
#pragma unroll
    for (int j = 0; j < M; ++j) c = fma(op.I[qb * M + j], src[j * Q], c);
    sB[v * EPB * M * Q2 + el * M * Q2 + s2] = c;
  }
  __syncthreads();
  for (int t = tid; t < 5 * nel * Q3; t += NT) {
    const int v = t / (nel * Q3), r = t - v * nel * Q3, el = r / Q3, s2 = r - el * Q3;
    const int qc = s2 / Q2, qba = s2 - qc * Q2;
    const double* src = sB + v * EPB * M * Q2 + el * M * Q2 + qba;
    double c = 0.0;
#pragma unroll
    for (int k = 0; k < M; ++k) c = fma(op.I[qc * M + k], src[k * Q2], c);
    sC[v * EPB * Q3 + el * Q3 + s2] = c;
  }
  __syncthreads();
  const double gm1 = gamma - 1.0;
  // 1/rho and p at this thread's Gauss points, once for the three flux directions (a thread
  // handles the same Gauss points in every direction's pass)
  constexpr int GPT = (EPB * Q3 + NT - 1) / NT;
  double g_ir[GPT], g_p[GPT];
#pragma unroll
  for (int s = 0; s < GPT; ++s) {
    const int t = tid + s * NT;
    g_ir[s] = g_p[s] = 0.0;
    if (t < nel * Q3) {
      const double r = sC[t], mx = sC[EPB * Q3 + t], my = sC[2 * EPB * Q3 + t], mz = sC[3 * EPB * Q3 + t];
      g_ir[s] = rcp_nr(r);
      g_p[s] = gm1 * (sC[4 * EPB * Q3 + t] - 0.5 * g_ir[s] * (mx * mx + my * my + mz * mz));
      if (!(r > 0.0) || !(g_p[s] > 0.0)) atomicOr(status, DG_STATUS_NONPHYSICAL);
    }
  }
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    if constexpr (DIF) {
      // the diffusive flux along d, row v: the viscous tau_(v-1)d or Q_d (VISC) plus the artificial
      // sigma_dv where the element has eps > 0 (AV).  A degree-N nodal field is its own interpolant
      // and the Q >= N + 1 Gauss points integrate its products with the test functions exactly, so
      // its part of the volume term is (A I) (x) (B I) (x) (B I) on the nodes: three M x M passes
      // through the sA and sB scratch instead of interpolating it to the Q^3 points.
      for (int t = tid; t < 5 * nn; t += NT) {
        const int v = t / nn, r = t - v * nn;
        double f = 0.0;
        if (VISC && v > 0) f = fv[(v < 4 ? hex_tau(v - 1, d) : 6 + d) * KNp + base + r];
        if (AV && eps[e0 + r / Np] > 0.0) f += sig[(5 * d + v) * KNp + base + r];
        sFvN[v * EPB * Np + r] = f;
      }
      __syncthreads();
      const double* Xn = d == 0 ? op.An : op.Bn;
      const double* Yn = d == 1 ? op.An : op.Bn;
      const double* Zn = d == 2 ? op.An : op.Bn;
      for (int t = tid; t < 5 * nn; t += NT) {  // along x: node (k M + j) M + i
        const int v = t / nn, r = t - v * nn, el = r / Np, node = r - el * Np;
        const int i = node % M, kj = node / M;
        const double* src = sFvN + v * EPB * Np + el * Np + kj * M;
        double c = 0.0;
#pragma unroll
        for (int x = 0; x < M; ++x) c = fma(Xn[i * M + x], src[x], c);
        sA[v * EPB * Np + r] = c;
      }
      __syncthreads();
      for (int t = tid; t < 5 * nn; t += NT) {  // along y
        const int v = t / nn, r = t - v * nn, el = r / Np, node = r - el * Np;
        const int k = node / M2, j = (node / M) % M, i = node % M;
        const double* src = sA + v * EPB * Np + el * Np + k * M2 + i;
        double c = 0.0;
#pragma unroll
        for (int x = 0; x < M; ++x) c = fma(Yn[j * M + x], src[x * M], c);
        sB[v * EPB * Np + r] = c;
      }
      __syncthreads();
      const double fac = -geo.dsc[d];
      for (int t = tid; t < 5 * nn; t += NT) {  // along z, subtracted from the volume term (G = F - Fd)
        const int v = t / nn, r = t - v * nn, el = r / Np, node = r - el * Np;
        const int k = node / M2, ji = node - k * M2;
        const double* src = sB + v * EPB * Np + el * Np + ji;
        double c = 0.0;
#pragma unroll
        for (int x = 0; x < M; ++x) c = fma(Zn[k * M + x], src[x * M2], c);
        acc[v * EPB * Np + r] = fma(-fac, c, acc[v * EPB * Np + r]);
      }
      __syncthreads();
    }
    // fluxes along d at the Gauss points
#pragma unroll
    for (int s = 0; s < GPT; ++s) {
      const int t = tid + s * NT;
      if (t >= nel * Q3) break;
      double qv[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) qv[v] = sC[v * EPB * Q3 + t];
      const double ir = g_ir[s], p = g_p[s];
      const double md = d == 0 ? qv[1] : (d == 1 ? qv[2] : qv[3]);  // a select: qv stays in registers
      const double ud = md * ir;
      sF[0 * EPB * Q3 + t] = md;
      sF[1 * EPB * Q3 + t] = qv[1] * ud + (d == 0 ? p : 0.0);
      sF[2 * EPB * Q3 + t] = qv[2] * ud + (d == 1 ? p : 0.0);
      sF[3 * EPB * Q3 + t] = qv[3] * ud + (d == 2 ? p : 0.0);
      sF[4 * EPB * Q3 + t] = ud * (qv[4] + p);
    }
    __syncthreads();
    // contraction along x: [Q][Q][Q] -> [Q][Q][M] (into the sB region)
    const double* Mx = d == 0 ? op.A : op.B;
    const double* My = d == 1 ? op.A : op.B;
    const double* Mz = d == 2 ? op.A : op.B;
    for (int t = tid; t < 5 * nel * Q2 * M; t += NT) {
      const int v = t / (nel * Q2 * M), r = t - v * nel * Q2 * M, el = r / (Q2 * M), s2 = r - el * Q2 * M;
      const int cb = s2 / M, i = s2 - cb * M;  // cb = qc Q + qb
      const double* src = sF + v * EPB * Q3 + el * Q3 + cb * Q;
      double c = 0.0;
#pragma unroll
      for (int qa = 0; qa < Q; ++qa) c = fma(Mx[i * Q + qa], src[qa], c);
      sB[v * EPB * M * Q2 + el * M * Q2 + s2] = c;
    }
    __syncthreads();
    // along y: [Q][Q][M] -> [Q][M][M] (into the sA region)
    for (int t = tid; t < 5 * nel * Q * M2; t += NT) {
      const int v = t / (nel * Q * M2), r = t - v * nel * Q * M2, el = r / (Q * M2), s2 = r - el * Q * M2;
      const int qc = s2 / M2, j = (s2 / M) % M, i = s2 % M;
      const double* src = sB + v * EPB * M * Q2 + el * M * Q2 + qc * Q * M + i;
      double c = 0.0;
#pragma unroll
      for (int qb = 0; qb < Q; ++qb) c = fma(My[j * Q + qb], src[qb * M], c);
      sA[v * EPB * M2 * Q + el * M2 * Q + s2] = c;
    }
    __syncthreads();
    // along z: [Q][M][M] -> [M][M][M], added to the volume term with the factor (2/h_d) s
    const double fac = -geo.dsc[d];
    for (int t = tid; t < 5 * nn; t += NT) {
      const int v = t / nn, r = t - v * nn, el = r / Np, node = r - el * Np;
      const int k = node / M2, ji = node - k * M2;
      const double* src = sA + v * EPB * M2 * Q + el * M2 * Q + ji;
      double c = 0.0;
#pragma unroll
      for (int qc = 0; qc < Q; ++qc) c = fma(Mz[k * Q + qc], src[qc * M2], c);
      acc[v * EPB * Np + r] = fma(fac, c, acc[v * EPB * Np + r]);
    }
    __syncthreads();
  }
  // weak-form face terms -(2/h_d)/w_end n.F* (times s), one axis per pass
  constexpr int FPA = 2 * M * M;
  constexpr int stride[3] = {1, M, M * M};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int s1 = stride[(d + 1) % 3], s2 = stride[(d + 2) % 3];
    for (int w = tid; w < nel * FPA; w += NT) {
      const int el = w / FPA, rem = w - el * FPA, end = rem / (M * M), ab = rem - end * M * M;
      const int node = (end ? N : 0) * stride[d] + (ab % M) * s1 + (ab / M) * s2;
      const int loc = el * Np + node;
      const int nnode = node + (end ? -N : N) * stride[d];
      const int enb = sNb[el][2 * d + end];
      const size_t gP = enb >= 0 ? (size_t)enb * Np + nnode : base + loc;
      double qm[5], qp[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        qm[v] = sq[v * EPB * Np + loc];
        qp[v] = q[v * KNp + gP];
      }
      if (enb < 0) hex_ghost(-enb, d, geo, qp);
      double irm, pm, cm, irp, pp, cp;
      pc(gamma, qm, irm, pm, cm);
      pc(gamma, qp, irp, pp, cp);
      if (enb < 0 && (!(qp[0] > 0.0) || !(pp > 0.0))) atomicOr(status, DG_STATUS_NONPHYSICAL);
      const double um = qm[1 + d] * irm, up = qp[1 + d] * irp;
      const double lam = fmax(fabs(um) + cm, fabs(up) + cp);
      double fm[5], fp[5];
      fm[0] = qm[1 + d];
      fp[0] = qp[1 + d];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        fm[1 + i] = qm[1 + i] * um;
        fp[1 + i] = qp[1 + i] * up;
      }
      fm[1 + d] += pm;
      fp[1 + d] += pp;
      fm[4] = um * (qm[4] + pm);
      fp[4] = up * (qp[4] + pp);
      if constexpr (VISC) {  // G_d = F_d - Fv_d on both traces: the central viscous flux
        const size_t gM = base + loc;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          fm[1 + i] -= fv[hex_tau(i, d) * KNp + gM];
          fp[1 + i] -= fv[hex_tau(i, d) * KNp + gP];
        }
        fm[4] -= fv[(6 + d) * KNp + gM];
        fp[4] -= fv[(6 + d) * KNp + gP];
        // at a box boundary gP is the node itself: walls are adiabatic (E_d+ = -E_d-) and a slip
        // wall is shear-free (tau_id+ = -tau_id- for i != d)
        if (enb == -DG_BC_SLIP_WALL || enb == -DG_BC_NOSLIP_WALL) {
          fp[4] += 2.0 * fv[(6 + d) * KNp + gM];
          if (enb == -DG_BC_SLIP_WALL)
#pragma unroll
            for (int i = 0; i < 3; ++i)
              if (i != d) fp[1 + i] += 2.0 * fv[hex_tau(i, d) * KNp + gM];
        }
      }
      if constexpr (AV) {  // the central AV flux; at a box boundary the exterior flux is the interior one
        const size_t gM = base + loc;
        const bool onM = eps[e0 + el] > 0.0, onP = enb >= 0 ? eps[enb] > 0.0 : onM;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          if (onM) fm[v] -= sig[(5 * d + v) * KNp + gM];
          if (onP) fp[v] -= sig[(5 * d + v) * KNp + gP];
        }
      }
      // -(2/h_d)/w_end n.G* = -(sgn (G_d- + G_d+) + lam (q- - q+)) (2/h_d)/w_end / 2 (times s)
      const double lf = end ? geo.lf[d][1] : geo.lf[d][0];
      const double sgnlf = end ? lf : -lf;
#pragma unroll
      for (int v = 0; v < 5; ++v)
        sS[v * EPB * Np + loc] -= fma(sgnlf, fm[v] + fp[v], lf * lam * (qm[v] - qp[v]));
    }
    __syncthreads();
  }
  for (int t = tid; t < 5 * nn; t += NT) {
    const int v = t / nn, r = t - v * nn;
    const double rv = acc[v * EPB * Np + r] + sS[v * EPB * Np + r];  // s rhs
    const size_t gi = v * KNp + base + r;
    if (RK) {
      const double kk = accumulate ? fma(a, kreg[gi], rv) : rv;
      kreg[gi] = kk;
      out[gi] = fma(b, kk, sq[v * EPB * Np + r]);
    } else {
      out[gi] = rv;
    }
  }
}

// Scalar advection du/dt + a . grad u = 0 (the paper's GPU comparison workload, Sec. 5.2): F_d = a_d u
// and the Lax-Friedrichs flux with lambda = |a . n|, i.e. the upwind flux, so that a face adds
//   (2/h_d)/w_end (n.F- - n.F*) = (2/h_d)/w_end (s a_d - |a_d|)/2 (u- - u+),  s = -1 (end 0), +1 (end 1),
// which vanishes on outflow faces: per axis only the inflow face of an element contributes.
// As for the Euler kernel, the stage's dt (s) is folded into the coefficients.
struct AdvCoef {
  int n[3];
  int inflow;         // bit 2d + end set where face[d][end] != 0 (tested on the integer pipe)
  double dsc[3];      // -a_d (2/h_d) s
  double face[3][2];  // (2/h_d)/w_end (sgn a_d - |a_d|) s / 2, sgn = -1 (end 0), +1 (end 1)
};

template <int N, bool RK>
__global__ void __launch_bounds__(HexCfg<N>::NT) hex_adv_kernel(const double* __restrict__ u, double* __restrict__ out,
                                                                 double* __restrict__ kreg,
                                                                 const double* __restrict__ D_g, const AdvCoef cf,
                                                                 const int64_t K, const double a, const double b,
                                                                 const int accumulate) {
  using C = HexCfg<N>;
  constexpr int M = C::M, Np = C::Np, EPB = C::EPB, NODES = C::NODES, NT = C::NT;
  __shared__ double sD[3][M * M];  // -a_d (2/h_d) s D per axis
  __shared__ double sU[NODES];
  __shared__ double sS[NODES];
  __shared__ int sNb[EPB][6];
  const int tid = threadIdx.x;
#pragma unroll
  for (int d = 0; d < 3; ++d)
    for (int i = tid; i < M * M; i += NT) sD[d][i] = cf.dsc[d] * D_g[i];
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  const int nel = (int)min((int64_t)EPB, K - e0);
  const int nn = nel * Np;
  const size_t base = (size_t)e0 * Np;
  double uv = 0.0;
  if (tid < nel) hex_neighbours((unsigned)(e0 + tid), cf.n, sNb[tid]);
  if (tid < nn) {
    uv = u[base + tid];
    sU[tid] = uv;
    sS[tid] = 0.0;
  }
  __syncthreads();

  constexpr int stride[3] = {1, M, M * M};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int s1 = stride[(d + 1) % 3], s2 = stride[(d + 2) % 3];
#pragma unroll
    for (int end = 0; end < 2; ++end) {
      if (!(cf.inflow >> (2 * d + end) & 1)) continue;  // outflow face (or a_d = 0): uniform
      const double c = cf.face[d][end];
      for (int w = tid; w < nel * M * M; w += NT) {
        const int el = w / (M * M), ab = w - el * M * M;
        const int node = (end ? N : 0) * stride[d] + (ab % M) * s1 + (ab / M) * s2;
        const int loc = el * Np + node;
        const int nnode = node + (end ? -N : N) * stride[d];
        sS[loc] = fma(c, sU[loc] - u[(size_t)sNb[el][2 * d + end] * Np + nnode], sS[loc]);
      }
    }
    __syncthreads();
  }
  if (tid >= nn) return;

  const int el = tid / Np, node = tid - el * Np;
  const int idx[3] = {node % M, (node / M) % M, node / (M * M)};
  double acc = sS[tid];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int line0 = el * Np + node - idx[d] * stride[d];
    const double* Drow = sD[d] + idx[d] * M;
#pragma unroll
    for (int l = 0; l < M; ++l) acc = fma(Drow[l], sU[line0 + l * stride[d]], acc);
  }
  const size_t gi = base + tid;
  if (RK) {
    const double kk = accumulate ? fma(a, kreg[gi], acc) : acc;  // acc = dt rhs
    kreg[gi] = kk;
    out[gi] = fma(b, kk, uv);
  } else {
    out[gi] = acc;
  }
}

template <int N, bool RK>
cudaError_t launch_adv_t(const dg_hex_mesh_s& m, const double* vel, const double* u, double* out, double* k, double a,
                         double b, double dt, cudaStream_t s) {
  using C = HexCfg<N>;
  const double sc = RK ? dt : 1.0;
  AdvCoef cf;
  for (int d = 0; d < 3; ++d) {
    cf.n[d] = m.n[d];
    const double two_h = 2.0 / (m.L[d] / m.n[d]);
    cf.dsc[d] = -vel[d] * two_h * sc;
    cf.face[d][0] = two_h / m.w[0] * 0.5 * (-vel[d] - std::fabs(vel[d])) * sc;
    cf.face[d][1] = two_h / m.w[N] * 0.5 * (vel[d] - std::fabs(vel[d])) * sc;
  }
  cf.inflow = 0;
  for (int d = 0; d < 3; ++d)
    for (int end = 0; end < 2; ++end)
      if (cf.face[d][end] != 0.0) cf.inflow |= 1 << (2 * d + end);
  const int64_t blocks = (m.K + C::EPB - 1) / C::EPB;
  hex_adv_kernel<N, RK><<<(unsigned)blocks, C::NT, 0, s>>>(u, out, k, m.D_dev, cf, m.K, a, b, a != 0.0);
  return cudaGetLastError();
}

cudaError_t launch_adv(const dg_hex_mesh_s& m, const double* vel, const double* u, double* out, double* k, bool rk,
                       double a, double b, double dt, cudaStream_t s) {
  switch (m.N) {
#define DG_CASE(NN)                                                         \
  case NN:                                                                  \
    return rk ? launch_adv_t<NN, true>(m, vel, u, out, k, a, b, dt, s)      \
              : launch_adv_t<NN, false>(m, vel, u, out, k, a, b, dt, s);
    DG_CASE(1)
    DG_CASE(2)
    DG_CASE(3)
    DG_CASE(4)
#undef DG_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <int N>
HexGeo make_geo(const dg_hex_mesh_s& m, double sc) {
  HexGeo geo;
  for (int f = 0; f < 6; ++f) geo.bc[f] = m.bc[f];
  for (int v = 0; v < 5; ++v) geo.q_in[v] = m.q_in[v];
  for (int d = 0; d < 3; ++d) {
    geo.n[d] = m.n[d];
    const double two_h = 2.0 / (m.L[d] / m.n[d]);
    geo.dsc[d] = -two_h * sc;
    geo.lf[d][0] = 0.5 * two_h / m.w[0] * sc;
    geo.lf[d][1] = 0.5 * two_h / m.w[N] * sc;
  }
  return geo;
}

template <int N>
cudaError_t launch_vis_t(const dg_hex_mesh_s& m, const GasParams& g, const double* q, cudaStream_t s) {
  using C = HexCfg<N>;
  const int64_t blocks = (m.K + C::EPB - 1) / C::EPB;
  hex_vis_kernel<N><<<(unsigned)blocks, C::NT, 0, s>>>(q, m.fv_dev, m.D_dev, make_geo<N>(m, 1.0), m.K, g.gamma, g.R,
                                                       g.mu, g.kappa, m.prim);
  return cudaGetLastError();
}

template <int N>
HexAv make_av(const dg_hex_mesh_s& m) {
  HexAv av{};
  for (size_t i = 0; i < m.modal.size(); ++i) av.T[i] = m.modal[i];
  for (size_t a = 0; a < m.modal_norm.size(); ++a) av.nrm[a] = m.modal_norm[a];
  av.eps0 = m.av_eps0;
  av.s0 = m.av_s0;
  av.kappa = m.av_kappa;
  return av;
}

template <int N>
cudaError_t launch_av_sensor_t(const dg_hex_mesh_s& m, const double* q, double* eps, cudaStream_t s) {
  using C = HexCfg<N>;
  const int64_t blocks = (m.K + C::EPB - 1) / C::EPB;
  hex_av_sensor_kernel<N><<<(unsigned)blocks, C::NT, 0, s>>>(q, make_av<N>(m), m.K, eps);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_av_flux_t(const dg_hex_mesh_s& m, const double* q, cudaStream_t s) {
  using C = HexCfg<N>;
  const int64_t blocks = (m.K + C::EPB - 1) / C::EPB;
  hex_av_flux_kernel<N><<<(unsigned)blocks, C::NT, 0, s>>>(q, m.av_eps, m.av_sig, m.D_dev, make_geo<N>(m, 1.0), m.K);
  return cudaGetLastError();
}

template <int N, bool RK, bool VISC, bool AV>
cudaError_t launch_t(const dg_hex_mesh_s& m, double gamma, const double* q, double* out, double* k, double a, double b,
                     double dt, cudaStream_t s) {
  using C = HexCfg<N>;
  const HexGeo geo = make_geo<N>(m, RK ? dt : 1.0);
  const int64_t blocks = (m.K + C::EPB - 1) / C::EPB;
  hex_rhs_kernel<N, RK, VISC, AV><<<(unsigned)blocks, C::NT, 0, s>>>(q, out, k, m.D_dev, geo, m.K, gamma, a, b,
                                                                     a != 0.0, m.status, m.fv_dev, m.av_sig,
                                                                     m.av_eps, m.prim);
  return cudaGetLastError();
}

template <int N, bool VISC, bool AV>
cudaError_t launch_rk(const dg_hex_mesh_s& m, const GasParams& g, const double* q, double* out, double* k, bool rk,
                      double a, double b, double dt, cudaStream_t s) {
  return rk ? launch_t<N, true, VISC, AV>(m, g.gamma, q, out, k, a, b, dt, s)
            : launch_t<N, false, VISC, AV>(m, g.gamma, q, out, k, a, b, dt, s);
}

template <int N, bool RK, bool VISC, bool AV>
cudaError_t launch_oi_t(const dg_hex_mesh_s& m, double gamma, const double* q, double* out, double* k, double a,
                        double b, double dt, cudaStream_t s) {
  using C = OiCfg<N, VISC, AV>;
  static bool configured = false;
  if (!configured) {
    const cudaError_t e = cudaFuncSetAttribute(hex_oi_kernel<N, RK, VISC, AV>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  HexOI op{};
  for (size_t i = 0; i < m.oi_I.size(); ++i) op.I[i] = m.oi_I[i];
  for (size_t i = 0; i < m.oi_A.size(); ++i) op.A[i] = m.oi_A[i];
  for (size_t i = 0; i < m.oi_B.size(); ++i) op.B[i] = m.oi_B[i];
  for (size_t i = 0; i < m.oi_An.size(); ++i) op.An[i] = m.oi_An[i];
  for (size_t i = 0; i < m.oi_Bn.size(); ++i) op.Bn[i] = m.oi_Bn[i];
  const int64_t blocks = (m.K + C::EPB - 1) / C::EPB;
  hex_oi_kernel<N, RK, VISC, AV><<<(unsigned)blocks, C::NT, C::SMEM, s>>>(
      q, out, k, make_geo<N>(m, RK ? dt : 1.0), op, m.K, gamma, a, b, a != 0.0, m.status, m.fv_dev, m.av_sig, m.av_eps);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_n(const dg_hex_mesh_s& m, const GasParams& g, const double* q, double* out, double* k, bool rk,
                     double a, double b, double dt, cudaStream_t s) {
  const bool av = m.av_eps0 > 0;
  if (m.overint && !(g.mu > 0) && !av)
    return rk ? launch_oi_t<N, true, false, false>(m, g.gamma, q, out, k, a, b, dt, s)
              : launch_oi_t<N, false, false, false>(m, g.gamma, q, out, k, a, b, dt, s);
  cudaError_t e;
  if (!m.overint || g.mu > 0) {  // the primitives of the collocated kernels and of the BR1 pass
    const int64_t n = m.K * m.Np, want = (n + 255) / 256;
    hex_prims_kernel<<<(unsigned)(want < 65535 ? want : 65535), 256, 0, s>>>(q, m.prim, n, g.gamma, m.status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (g.mu > 0 && (e = launch_vis_t<N>(m, g, q, s)) != cudaSuccess) return e;
  if (av) {
    if ((e = launch_av_sensor_t<N>(m, q, m.av_eps, s)) != cudaSuccess) return e;
    if ((e = launch_av_flux_t<N>(m, q, s)) != cudaSuccess) return e;
  }
  if (m.overint) {  // the BR1 and AV passes above, then the over-integrated right-hand side
    if (g.mu > 0)
      return av ? (rk ? launch_oi_t<N, true, true, true>(m, g.gamma, q, out, k, a, b, dt, s)
                      : launch_oi_t<N, false, true, true>(m, g.gamma, q, out, k, a, b, dt, s))
                : (rk ? launch_oi_t<N, true, true, false>(m, g.gamma, q, out, k, a, b, dt, s)
                      : launch_oi_t<N, false, true, false>(m, g.gamma, q, out, k, a, b, dt, s));
    return rk ? launch_oi_t<N, true, false, true>(m, g.gamma, q, out, k, a, b, dt, s)
              : launch_oi_t<N, false, false, true>(m, g.gamma, q, out, k, a, b, dt, s);
  }
  if (g.mu > 0)
    return av ? launch_rk<N, true, true>(m, g, q, out, k, rk, a, b, dt, s)
              : launch_rk<N, true, false>(m, g, q, out, k, rk, a, b, dt, s);
  return av ? launch_rk<N, false, true>(m, g, q, out, k, rk, a, b, dt, s)
            : launch_rk<N, false, false>(m, g, q, out, k, rk, a, b, dt, s);
}

cudaError_t launch_av_sensor(const dg_hex_mesh_s& m, const double* q, double* eps, cudaStream_t s) {
  switch (m.N) {
    case 1: return launch_av_sensor_t<1>(m, q, eps, s);
    case 2: return launch_av_sensor_t<2>(m, q, eps, s);
    case 3: return launch_av_sensor_t<3>(m, q, eps, s);
    case 4: return launch_av_sensor_t<4>(m, q, eps, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch(const dg_hex_mesh_s& m, const GasParams& g, const double* q, double* out, double* k, bool rk,
                   double a, double b, double dt, cudaStream_t s) {
  switch (m.N) {
#define DG_CASE(NN) \
  case NN:          \
    return launch_n<NN>(m, g, q, out, k, rk, a, b, dt, s);
    DG_CASE(1)
    DG_CASE(2)
    DG_CASE(3)
    DG_CASE(4)
#undef DG_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

// Quadrature weights and differentiation matrix of the Lagrange basis through the nodes, in long
// double: barycentric weights lambda_j = 1 / prod_{k != j} (x_j - x_k); D[i][j] = (lambda_j /
// lambda_i) / (x_i - x_j) off the diagonal, the diagonal from D 1 = 0; w_j = integral of l_j by
// (N+2)-point Gauss-Legendre quadrature (exact for degree <= 2N+3) of the barycentric l_j.
bool build_operators(const std::vector<double>& x, std::vector<double>& w, std::vector<double>& D, std::string& err) {
  const int m = (int)x.size();
  typedef long double ld;
  std::vector<ld> lam(m, 1.0L);
  for (int j = 0; j < m; ++j)
    for (int k = 0; k < m; ++k)
      if (k != j) {
        const ld dx = (ld)x[j] - (ld)x[k];
        if (!(dx != 0.0L)) {
          err = "repeated node in the 1-D node set";
          return false;
        }
        lam[j] /= dx;
      }
  D.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) {
    ld diag = 0.0L;
    for (int j = 0; j < m; ++j)
      if (j != i) {
        const ld dij = (lam[j] / lam[i]) / ((ld)x[i] - (ld)x[j]);
        D[(size_t)i * m + j] = (double)dij;
        diag -= dij;
      }
    D[(size_t)i * m + i] = (double)diag;
  }
  // Gauss-Legendre points and weights of order G by Newton on P_G (recurrence in long double)
  const int G = m + 1;
  std::vector<ld> gx(G), gw(G);
  const ld pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < G; ++i) {
    ld z = cosl(pi * (i + 0.75L) / (G + 0.5L));
    ld dp = 1.0L;
    for (int it = 0; it < 100; ++it) {
      ld p0 = 1.0L, p1 = z;
      for (int n = 2; n <= G; ++n) {
        const ld p2 = ((2 * n - 1) * z * p1 - (n - 1) * p0) / n;
        p0 = p1;
        p1 = p2;
      }
      dp = G * (z * p1 - p0) / (z * z - 1.0L);
      const ld dz = p1 / dp;
      z -= dz;
      if (fabsl(dz) < 1e-19L) break;
    }
    gx[i] = z;
    gw[i] = 2.0L / ((1.0L - z * z) * dp * dp);
  }
  w.assign(m, 0.0);
  for (int j = 0; j < m; ++j) {
    ld s = 0.0L;
    for (int g = 0; g < G; ++g) {
      ld l = 1.0L;
      for (int k = 0; k < m; ++k)
        if (k != j) l *= (gx[g] - (ld)x[k]) / ((ld)x[j] - (ld)x[k]);
      s += gw[g] * l;
    }
    w[j] = (double)s;
  }
  return true;
}

}  // namespace hexk
}  // namespace dg

extern "C" {

int dg_hex_mesh_create(const dg_hex_desc* d, dg_hex_mesh* out) {
  if (!d || !out) return dg::fail(DG_ERR_INVALID_ARG, "NULL descriptor or output handle");
  *out = nullptr;
  if (d->N < 1 || d->N > DG_MAX_ORDER) return dg::fail(DG_ERR_INVALID_ARG, "N must be in 1..4");
  if (!d->nodes1d) return dg::fail(DG_ERR_INVALID_ARG, "NULL 1-D node set");
  for (int k = 0; k < 3; ++k) {
    if (d->n[k] < 1) return dg::fail(DG_ERR_INVALID_ARG, "need at least one hexahedron per direction");
    if (!(d->L[k] > 0.0)) return dg::fail(DG_ERR_INVALID_ARG, "box lengths must be positive");
  }
  const int M = d->N + 1;
  std::vector<double> x(d->nodes1d, d->nodes1d + M);
  if (x[0] != -1.0 || x[M - 1] != 1.0) return dg::fail(DG_ERR_INVALID_ARG, "the node set must start at -1 and end at 1");
  for (int i = 1; i < M; ++i)
    if (!(x[i] > x[i - 1])) return dg::fail(DG_ERR_INVALID_ARG, "the node set must be ascending");
  for (int k = 0; k < 3; ++k) {
    const int a = d->bc[2 * k], b = d->bc[2 * k + 1];
    if ((a == 0) != (b == 0)) return dg::fail(DG_ERR_INVALID_ARG, "a box axis is periodic at both ends or at neither");
    for (int c : {a, b})
      if (c < 0 || c > DG_BC_OUTFLOW) return dg::fail(DG_ERR_INVALID_ARG, "unknown boundary-condition code");
  }
  dg_hex_mesh_s* m = new dg_hex_mesh_s();
  for (int k = 0; k < 3; ++k) {
    m->n[k] = d->n[k];
    m->L[k] = d->L[k];
  }
  for (int f = 0; f < 6; ++f) m->bc[f] = d->bc[f];
  m->N = d->N;
  m->M = M;
  m->Np = M * M * M;
  m->K = (int64_t)d->n[0] * d->n[1] * d->n[2];
  if (m->K > INT32_MAX) {
    delete m;
    return dg::fail(DG_ERR_INVALID_ARG, "at most 2^31 - 1 hexahedra");
  }
  m->nodes = x;
  std::string err;
  if (!dg::hexk::build_operators(x, m->w, m->D, err)) {
    delete m;
    return dg::fail(DG_ERR_INVALID_ARG, err);
  }
  {  // Legendre modal analysis at the nodes (long double recurrence), for the AV indicator
    std::vector<long double> L((size_t)M * M);  // L[a][j]
    for (int j = 0; j < M; ++j) {
      long double p0 = 1.0L, p1 = (long double)x[j];
      L[j] = p0;
      if (M > 1) L[M + j] = p1;
      for (int a = 1; a + 1 < M; ++a) {
        const long double p2 = ((2 * a + 1) * (long double)x[j] * p1 - a * p0) / (a + 1);
        L[(size_t)(a + 1) * M + j] = p2;
        p0 = p1;
        p1 = p2;
      }
    }
    m->modal.assign((size_t)M * M, 0.0);
    m->modal_norm.assign(M, 0.0);
    for (int a = 0; a < M; ++a) {
      long double nrm = 0.0L;
      for (int j = 0; j < M; ++j) nrm += (long double)m->w[j] * L[(size_t)a * M + j] * L[(size_t)a * M + j];
      m->modal_norm[a] = (double)nrm;
      for (int j = 0; j < M; ++j) m->modal[(size_t)a * M + j] = (double)((long double)m->w[j] * L[(size_t)a * M + j] / nrm);
    }
  }
  cudaError_t e = cudaMalloc((void**)&m->D_dev, sizeof(double) * M * M);
  if (e == cudaSuccess) e = cudaMemcpy(m->D_dev, m->D.data(), sizeof(double) * M * M, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->status, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(m->status, 0, sizeof(unsigned));
  if (e != cudaSuccess) {
    cudaFree(m->D_dev);
    cudaFree(m->status);
    delete m;
    return dg::cuda_fail(e, "hexahedral mesh upload");
  }
  *out = m;
  return DG_OK;
}

int dg_hex_mesh_free(dg_hex_mesh m) {
  if (!m) return DG_OK;
  cudaFree(m->D_dev);
  cudaFree(m->fv_dev);
  cudaFree(m->prim);
  cudaFree(m->av_eps);
  cudaFree(m->av_sig);
  cudaFree(m->status);
  delete m;
  return DG_OK;
}

int dg_hex_operators(dg_hex_mesh m, double* D_host, double* w_host) {
  if (!m) return dg::fail(DG_ERR_INVALID_ARG, "NULL mesh");
  if (D_host) std::copy(m->D.begin(), m->D.end(), D_host);
  if (w_host) std::copy(m->w.begin(), m->w.end(), w_host);
  return DG_OK;
}

static int hex_run(dg_hex_mesh m, dg_gas gas, const double* q, double* out, double* k, bool rk, int stage, double dt,
                   void* stream) {
  if (!m || !gas) return dg::fail(DG_ERR_INVALID_ARG, "NULL mesh or gas");
  if (!q || !out) return dg::fail(DG_ERR_INVALID_ARG, "NULL state or output");
  if (rk && !k) return dg::fail(DG_ERR_INVALID_ARG, "NULL RK register k");
  if (rk && (stage < 0 || stage > 4)) return dg::fail(DG_ERR_INVALID_ARG, "stage must be in 0..4");
  if (rk && !std::isfinite(dt)) return dg::fail(DG_ERR_INVALID_ARG, "dt must be finite");
  if (gas->p.model != DG_GAS_PERFECT)
    return dg::fail(DG_ERR_UNSUPPORTED, "the hexahedral path takes a perfect gas");
  // the primitives buffer, which the collocated kernels and the BR1 pass read (launch_n runs the
  // primitives pass under the same condition)
  if ((!m->overint || gas->p.mu > 0) && !m->prim) {
    const cudaError_t e = cudaMalloc((void**)&m->prim, sizeof(double) * 3 * (size_t)m->K * m->Np);
    if (e != cudaSuccess) return dg::cuda_fail(e, "hexahedral primitives buffer");
  }
  if (gas->p.mu > 0) {
    if (!m->fv_dev) {
      const cudaError_t e = cudaMalloc((void**)&m->fv_dev, sizeof(double) * 9 * (size_t)m->K * m->Np);
      if (e != cudaSuccess) return dg::cuda_fail(e, "hexahedral viscous-flux buffer");
    }
  }
  const size_t n = (size_t)5 * m->K * m->Np;
  if (q == out || (q < out + n && out < q + n)) return dg::fail(DG_ERR_INVALID_ARG, "output overlaps the input state");
  for (int f = 0; f < 6; ++f)
    if (m->bc[f] == DG_BC_INFLOW && !m->has_inflow)
      return dg::fail(DG_ERR_INVALID_ARG, "the box has an inflow face: set its state with dg_hex_set_inflow");
  const double a = rk ? dg::kRK4A[stage] : 0.0, b = rk ? dg::kRK4B[stage] : 0.0;
  const cudaError_t e = dg::hexk::launch(*m, gas->p, q, out, k, rk, a, b, dt, (cudaStream_t)stream);
  return e == cudaSuccess ? DG_OK : dg::cuda_fail(e, "hexahedral right-hand-side kernel");
}

int dg_hex_rhs(dg_hex_mesh m, dg_gas gas, const double* q, double* rhs, void* stream) {
  return hex_run(m, gas, q, rhs, nullptr, false, 0, 0.0, stream);
}

int dg_hex_rk_stage(dg_hex_mesh m, dg_gas gas, int32_t stage, double dt, const double* q_in, double* q_out, double* k,
                    void* stream) {
  return hex_run(m, gas, q_in, q_out, k, true, stage, dt, stream);
}

static int hex_adv_run(dg_hex_mesh m, const double* vel, const double* u, double* out, double* k, bool rk, int stage,
                       double dt, void* stream) {
  if (!m || !vel) return dg::fail(DG_ERR_INVALID_ARG, "NULL mesh or velocity");
  if (!u || !out) return dg::fail(DG_ERR_INVALID_ARG, "NULL state or output");
  if (rk && !k) return dg::fail(DG_ERR_INVALID_ARG, "NULL RK register k");
  if (rk && (stage < 0 || stage > 4)) return dg::fail(DG_ERR_INVALID_ARG, "stage must be in 0..4");
  if (rk && !std::isfinite(dt)) return dg::fail(DG_ERR_INVALID_ARG, "dt must be finite");
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(vel[d])) return dg::fail(DG_ERR_INVALID_ARG, "the velocity must be finite");
  for (int f = 0; f < 6; ++f)
    if (m->bc[f]) return dg::fail(DG_ERR_UNSUPPORTED, "the advection runs on periodic boxes");
  const size_t n = (size_t)m->K * m->Np;
  if (u == out || (u < out + n && out < u + n)) return dg::fail(DG_ERR_INVALID_ARG, "output overlaps the input state");
  const double a = rk ? dg::kRK4A[stage] : 0.0, b = rk ? dg::kRK4B[stage] : 0.0;
  const cudaError_t e = dg::hexk::launch_adv(*m, vel, u, out, k, rk, a, b, dt, (cudaStream_t)stream);
  return e == cudaSuccess ? DG_OK : dg::cuda_fail(e, "hexahedral advection kernel");
}

int dg_hex_advection_rhs(dg_hex_mesh m, const double* velocity, const double* u, double* rhs, void* stream) {
  return hex_adv_run(m, velocity, u, rhs, nullptr, false, 0, 0.0, stream);
}

int dg_hex_advection_rk_stage(dg_hex_mesh m, const double* velocity, int32_t stage, double dt, const double* u_in,
                              double* u_out, double* k, void* stream) {
  return hex_adv_run(m, velocity, u_in, u_out, k, true, stage, dt, stream);
}

int dg_hex_set_av(dg_hex_mesh m, const dg_av_params* p) {
  if (!m) return dg::fail(DG_ERR_INVALID_ARG, "NULL mesh");
  if (!p || p->eps0 == 0.0) {
    m->av_eps0 = 0.0;
    return DG_OK;
  }
  if (!(p->eps0 > 0) || !std::isfinite(p->eps0) || !std::isfinite(p->s0) || !(p->kappa > 0) ||
      !std::isfinite(p->kappa))
    return dg::fail(DG_ERR_INVALID_ARG, "need eps0 >= 0, kappa > 0, all finite");
  if (!m->av_eps) {
    cudaError_t e = cudaMalloc((void**)&m->av_eps, sizeof(double) * (size_t)m->K);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->av_sig, sizeof(double) * 15 * (size_t)m->K * m->Np);
    if (e != cudaSuccess) {
      cudaFree(m->av_eps);
      cudaFree(m->av_sig);
      m->av_eps = m->av_sig = nullptr;
      return dg::cuda_fail(e, "hexahedral artificial-viscosity scratch");
    }
  }
  m->av_eps0 = p->eps0;
  m->av_s0 = p->s0;
  m->av_kappa = p->kappa;
  return DG_OK;
}

int dg_hex_av_viscosity(dg_hex_mesh m, const double* q, double* eps, void* stream) {
  if (!m || !q || !eps) return dg::fail(DG_ERR_INVALID_ARG, "NULL mesh, state or output");
  const cudaError_t e = dg::hexk::launch_av_sensor(*m, q, eps, (cudaStream_t)stream);
  return e == cudaSuccess ? DG_OK : dg::cuda_fail(e, "hexahedral smoothness-indicator kernel");
}

int dg_hex_set_overintegration(dg_hex_mesh m, int32_t enable) {
  if (!m) return dg::fail(DG_ERR_INVALID_ARG, "NULL mesh");
  m->overint = enable != 0;
  if (!m->overint || !m->oi_I.empty()) return DG_OK;
  // Q = ceil(3 (N+1) / 2) Gauss-Legendre points (Newton on P_Q, long double), the interpolation
  // from the nodes and the two contraction matrices
  const int M = m->M, Q = (3 * M + 1) / 2;
  typedef long double ld;
  std::vector<ld> xg(Q), wg(Q);
  const ld pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < Q; ++i) {
    ld z = cosl(pi * (i + 0.75L) / (Q + 0.5L)), dp = 1.0L;
    for (int it = 0; it < 100; ++it) {
      ld p0 = 1.0L, p1 = z;
      for (int n = 2; n <= Q; ++n) {
        const ld p2 = ((2 * n - 1) * z * p1 - (n - 1) * p0) / n;
        p0 = p1;
        p1 = p2;
      }
      dp = Q * (z * p1 - p0) / (z * z - 1.0L);
      const ld dz = p1 / dp;
      z -= dz;
      if (fabsl(dz) < 1e-19L) break;
    }
    xg[i] = z;
    wg[i] = 2.0L / ((1.0L - z * z) * dp * dp);
  }
  std::vector<ld> I((size_t)Q * M, 1.0L);
  for (int g = 0; g < Q; ++g)
    for (int j = 0; j < M; ++j)
      for (int k = 0; k < M; ++k)
        if (k != j) I[(size_t)g * M + j] *= (xg[g] - (ld)m->nodes[k]) / ((ld)m->nodes[j] - (ld)m->nodes[k]);
  m->oi_I.assign((size_t)Q * M, 0.0);
  m->oi_A.assign((size_t)M * Q, 0.0);
  m->oi_B.assign((size_t)M * Q, 0.0);
  for (int g = 0; g < Q; ++g)
    for (int i = 0; i < M; ++i) {
      m->oi_I[(size_t)g * M + i] = (double)I[(size_t)g * M + i];
      ld id = 0.0L;  // (I D)[g][i]
      for (int k = 0; k < M; ++k) id += I[(size_t)g * M + k] * (ld)m->D[(size_t)k * M + i];
      m->oi_A[(size_t)i * Q + g] = (double)(id * wg[g] / (ld)m->w[i]);
      m->oi_B[(size_t)i * Q + g] = (double)(I[(size_t)g * M + i] * wg[g] / (ld)m->w[i]);
    }
  // A I and B I: the contractions of a degree-N nodal field's interpolant, M x M
  m->oi_An.assign((size_t)M * M, 0.0);
  m->oi_Bn.assign((size_t)M * M, 0.0);
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) {
      ld an = 0.0L, bn = 0.0L;
      for (int g = 0; g < Q; ++g) {
        ld id = 0.0L;
        for (int k = 0; k < M; ++k) id += I[(size_t)g * M + k] * (ld)m->D[(size_t)k * M + i];
        an += id * wg[g] * I[(size_t)g * M + j];
        bn += I[(size_t)g * M + i] * wg[g] * I[(size_t)g * M + j];
      }
      m->oi_An[(size_t)i * M + j] = (double)(an / (ld)m->w[i]);
      m->oi_Bn[(size_t)i * M + j] = (double)(bn / (ld)m->w[i]);
    }
  return DG_OK;
}

int dg_hex_set_inflow(dg_hex_mesh m, const double* q_in, int32_t nvar) {
  if (!m || !q_in) return dg::fail(DG_ERR_INVALID_ARG, "NULL mesh or inflow state");
  if (nvar != 5) return dg::fail(DG_ERR_INVALID_ARG, "the hexahedral path takes 5 conserved variables");
  for (int v = 0; v < 5; ++v)
    if (!std::isfinite(q_in[v])) return dg::fail(DG_ERR_INVALID_ARG, "the inflow state must be finite");
  if (!(q_in[0] > 0)) return dg::fail(DG_ERR_INVALID_ARG, "the inflow density must be positive");
  for (int v = 0; v < 5; ++v) m->q_in[v] = q_in[v];
  m->has_inflow = true;
  return DG_OK;
}

int dg_hex_status(dg_hex_mesh m, uint32_t* bits, int reset) {
  if (!m || !bits) return dg::fail(DG_ERR_INVALID_ARG, "NULL mesh or bits");
  cudaError_t e = cudaDeviceSynchronize();
  unsigned v = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&v, m->status, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && reset) e = cudaMemset(m->status, 0, sizeof(unsigned));
  if (e != cudaSuccess) return dg::cuda_fail(e, "hexahedral mesh status");
  *bits = v;
  return DG_OK;
}

}  // extern "C"
