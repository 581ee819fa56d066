// Navier-Stokes right-hand side of a NASA-7 mixture with species diffusion, FP64.
// The paper's solver targets viscous multi-species flows (Sec. 4-5) and names no transport
// model; the reading here: constant viscosity mu (Stokes hypothesis), heat conduction
// kappa = mu cp_mix(T, Y) / Pr, Fickian diffusion at a constant Schmidt number with the
// correction that makes the fluxes sum to zero,
//   J_k = -(mu / Sc) (grad Y_k - Y_k sum_j grad Y_j),
// and the enthalpy they carry in the heat flux q = -kappa grad T + sum_k h_k(T) J_k.  Viscous
// flux (subtracted from the Euler flux): momentum tau, energy u.tau - q, species -J_k, stored as
// [9 + 3 k + d] (tau_xx, tau_yy, tau_zz, tau_xy, tau_xz, tau_yz, E_x, E_y, E_z, then species k
// along x_d).  BR1 gradients with the central flux of w = (rho, rho u, rho v, rho w, T, Y_k).
// At a boundary face node the exterior values are those of the ghost state: the momentum
// mirrored (slip wall) or reversed (no-slip wall) with the node's own rho, T and Y; the inflow
// state with its temperature; the node's own at outflow.
#include "dg_kernels.cuh"

namespace dg {
namespace kern {

constexpr int MIXW = 5 + DG_MAX_SPECIES;  // fields of w at most

template <int N>
constexpr size_t viscous_mix_smem() {
  using O = Ord<N>;
  return sizeof(double) * (O::OPS + O::EPB * GS + MIXW * O::NODES + MIXW * O::EPB * O::NF) + sizeof(int) * O::NF;
}

template <int N>
__global__ void __launch_bounds__(Ord<N>::NT) viscous_mix_kernel(
    const double* __restrict__ q, const double* __restrict__ Tg, double* __restrict__ fv_out,
    const double* __restrict__ ops_g, const int32_t* __restrict__ fmask_g, const double* __restrict__ geo_g,
    const int32_t* __restrict__ vmapP, const GasParams gp, const BcParams bc, const int K) {
  using O = Ord<N>;
  constexpr int Np = O::Np, Nfp = O::Nfp, NF = O::NF, EPB = O::EPB, NODES = O::NODES;
  extern __shared__ double smem[];
  double* sOps = smem;
  double* sGeo = sOps + O::OPS;
  double* sW = sGeo + EPB * GS;
  double* sJ = sW + MIXW * NODES;
  int* sFm = reinterpret_cast<int*>(sJ + MIXW * EPB * NF);

  const int tid = threadIdx.x;
  const int e0 = blockIdx.x * EPB;
  const int nel = min(EPB, K - e0);
  const int nn = nel * Np;
  const int ns = gp.ns, W = 5 + ns;
  const size_t KNp = (size_t)K * Np;
  const size_t base = (size_t)e0 * Np;

  for (int i = tid; i < O::OPS; i += blockDim.x) sOps[i] = ops_g[i];
  for (int i = tid; i < NF; i += blockDim.x) sFm[i] = fmask_g[i];
  for (int i = tid; i < nel * GS; i += blockDim.x) sGeo[i] = geo_g[(size_t)e0 * GS + i];
  if (tid < nn) {
    const double rho = q[base + tid], ir = 1.0 / rho;
    sW[tid] = rho;
#pragma unroll
    for (int v = 1; v < 4; ++v) sW[v * NODES + tid] = q[v * KNp + base + tid];
    sW[4 * NODES + tid] = Tg[base + tid];
    for (int k = 0; k < ns; ++k) sW[(5 + k) * NODES + tid] = q[(5 + k) * KNp + base + tid] * ir;
  }
  __syncthreads();

  // central-flux jumps (w+ - w-) Fscale / 2 at the block's face nodes
  for (int j = tid; j < nel * NF; j += blockDim.x) {
    const int e = j / NF, m = j - e * NF, f = m / Nfp;
    const double hf = 0.5 * sGeo[e * GS + 12 + 4 * f];
    const int own = e * Np + sFm[m];
    const int Pi = vmapP[(size_t)(e0 + e) * NF + m];  // < 0: boundary face node, -DG_BC_* code
    if (Pi >= 0) {
      const size_t P = (size_t)Pi;
      const double rp = q[P], irp = 1.0 / rp;
      sJ[j] = hf * (rp - sW[own]);
#pragma unroll
      for (int v = 1; v < 4; ++v) sJ[v * EPB * NF + j] = hf * (q[v * KNp + P] - sW[v * NODES + own]);
      sJ[4 * EPB * NF + j] = hf * (Tg[P] - sW[4 * NODES + own]);
      for (int k = 0; k < ns; ++k)
        sJ[(5 + k) * EPB * NF + j] = hf * (q[(5 + k) * KNp + P] * irp - sW[(5 + k) * NODES + own]);
    } else if (-Pi == DG_BC_INFLOW) {  // the inflow state at its temperature
      const double irp = 1.0 / bc.q_in[0];
      sJ[j] = hf * (bc.q_in[0] - sW[own]);
#pragma unroll
      for (int v = 1; v < 4; ++v) sJ[v * EPB * NF + j] = hf * (bc.q_in[v] - sW[v * NODES + own]);
      sJ[4 * EPB * NF + j] = hf * (bc.T_in - sW[4 * NODES + own]);
      for (int k = 0; k < ns; ++k) sJ[(5 + k) * EPB * NF + j] = hf * (bc.q_in[5 + k] * irp - sW[(5 + k) * NODES + own]);
    } else {  // walls and outflow: rho, T and Y jump by nothing; the momentum by its ghost's
      const double* G = sGeo + e * GS;
      const double n3[3] = {G[9 + 4 * f], G[10 + 4 * f], G[11 + 4 * f]};
      const double m3[3] = {sW[NODES + own], sW[2 * NODES + own], sW[3 * NODES + own]};
      const double mn = m3[0] * n3[0] + m3[1] * n3[1] + m3[2] * n3[2];
      sJ[j] = 0.0;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const double mp = -Pi == DG_BC_SLIP_WALL ? m3[i] - 2.0 * mn * n3[i] : (-Pi == DG_BC_NOSLIP_WALL ? -m3[i] : m3[i]);
        sJ[(1 + i) * EPB * NF + j] = hf * (mp - m3[i]);
      }
      sJ[4 * EPB * NF + j] = 0.0;
      for (int k = 0; k < ns; ++k) sJ[(5 + k) * EPB * NF + j] = 0.0;
    }
  }
  __syncthreads();

  if (tid < nn) {
    const int e = tid / Np, i = tid - e * Np;
    const double* G = sGeo + e * GS;
    const double* Dr = sOps + i * Np;
    const double* Ds = sOps + Np * Np + i * Np;
    const double* Dt = sOps + 2 * Np * Np + i * Np;
    const double* L = sOps + 3 * Np * Np + i * NF;
    // grad[d][v] = sum_a (dr_a/dx_d) D_a w_v + sum_f n_d,f LIFT_f jump_v
    double grad[3][MIXW];
#pragma unroll
    for (int v = 0; v < MIXW; ++v) {
      if (v >= W) break;
      double dr = 0.0, ds = 0.0, dt = 0.0;
#pragma unroll 4
      for (int jn = 0; jn < Np; ++jn) {
        const double w = sW[v * NODES + e * Np + jn];
        dr = fma(Dr[jn], w, dr);
        ds = fma(Ds[jn], w, ds);
        dt = fma(Dt[jn], w, dt);
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) grad[d][v] = fma(G[d], dr, fma(G[3 + d], ds, G[6 + d] * dt));
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        double lf = 0.0;
#pragma unroll 5
        for (int jj = 0; jj < Nfp; ++jj) lf = fma(L[f * Nfp + jj], sJ[v * EPB * NF + e * NF + f * Nfp + jj], lf);
#pragma unroll
        for (int d = 0; d < 3; ++d) grad[d][v] = fma(G[9 + 4 * f + d], lf, grad[d][v]);
      }
    }
    const double rho = sW[tid], ir = 1.0 / rho, T = sW[4 * NODES + tid];
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
    double Y[DG_MAX_SPECIES];
#pragma unroll
    for (int k = 0; k < DG_MAX_SPECIES; ++k) Y[k] = k < ns ? sW[(5 + k) * NODES + tid] : 0.0;
    double cp, Rmix;
    mixture_cp_R(gp, Y, T, cp, Rmix);
    const double kappa = mu * cp / gp.Pr, rD = mu / gp.Sc;
    const size_t gi = base + tid;
    fv_out[0 * KNp + gi] = tau[0][0];
    fv_out[1 * KNp + gi] = tau[1][1];
    fv_out[2 * KNp + gi] = tau[2][2];
    fv_out[3 * KNp + gi] = tau[0][1];
    fv_out[4 * KNp + gi] = tau[0][2];
    fv_out[5 * KNp + gi] = tau[1][2];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double sg = 0.0;  // sum_j d Y_j / d x_d
      for (int k = 0; k < ns; ++k) sg += grad[d][5 + k];
      double hJ = 0.0;  // sum_k h_k J_k along x_d
      for (int k = 0; k < ns; ++k) {
        const double* a = gp.a[k];
        const double hk =
            gp.Rk[k] * (T * (a[0] + T * (a[1] / 2 + T * (a[2] / 3 + T * (a[3] / 4 + T * (a[4] / 5))))) + a[5]);
        const double Jk = -rD * (grad[d][5 + k] - Y[k] * sg);
        hJ = fma(hk, Jk, hJ);
        fv_out[(9 + 3 * k + d) * KNp + gi] = -Jk;
      }
      fv_out[(6 + d) * KNp + gi] =
          fma(u[0], tau[0][d], fma(u[1], tau[1][d], fma(u[2], tau[2][d], kappa * grad[d][4]))) - hJ;
    }
  }
}

template <int N>
cudaError_t launch_visc_mix_t(const MeshDev& m, const GasParams& g, const double* q, const double* T,
                              cudaStream_t s) {
  using O = Ord<N>;
  constexpr size_t smem = viscous_mix_smem<N>();
  static bool configured = false;
  if (!configured) {
    cudaError_t e =
        cudaFuncSetAttribute(viscous_mix_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int blocks = (m.K + O::EPB - 1) / O::EPB;
  viscous_mix_kernel<N><<<blocks, O::NT, smem, s>>>(q, T, m.mix_fv, m.ops, m.fmask, m.geo, m.vmapP, g, m.bc, m.K);
  return cudaGetLastError();
}

}  // namespace kern

cudaError_t launch_viscous_mixture(const MeshDev& m, const GasParams& g, const double* q, const double* T,
                                   cudaStream_t s) {
  switch (m.N) {
    case 1: return kern::launch_visc_mix_t<1>(m, g, q, T, s);
    case 2: return kern::launch_visc_mix_t<2>(m, g, q, T, s);
    case 3: return kern::launch_visc_mix_t<3>(m, g, q, T, s);
    case 4: return kern::launch_visc_mix_t<4>(m, g, q, T, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_rhs_mixture_ns(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k,
                                  const double* T, bool rk, double a, double b, double dt, cudaStream_t s) {
  return kern::dispatch_rhs<5 + DG_MAX_SPECIES, kern::MIXTURE_NS>(m, g, q, out, k, T, rk, a, b, dt, s);
}

}  // namespace dg
