// Mixed-precision path: the per-case view of a mesh's tables and the primitives pass launcher
// (the tensor-core kernels are in k_tc.cu).
#include <algorithm>
#include <vector>

#include "dg_mixed.cuh"

namespace dg {

void free_mixed_ops(MeshDev& m) {
  cudaFree(m.mx.tc_rhs);
  cudaFree(m.mx.tc_vis);
  m.mx = MixedOps();
}

mixk::MixedCase make_mixed_case(const MeshDev& m, const GasParams& g, const double* qin, double* out, double* k,
                                double dt) {
  mixk::MixedCase c{};
  c.q[0] = const_cast<double*>(qin);
  c.q[1] = out;
  c.k = k;
  if (g.model == DG_GAS_NASA7) {
    c.mrec = mixk::mixture_records(m.scratch);
    c.mlo = mixk::mixture_lo(m.scratch, (size_t)m.K * m.Np);
  } else {
    const mixk::NodeTables t = mixk::node_tables(m.scratch, (size_t)m.K * m.Np);
    c.node = t.node;
    c.fv4 = t.fv4;
    c.fvz = t.fvz;
    c.temp = t.temp;
  }
  c.nvar = 5 + g.ns;
  c.geo = m.geo32;
  c.vmapP = m.vmapP;
  c.K = m.K;
  c.Np = m.Np;
  c.dt = dt;
  c.gas = mixk::MixedGas{g.gamma, g.R, g.mu, g.kappa, 1.0 / g.R};
  c.av_eps = m.av.eps0 > 0 ? m.av_eps : nullptr;
  c.av_sig = m.av.eps0 > 0 ? m.av_sig : nullptr;
  if (m.inflow_nvar == 5 && g.model == DG_GAS_PERFECT) {  // the inflow state as a node record
    const double* qi = m.bc.q_in;
    const double ke = 0.5 * (qi[1] * qi[1] + qi[2] * qi[2] + qi[3] * qi[3]) / qi[0];
    const double p = (g.gamma - 1.0) * (qi[4] - ke), T = p / (qi[0] * g.R);
    const float rho_hi = (float)qi[0], p_hi = (float)p, T_hi = (float)T;
    c.in_node[0] = make_float4(rho_hi, (float)qi[1], (float)qi[2], (float)qi[3]);
    c.in_node[1] = make_float4((float)qi[4], p_hi, (float)(p - (double)p_hi), (float)(qi[0] - (double)rho_hi));
    c.in_temp = make_float2(T_hi, (float)(T - (double)T_hi));
  }
  if (m.inflow_nvar == 5 + g.ns && g.model == DG_GAS_NASA7) {
    // the inflow state as a mixture record: p and c of its temperature, which the host solved for
    // before the call (BcParams::prim_in)
    const double* qi = m.bc.q_in;
    auto hi = [](double x) { return (float)x; };
    auto lo = [](double x) { return (float)(x - (double)(float)x); };
    const double p = m.bc.prim_in[1];
    float v[16] = {};
    v[0] = hi(qi[0]);
    for (int j = 1; j < 5; ++j) v[j] = hi(qi[j]);
    v[5] = hi(p);
    v[6] = lo(p);
    v[7] = (float)m.bc.prim_in[2];
    for (int k = 0; k < g.ns; ++k) v[8 + k] = hi(qi[5 + k]);
    for (int r = 0; r < 4; ++r) c.in_mrec[r] = make_float4(v[4 * r], v[4 * r + 1], v[4 * r + 2], v[4 * r + 3]);
    c.in_mlo = make_float4(lo(qi[1]), lo(qi[2]), lo(qi[3]), lo(qi[4]));
  }
  return c;
}

cudaError_t launch_prims_mixed(const MeshDev& m, const GasParams& g, const double* q, cudaStream_t s) {
  const size_t KNp = (size_t)m.K * m.Np;
  const mixk::MixedCase c = make_mixed_case(m, g, q, nullptr, nullptr, 0.0);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t want = (KNp + 255) / 256;
  const int blocks = (int)(want < (size_t)sms * 16 ? want : (size_t)sms * 16);
  mixk::prims_kernel<<<blocks, 256, 0, s>>>(c, q, KNp, m.status);
  return cudaGetLastError();
}

MixturePrims mixture_prims_out(const MeshDev& m) {
  MixturePrims mp;
  mp.rec = mixk::mixture_records(m.scratch);
  mp.lo = mixk::mixture_lo(m.scratch, (size_t)m.K * m.Np);
  mp.status = m.status;
  return mp;
}

}  // namespace dg
