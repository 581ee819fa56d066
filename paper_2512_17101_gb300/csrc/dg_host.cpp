// C ABI of libdg: argument checks, handle management and dispatch to the kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "dg_internal.h"

namespace dg {

namespace {
thread_local std::string g_last_error;
}

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) return fail(DG_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
  return fail(DG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Carpenter & Kennedy (1994), five-stage fourth-order 2N-storage scheme.
const double kRK4A[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                         -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kRK4B[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                         1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                         2277821191437.0 / 14882151754819.0};

}  // namespace dg

using dg::fail;
using dg::cuda_fail;

namespace {

void free_mesh_device(dg::MeshDev& d) {
  dg::free_mixed_ops(d);
  cudaFree(d.ops);
  cudaFree(d.fmask);
  cudaFree(d.geo);
  cudaFree(d.vmapP);
  cudaFree(d.scratch);
  cudaFree(d.geo32);
  cudaFree(d.status);
  cudaFree(d.modal);
  cudaFree(d.av_eps);
  cudaFree(d.av_sig);
  cudaFree(d.av_list);
  cudaFree(d.mix_fv);
  cudaFree(d.prim);
  cudaFree(d.wq);
  cudaFree(d.diag);
  cudaFree(d.oi_tab);
  d = dg::MeshDev();
}

template <typename T>
cudaError_t upload(T** dst, const T* src, size_t count) {
  cudaError_t e = cudaMalloc((void**)dst, count * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
}

// The primitives of a mixture's inflow state q[5 + ns] (host): its temperature T by Newton on
// e(T) = e, e(T) = sum_k Y_k sum_j fc[k][j] T^j with e = E/rho - |u|^2/2, from 1000 K until
// |dT| < the gas's tolerance (at least 100 steps allowed); then 1/rho, p = rho R_mix T and
// c = sqrt((p/rho)(1 + R_mix/cv)).  false when the solve does not reach a positive T.
bool mixture_inflow_prims(const dg::GasParams& g, const double* q, dg::BcParams& bc) {
  const double ir = 1.0 / q[0];
  const double e = q[4] * ir - 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) * ir * ir;
  double C[6] = {0, 0, 0, 0, 0, 0}, Rm = 0.0;
  for (int k = 0; k < g.ns; ++k) {
    const double Y = q[5 + k] * ir;
    for (int j = 0; j < 6; ++j) C[j] += Y * g.fc[k][j];
    Rm += Y * g.Rk[k];
  }
  auto cv_at = [&](double t) { return (((5.0 * C[5] * t + 4.0 * C[4]) * t + 3.0 * C[3]) * t + 2.0 * C[2]) * t + C[1]; };
  double T = 1000.0;
  bool done = false;
  const int it_max = std::max(g.newton_max_it, 100);
  for (int it = 0; it < it_max && !done; ++it) {
    const double ev = ((((C[5] * T + C[4]) * T + C[3]) * T + C[2]) * T + C[1]) * T + C[0];
    const double dT = (ev - e) / cv_at(T);
    if (!std::isfinite(dT)) return false;
    T -= dT;
    done = std::fabs(dT) < g.newton_tol;
  }
  const double cv = cv_at(T);
  if (!done || !(T > 0.0) || !(cv > 0.0) || !(Rm > 0.0)) return false;
  const double p = q[0] * Rm * T;
  bc.T_in = T;
  bc.prim_in[0] = ir;
  bc.prim_in[1] = p;
  bc.prim_in[2] = std::sqrt(p * ir * (1.0 + Rm / cv));
  return true;
}

int check_opts(const dg_opts* o) {
  if (!o) return DG_OK;
  if (o->precision != DG_PREC_FP64 && o->precision != DG_PREC_MIXED)
    return fail(DG_ERR_UNSUPPORTED, "unsupported precision mode");
  if (o->t_seed != DG_TSEED_INPUT && o->t_seed != DG_TSEED_CONST && o->t_seed != DG_TSEED_MLP)
    return fail(DG_ERR_INVALID_ARG, "unknown temperature seed mode");
  if (o->t_seed == DG_TSEED_CONST && !(o->t_const > 0)) return fail(DG_ERR_INVALID_ARG, "t_const must be > 0");
  if (o->wait_polls < 0) return fail(DG_ERR_INVALID_ARG, "wait_polls must be >= 0");
  return DG_OK;
}

int read_status(unsigned* dev, uint32_t* bits, int reset) {
  if (!bits) return fail(DG_ERR_INVALID_ARG, "bits is NULL");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "synchronize");
  unsigned v = 0;
  e = cudaMemcpy(&v, dev, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read status");
  *bits = v;
  if (reset) {
    e = cudaMemset(dev, 0, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(e, "reset status");
  }
  return DG_OK;
}

cudaEvent_t take_event(dg::KernelTimer& t) {
  if (!t.pool.empty()) {
    cudaEvent_t e = t.pool.back();
    t.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Records an event pair around launch() on stream s when timing is enabled.
template <typename F>
cudaError_t timed(dg_mesh mesh, int id, cudaStream_t s, F launch) {
  dg::KernelTimer& t = mesh->timer;
  if (!t.enabled) return launch();
  cudaEvent_t a = take_event(t), b = take_event(t);
  if (!a || !b) return cudaErrorMemoryAllocation;
  cudaEventRecord(a, s);
  cudaError_t e = launch();
  cudaEventRecord(b, s);
  t.pending[id].push_back({a, b});
  return e;
}

int resolve_timer(dg::KernelTimer& t) {
  for (int id = 0; id < DG_NUM_KERNELS; ++id) {
    for (auto& pr : t.pending[id]) {
      cudaError_t e = cudaEventSynchronize(pr.second);
      if (e != cudaSuccess) return cuda_fail(e, "event synchronize");
      float ms = 0;
      e = cudaEventElapsedTime(&ms, pr.first, pr.second);
      if (e != cudaSuccess) return cuda_fail(e, "event elapsed time");
      t.ms[id] += ms;
      t.count[id] += 1;
      t.pool.push_back(pr.first);
      t.pool.push_back(pr.second);
    }
    t.pending[id].clear();
  }
  return DG_OK;
}

// Shared front end of dg_rhs and dg_rk_stage.
int run_rhs(dg_mesh mesh, dg_gas gas, const double* q, double* out, double* k, double* T_io, const dg_opts* opts,
            void* stream, bool rk, int stage, double dt) {
  if (!mesh || !gas) return fail(DG_ERR_INVALID_ARG, "NULL mesh or gas handle");
  if (!mesh->d.ops) return fail(DG_ERR_INVALID_ARG, "the mesh was built with DG_MESH_HOST_ONLY");
  if (!q || !out) return fail(DG_ERR_INVALID_ARG, "NULL state or output pointer");
  if (rk && !k) return fail(DG_ERR_INVALID_ARG, "NULL RK register k");
  if (rk && (stage < 0 || stage > 4)) return fail(DG_ERR_INVALID_ARG, "stage must be in 0..4");
  if (rk && !std::isfinite(dt)) return fail(DG_ERR_INVALID_ARG, "dt must be finite");
  if (int rc = check_opts(opts)) return rc;
  const dg::MeshDev& m = mesh->d;
  const dg::GasParams& g = gas->p;
  const int V = 5 + g.ns;
  const bool av = m.av.eps0 > 0;
  // an element range: the FP64 form of a perfect gas without artificial viscosity only
  dg::ElemRange range;
  if (opts && opts->elem_range) {
    if (opts->elem_begin < 0 || opts->elem_end < opts->elem_begin || opts->elem_end > m.K)
      return fail(DG_ERR_INVALID_ARG, "need 0 <= elem_begin <= elem_end <= K");
    if (opts->precision != DG_PREC_FP64 || g.model != DG_GAS_PERFECT || av)
      return fail(DG_ERR_UNSUPPORTED, "element ranges are for the FP64 form of a perfect gas without AV");
    range.begin = opts->elem_begin;
    range.end = opts->elem_end;
  }
  const bool prims_given = opts && opts->prims_given;
  if (prims_given && (opts->precision != DG_PREC_FP64 || g.model != DG_GAS_PERFECT))
    return fail(DG_ERR_UNSUPPORTED, "prims_given is for the FP64 form of a perfect gas");
  if (m.oi_q > 0) {
    if ((opts && opts->precision == DG_PREC_MIXED) || g.model != DG_GAS_PERFECT || (opts && opts->elem_range) ||
        prims_given)
      return fail(DG_ERR_UNSUPPORTED, "over-integration runs in the FP64 form with a perfect gas over the whole mesh");
    if ((g.mu > 0 || av) && m.oi_q <= m.N)
      return fail(DG_ERR_UNSUPPORTED, "viscous and AV fluxes need at least N + 1 points per direction over-integrated");
    if (!dg::overint_fits(m.N, m.oi_q, m.oi_nnz, g.mu > 0, av))
      return fail(DG_ERR_UNSUPPORTED, "the over-integration tables and one element's viscous or AV work exceed a "
                                      "block's shared memory at this point count");
  }
  if (av && g.model != DG_GAS_PERFECT) return fail(DG_ERR_UNSUPPORTED, "artificial viscosity needs a perfect gas");
  if (m.boundary_faces > 0) {
    if (m.inflow_faces > 0 && m.inflow_nvar != V)
      return fail(DG_ERR_INVALID_ARG, "the mesh has inflow faces: set the inflow state with dg_mesh_set_inflow");
    if (m.inflow_faces > 0 && g.model == DG_GAS_NASA7 && !mixture_inflow_prims(g, m.bc.q_in, mesh->d.bc))
      return fail(DG_ERR_INVALID_ARG, "the inflow state has no temperature: its Newton solve did not converge");
  }
  const size_t bytes = sizeof(double) * (size_t)V * m.K * m.Np;
  if (q == out || (q < out + bytes / sizeof(double) && out < q + bytes / sizeof(double)))
    return fail(DG_ERR_INVALID_ARG, "output overlaps the input state");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  const double a = rk ? dg::kRK4A[stage] : 0.0, b = rk ? dg::kRK4B[stage] : 0.0;
  if (opts && opts->precision == DG_PREC_MIXED) {
    if (g.model == DG_GAS_NASA7) {
      // FP64 Newton temperature (seeded as opts says), which at the converged temperature also
      // writes the FP64 pressure, the sound speed and the float state copy; then the
      // tensor-core right-hand side of the mixture
      if (!T_io) return fail(DG_ERR_INVALID_ARG, "a NASA-7 gas needs the temperature buffer T_io");
      if (g.mu > 0) return fail(DG_ERR_UNSUPPORTED, "the mixed-precision mixture path is inviscid");
      const int mode = opts->t_seed;
      if (mode == DG_TSEED_MLP && !gas->has_mlp) return fail(DG_ERR_INVALID_ARG, "DG_TSEED_MLP needs a trained MLP");
      const dg::MixturePrims mp = dg::mixture_prims_out(m);
      e = timed(mesh, DG_KERNEL_TEMPERATURE, s, [&] {
        if (mode == DG_TSEED_MLP)
          return dg::launch_temperature_mlp(gas, (int64_t)m.K * m.Np, q, T_io, nullptr, 0, s, mp, opts->wait_polls);
        return dg::launch_temperature(g, (int64_t)m.K * m.Np, q, T_io, nullptr, mode, opts->t_const, gas->status, s,
                                      mp);
      });
      if (e != cudaSuccess) return cuda_fail(e, "temperature kernel");
    } else {
      e = timed(mesh, DG_KERNEL_PRIMS, s, [&] { return dg::launch_prims_mixed(m, g, q, s); });
      if (e != cudaSuccess) return cuda_fail(e, "mixed primitives kernel");
      if (g.mu > 0) {
        e = timed(mesh, DG_KERNEL_VISCOUS, s, [&] { return dg::launch_viscous_tc(m, g, q, s, opts->wait_polls); });
        if (e != cudaSuccess) return cuda_fail(e, "mixed viscous kernel");
      }
      if (av) {  // the element viscosities and the AV flux in FP32 arithmetic, for the tensor-core
                 // right-hand side, which takes sigma as one of its FP32 terms
        e = timed(mesh, DG_KERNEL_AV, s, [&] {
          cudaError_t e2 = dg::launch_av_sensor(m, q, m.av_eps, s, m.av_list, true);
          return e2 == cudaSuccess ? dg::launch_av_flux(m, g, q, s, true) : e2;
        });
        if (e != cudaSuccess) return cuda_fail(e, "artificial-viscosity kernels");
      }
    }
    e = timed(mesh, DG_KERNEL_RHS, s, [&] {
      return dg::launch_rhs_tc(m, g, q, out, k, rk, a, b, dt, s, opts->wait_polls);
    });
    if (e != cudaSuccess) return cuda_fail(e, "mixed right-hand-side kernel");
    return DG_OK;
  }
  const double* T = nullptr;
  if (g.model == DG_GAS_NASA7) {
    if (!T_io) return fail(DG_ERR_INVALID_ARG, "a NASA-7 gas needs the temperature buffer T_io");
    const int mode = opts ? opts->t_seed : DG_TSEED_INPUT;
    const double tc = opts ? opts->t_const : 0.0;
    if (mode == DG_TSEED_MLP && !gas->has_mlp) return fail(DG_ERR_INVALID_ARG, "DG_TSEED_MLP needs a trained MLP");
    dg::MixturePrims mp64;  // 1/rho, p, c at the converged temperature, for the right-hand side
    mp64.prim = m.prim;
    mp64.status = m.status;
    e = timed(mesh, DG_KERNEL_TEMPERATURE, s, [&] {
      if (mode == DG_TSEED_MLP)
        return dg::launch_temperature_mlp(gas, (int64_t)m.K * m.Np, q, T_io, nullptr, 0, s, mp64);
      return dg::launch_temperature(g, (int64_t)m.K * m.Np, q, T_io, nullptr, mode, tc, gas->status, s, mp64);
    });
    if (e != cudaSuccess) return cuda_fail(e, "temperature kernel");
    T = T_io;
  }
  const bool mix_ns = g.model == DG_GAS_NASA7 && g.mu > 0;
  if (mix_ns) {
    if (!m.mix_fv) {  // first viscous-mixture call on this mesh: its flux buffer
      e = cudaMalloc((void**)&mesh->d.mix_fv, sizeof(double) * (9 + 3 * DG_MAX_SPECIES) * (size_t)m.K * m.Np);
      if (e != cudaSuccess) return cuda_fail(e, "mixture viscous-flux buffer");
    }
    e = timed(mesh, DG_KERNEL_VISCOUS, s, [&] { return dg::launch_viscous_mixture(m, g, q, T, s); });
    if (e != cudaSuccess) return cuda_fail(e, "mixture viscous flux kernel");
    e = timed(mesh, DG_KERNEL_RHS, s,
              [&] { return dg::launch_rhs_mixture_ns(m, g, q, out, k, T, rk, a, b, dt, s); });
    if (e != cudaSuccess) return cuda_fail(e, "right-hand-side kernel");
    return DG_OK;
  }
  // (1/rho, p, c) once per node for the next kernels (the over-integrated Euler kernel reads none)
  if (g.model == DG_GAS_PERFECT && !prims_given && !(m.oi_q > 0 && g.mu == 0)) {
    e = timed(mesh, DG_KERNEL_PRIMS, s, [&] { return dg::launch_prims_fp64(m, g, q, s); });
    if (e != cudaSuccess) return cuda_fail(e, "primitives kernel");
  }
  if (g.mu > 0 && !(opts && opts->viscous_given)) {
    // the whole mesh: the range's right-hand side reads its neighbours' viscous flux
    e = timed(mesh, DG_KERNEL_VISCOUS, s, [&] { return dg::launch_viscous_flux(m, g, q, s); });
    if (e != cudaSuccess) return cuda_fail(e, "viscous flux kernel");
  }
  if (av) {
    e = timed(mesh, DG_KERNEL_AV, s, [&] {
      cudaError_t e2 = dg::launch_av_sensor(m, q, m.av_eps, s, m.av_list);
      return e2 == cudaSuccess ? dg::launch_av_flux(m, g, q, s) : e2;
    });
    if (e != cudaSuccess) return cuda_fail(e, "artificial-viscosity kernels");
  }
  if (m.oi_q > 0) {
    e = timed(mesh, DG_KERNEL_RHS, s, [&] { return dg::launch_rhs_overint(m, g, q, out, k, rk, a, b, dt, s); });
    if (e != cudaSuccess) return cuda_fail(e, "over-integrated right-hand-side kernel");
    return DG_OK;
  }
  if (av) {
    e = timed(mesh, DG_KERNEL_RHS, s, [&] { return dg::launch_rhs_av(m, g, q, out, k, rk, a, b, dt, s); });
    if (e != cudaSuccess) return cuda_fail(e, "right-hand-side kernel");
    return DG_OK;
  }
  e = timed(mesh, DG_KERNEL_RHS, s, [&] { return dg::launch_rhs(m, g, q, out, k, T, rk, a, b, dt, s, range); });
  if (e != cudaSuccess) return cuda_fail(e, "right-hand-side kernel");
  return DG_OK;
}

}  // namespace

extern "C" {

const char* dg_last_error(void) { return dg::g_last_error.c_str(); }

int dg_lsrk4_coefficients(double* a_host, double* b_host) {
  if (!a_host || !b_host) return fail(DG_ERR_INVALID_ARG, "NULL output");
  for (int s = 0; s < 5; ++s) {
    a_host[s] = dg::kRK4A[s];
    b_host[s] = dg::kRK4B[s];
  }
  return DG_OK;
}

int dg_mesh_upload(const dg_mesh_desc* desc, dg_mesh* out) {
  if (!desc || !out) return fail(DG_ERR_INVALID_ARG, "NULL descriptor or output handle");
  *out = nullptr;
  if (desc->K < 1) return fail(DG_ERR_INVALID_ARG, "K must be >= 1");
  if (desc->N < 1 || desc->N > DG_MAX_ORDER) return fail(DG_ERR_INVALID_ARG, "N must be in 1..4");
  if (!desc->ref_nodes || !desc->vertices) return fail(DG_ERR_INVALID_ARG, "NULL ref_nodes or vertices");
  for (int x = 0; x < 3; ++x)
    if (!(desc->period[x] >= 0) || !std::isfinite(desc->period[x]))
      return fail(DG_ERR_INVALID_ARG, "period must be finite and >= 0");
  const int n_ops = !!desc->Dr + !!desc->Ds + !!desc->Dt + !!desc->LIFT + !!desc->Fmask;
  if (n_ops != 0 && n_ops != 5) return fail(DG_ERR_INVALID_ARG, "give all of Dr, Ds, Dt, LIFT and Fmask, or none");
  if (!desc->EToE != !desc->EToF) return fail(DG_ERR_INVALID_ARG, "give EToE and EToF together");
  dg_mesh m = new (std::nothrow) dg_mesh_s();
  if (!m) return fail(DG_ERR_OOM, "host allocation failed");
  std::string err;
  const int K = desc->K;
  bool ok = dg::build_ref_ops(desc->N, desc->ref_nodes, m->ops, err);
  if (ok) m->ref_nodes.assign(desc->ref_nodes, desc->ref_nodes + 3 * m->ops.Np);
  if (ok && n_ops == 5) {  // the caller's operators replace the built ones
    const int Np = m->ops.Np, Nfp = m->ops.Nfp;
    ok = dg::check_ref_ops(desc->N, desc->ref_nodes, desc->Dr, desc->Ds, desc->Dt, desc->LIFT, desc->Fmask, err);
    if (ok) {
      m->ops.Dr.assign(desc->Dr, desc->Dr + Np * Np);
      m->ops.Ds.assign(desc->Ds, desc->Ds + Np * Np);
      m->ops.Dt.assign(desc->Dt, desc->Dt + Np * Np);
      m->ops.LIFT.assign(desc->LIFT, desc->LIFT + (size_t)Np * 4 * Nfp);
      m->ops.Fmask.assign(desc->Fmask, desc->Fmask + 4 * Nfp);
    }
  }
  if (ok) {
    if (desc->geo) {
      ok = dg::check_geometry(K, desc->geo, err);
      if (ok) m->geo.assign(desc->geo, desc->geo + (size_t)K * DG_GEO_STRIDE);
    } else {
      ok = dg::build_geometry(K, desc->vertices, m->geo, err);
    }
  }
  if (ok) {
    if (desc->vmapP) {
      ok = dg::check_connectivity(K, desc->vertices, desc->period, m->ops, desc->ref_nodes, desc->face_bc,
                                  desc->vmapP, m->partner, err);
      if (ok) m->vmapP.assign(desc->vmapP, desc->vmapP + (size_t)K * 4 * m->ops.Nfp);
    } else if (desc->EToE) {
      ok = dg::build_connectivity_from_faces(K, desc->vertices, desc->period, m->ops, desc->ref_nodes, desc->face_bc,
                                             desc->EToE, desc->EToF, m->vmapP, err, m->partner);
    } else {
      ok = dg::build_connectivity(K, desc->vertices, desc->period, m->ops, desc->ref_nodes, desc->face_bc,
                                  m->vmapP, err, &m->partner);
    }
  }
  if (ok && desc->EToE && desc->vmapP) {  // both given: they must describe the same pairing
    for (int kf = 0; kf < 4 * K && ok; ++kf) {
      const int pf = m->partner[kf];
      const int e2 = pf < 0 ? -1 : pf / 4, f2 = pf < 0 ? -1 : pf % 4;
      if (desc->EToE[kf] != e2 || (e2 >= 0 && desc->EToF[kf] != f2)) {
        err = "EToE / EToF disagree with vmapP at face " + std::to_string(kf % 4) + " of element " +
              std::to_string(kf / 4);
        ok = false;
      }
    }
  }
  if (ok && desc->EToV) ok = dg::check_vertex_numbers(K, desc->EToV, m->partner, err);
  if (!ok) {
    delete m;
    return fail(DG_ERR_INVALID_ARG, err);
  }
  dg::MeshDev& d = m->d;
  d.K = desc->K;
  d.N = desc->N;
  d.Np = m->ops.Np;
  d.Nfp = m->ops.Nfp;
  for (int k = 0; k < d.K; ++k)
    for (int f = 0; f < 4; ++f) {
      const int32_t v = m->vmapP[(size_t)k * 4 * d.Nfp + f * d.Nfp];
      d.boundary_faces += v < 0;
      d.inflow_faces += v == -DG_BC_INFLOW;
    }
  if (desc->flags & DG_MESH_HOST_ONLY) {
    *out = m;
    return DG_OK;
  }
  cudaGetDevice(&m->device);
  const int Np = d.Np, NF = 4 * d.Nfp;
  std::vector<double> ops;
  ops.reserve(3 * Np * Np + Np * NF);
  ops.insert(ops.end(), m->ops.Dr.begin(), m->ops.Dr.end());
  ops.insert(ops.end(), m->ops.Ds.begin(), m->ops.Ds.end());
  ops.insert(ops.end(), m->ops.Dt.begin(), m->ops.Dt.end());
  ops.insert(ops.end(), m->ops.LIFT.begin(), m->ops.LIFT.end());
  cudaError_t e = upload(&d.ops, ops.data(), ops.size());
  if (e == cudaSuccess) e = upload(&d.fmask, m->ops.Fmask.data(), m->ops.Fmask.size());
  if (e == cudaSuccess) e = upload(&d.geo, m->geo.data(), m->geo.size());
  if (e == cudaSuccess) e = upload(&d.vmapP, m->vmapP.data(), m->vmapP.size());
  if (e == cudaSuccess) {
    std::vector<float> g32(m->geo.begin(), m->geo.end());
    e = upload(&d.geo32, g32.data(), g32.size());
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&d.scratch, sizeof(double) * 10 * (size_t)d.K * Np);
  if (e == cudaSuccess) e = cudaMalloc((void**)&d.prim, sizeof(double) * 3 * (size_t)d.K * Np);
  if (e == cudaSuccess) e = cudaMalloc((void**)&d.status, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(d.status, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = dg::build_tc_ops(d, m->ops);
  if (e == cudaSuccess) e = upload(&d.modal, m->ops.modal.data(), m->ops.modal.size());
  if (e == cudaSuccess) e = upload(&d.wq, m->ops.wq.data(), m->ops.wq.size());
  if (e == cudaSuccess) e = cudaMalloc((void**)&d.diag, dg::kDiagPartialBytes);
  d.ntop = m->ops.ntop;
  if (e != cudaSuccess) {
    free_mesh_device(d);
    delete m;
    return cuda_fail(e, "mesh upload");
  }
  *out = m;
  return DG_OK;
}

int dg_mesh_set_timing(dg_mesh mesh, int enable) {
  if (!mesh) return fail(DG_ERR_INVALID_ARG, "NULL mesh");
  if (!mesh->d.ops) return fail(DG_ERR_INVALID_ARG, "the mesh was built with DG_MESH_HOST_ONLY");
  mesh->timer.enabled = enable != 0;
  return DG_OK;
}

int dg_mesh_kernel_times(dg_mesh mesh, double* ms, int64_t* launches, int reset) {
  if (!mesh) return fail(DG_ERR_INVALID_ARG, "NULL mesh");
  if (int rc = resolve_timer(mesh->timer)) return rc;
  for (int id = 0; id < DG_NUM_KERNELS; ++id) {
    if (ms) ms[id] = mesh->timer.ms[id];
    if (launches) launches[id] = mesh->timer.count[id];
    if (reset) {
      mesh->timer.ms[id] = 0;
      mesh->timer.count[id] = 0;
    }
  }
  return DG_OK;
}

int dg_mesh_free(dg_mesh mesh) {
  if (!mesh) return DG_OK;
  resolve_timer(mesh->timer);
  for (cudaEvent_t e : mesh->timer.pool) cudaEventDestroy(e);
  free_mesh_device(mesh->d);
  delete mesh;
  return DG_OK;
}

int dg_mesh_info(dg_mesh mesh, int32_t* K, int32_t* N, int32_t* Np, int32_t* Nfp) {
  if (!mesh) return fail(DG_ERR_INVALID_ARG, "NULL mesh");
  if (K) *K = mesh->d.K;
  if (N) *N = mesh->d.N;
  if (Np) *Np = mesh->d.Np;
  if (Nfp) *Nfp = mesh->d.Nfp;
  return DG_OK;
}

int dg_mesh_operators(dg_mesh mesh, double* Dr, double* Ds, double* Dt, double* LIFT, int32_t* Fmask) {
  if (!mesh) return fail(DG_ERR_INVALID_ARG, "NULL mesh");
  const dg::RefOps& o = mesh->ops;
  if (Dr) std::memcpy(Dr, o.Dr.data(), sizeof(double) * o.Dr.size());
  if (Ds) std::memcpy(Ds, o.Ds.data(), sizeof(double) * o.Ds.size());
  if (Dt) std::memcpy(Dt, o.Dt.data(), sizeof(double) * o.Dt.size());
  if (LIFT) std::memcpy(LIFT, o.LIFT.data(), sizeof(double) * o.LIFT.size());
  if (Fmask) std::memcpy(Fmask, o.Fmask.data(), sizeof(int32_t) * o.Fmask.size());
  return DG_OK;
}

int dg_mesh_set_inflow(dg_mesh mesh, const double* q_in, int32_t nvar) {
  if (!mesh || !q_in) return fail(DG_ERR_INVALID_ARG, "NULL mesh or inflow state");
  if (nvar < 5 || nvar > 5 + DG_MAX_SPECIES) return fail(DG_ERR_INVALID_ARG, "nvar must be in 5..5+DG_MAX_SPECIES");
  for (int v = 0; v < nvar; ++v)
    if (!std::isfinite(q_in[v])) return fail(DG_ERR_INVALID_ARG, "the inflow state must be finite");
  if (!(q_in[0] > 0)) return fail(DG_ERR_INVALID_ARG, "the inflow density must be positive");
  for (int v = 0; v < 5 + DG_MAX_SPECIES; ++v) mesh->d.bc.q_in[v] = v < nvar ? q_in[v] : 0.0;
  mesh->d.inflow_nvar = nvar;
  return DG_OK;
}

int dg_mesh_set_av(dg_mesh mesh, const dg_av_params* p) {
  if (!mesh) return fail(DG_ERR_INVALID_ARG, "NULL mesh");
  if (!mesh->d.ops) return fail(DG_ERR_INVALID_ARG, "the mesh was built with DG_MESH_HOST_ONLY");
  dg::MeshDev& d = mesh->d;
  if (!p || p->eps0 == 0.0) {
    d.av = dg::AvParams{0.0, 0.0, 1.0};
    return DG_OK;
  }
  if (!(p->eps0 > 0) || !std::isfinite(p->eps0) || !std::isfinite(p->s0) || !(p->kappa > 0) ||
      !std::isfinite(p->kappa))
    return fail(DG_ERR_INVALID_ARG, "need eps0 >= 0, kappa > 0, all finite");
  if (!d.av_eps) {
    cudaError_t e = cudaMalloc((void**)&d.av_eps, sizeof(double) * (size_t)d.K);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d.av_sig, sizeof(double) * 15 * (size_t)d.K * d.Np);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d.av_list, sizeof(int) * (1 + (size_t)d.K));
    if (e != cudaSuccess) {
      cudaFree(d.av_eps);
      cudaFree(d.av_sig);
      cudaFree(d.av_list);
      d.av_eps = d.av_sig = nullptr;
      d.av_list = nullptr;
      return cuda_fail(e, "artificial-viscosity scratch");
    }
  }
  d.av = dg::AvParams{p->eps0, p->s0, p->kappa};
  return DG_OK;
}

int dg_tet_quadrature(int32_t q, double* rst, double* w) {
  if (!rst || !w) return fail(DG_ERR_INVALID_ARG, "NULL output");
  std::vector<double> r, ww;
  std::string err;
  if (!dg::tet_quadrature(q, r, ww, err)) return fail(DG_ERR_INVALID_ARG, err);
  std::memcpy(rst, r.data(), sizeof(double) * r.size());
  std::memcpy(w, ww.data(), sizeof(double) * ww.size());
  return DG_OK;
}

int dg_mesh_set_overint(dg_mesh mesh, int32_t q) {
  if (!mesh) return fail(DG_ERR_INVALID_ARG, "NULL mesh");
  if (!mesh->d.ops) return fail(DG_ERR_INVALID_ARG, "the mesh was built with DG_MESH_HOST_ONLY");
  if (q < DG_OVERINT_DEFAULT || q > DG_MAX_OVERINT_POINTS)
    return fail(DG_ERR_INVALID_ARG, "points per direction must be DG_OVERINT_DEFAULT, 0 or 1..DG_MAX_OVERINT_POINTS");
  dg::MeshDev& d = mesh->d;
  if (q == 0) {
    cudaFree(d.oi_tab);
    d.oi_tab = nullptr;
    d.oi_q = d.oi_ng = d.oi_nnz = 0;
    return DG_OK;
  }
  if (q == DG_OVERINT_DEFAULT) q = (3 * d.N + 1) / 2;
  dg::OverintOps o;
  std::string err;
  if (!dg::build_overint_ops(d.N, mesh->ref_nodes.data(), q, o, err)) return fail(DG_ERR_INVALID_ARG, err);
  if (!dg::overint_fits(d.N, q, (int)o.Dh_val.size(), false, false))
    return fail(DG_ERR_UNSUPPORTED, "the over-integration tables and one element's work exceed a block's shared memory");
  // device layout: A | Aw | B | Bw | C | Cw | V_o^-T | V_o^T | Dh_val | Dh_ptr | Dh_idx | Dh_col (the
  // kernel's order; the small integers of the last three exact as doubles)
  std::vector<double> tab;
  for (const std::vector<double>* t : {&o.A, &o.Aw, &o.B, &o.Bw, &o.C, &o.Cw, &o.VinvT, &o.VoT, &o.Dh_val})
    tab.insert(tab.end(), t->begin(), t->end());
  for (const std::vector<int>* t : {&o.Dh_ptr, &o.Dh_idx, &o.Dh_col}) tab.insert(tab.end(), t->begin(), t->end());
  double* dev = nullptr;
  cudaError_t e = cudaMalloc((void**)&dev, sizeof(double) * tab.size());
  if (e == cudaSuccess) e = cudaMemcpy(dev, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(dev);
    return cuda_fail(e, "over-integration tables");
  }
  cudaFree(d.oi_tab);
  d.oi_tab = dev;
  d.oi_q = q;
  d.oi_ng = o.Ng;
  d.oi_nnz = (int)o.Dh_val.size();
  return DG_OK;
}

int dg_av_viscosity(dg_mesh mesh, const double* q, double* eps, void* stream) {
  if (!mesh || !q || !eps) return fail(DG_ERR_INVALID_ARG, "NULL mesh, state or output");
  if (!mesh->d.ops) return fail(DG_ERR_INVALID_ARG, "the mesh was built with DG_MESH_HOST_ONLY");
  const cudaError_t e = dg::launch_av_sensor(mesh->d, q, eps, (cudaStream_t)stream);
  return e == cudaSuccess ? DG_OK : cuda_fail(e, "smoothness-indicator kernel");
}

namespace {
// Arguments shared by the ranged FP64 perfect-gas entry points.
int check_range_call(dg_mesh mesh, dg_gas gas, const double* q, int32_t b, int32_t e, bool viscous) {
  if (!mesh || !gas || !q) return fail(DG_ERR_INVALID_ARG, "NULL mesh, gas or state");
  if (!mesh->d.ops) return fail(DG_ERR_INVALID_ARG, "the mesh was built with DG_MESH_HOST_ONLY");
  if (gas->p.model != DG_GAS_PERFECT || (viscous && !(gas->p.mu > 0)))
    return fail(DG_ERR_INVALID_ARG, viscous ? "the viscous pass needs a viscous perfect gas"
                                            : "the primitives pass needs a perfect gas");
  if (b < 0 || e < b || e > mesh->d.K) return fail(DG_ERR_INVALID_ARG, "need 0 <= elem_begin <= elem_end <= K");
  return DG_OK;
}
}  // namespace

int dg_primitives(dg_mesh mesh, dg_gas gas, const double* q, int32_t elem_begin, int32_t elem_end, void* stream) {
  if (int rc = check_range_call(mesh, gas, q, elem_begin, elem_end, false)) return rc;
  dg::ElemRange r;
  r.begin = elem_begin;
  r.end = elem_end;
  const cudaError_t e = dg::launch_prims_fp64(mesh->d, gas->p, q, (cudaStream_t)stream, r);
  return e == cudaSuccess ? DG_OK : cuda_fail(e, "primitives kernel");
}

int dg_viscous_flux_range(dg_mesh mesh, dg_gas gas, const double* q, int32_t elem_begin, int32_t elem_end,
                          void* stream) {
  if (int rc = check_range_call(mesh, gas, q, elem_begin, elem_end, true)) return rc;
  dg::ElemRange r;
  r.begin = elem_begin;
  r.end = elem_end;
  const cudaError_t e = dg::launch_viscous_flux(mesh->d, gas->p, q, (cudaStream_t)stream, r);
  return e == cudaSuccess ? DG_OK : cuda_fail(e, "viscous flux kernel");
}

int dg_viscous_flux(dg_mesh mesh, dg_gas gas, const double* q, void* stream) {
  if (int rc = check_range_call(mesh, gas, q, 0, mesh ? mesh->d.K : 0, true)) return rc;
  cudaError_t e = dg::launch_prims_fp64(mesh->d, gas->p, q, (cudaStream_t)stream);
  if (e == cudaSuccess) e = dg::launch_viscous_flux(mesh->d, gas->p, q, (cudaStream_t)stream);
  return e == cudaSuccess ? DG_OK : cuda_fail(e, "viscous flux kernels");
}

int dg_mesh_viscous_buffer(dg_mesh mesh, double** fv) {
  if (!mesh || !fv) return fail(DG_ERR_INVALID_ARG, "NULL mesh or output");
  if (!mesh->d.scratch) return fail(DG_ERR_INVALID_ARG, "the mesh was built with DG_MESH_HOST_ONLY");
  *fv = mesh->d.scratch;
  return DG_OK;
}

int dg_mesh_connectivity(dg_mesh mesh, int32_t* vmapP, double* geo) {
  if (!mesh) return fail(DG_ERR_INVALID_ARG, "NULL mesh");
  if (vmapP) std::memcpy(vmapP, mesh->vmapP.data(), sizeof(int32_t) * mesh->vmapP.size());
  if (geo) std::memcpy(geo, mesh->geo.data(), sizeof(double) * mesh->geo.size());
  return DG_OK;
}

int dg_mesh_face_pairs(dg_mesh mesh, int32_t* EToE, int32_t* EToF) {
  if (!mesh) return fail(DG_ERR_INVALID_ARG, "NULL mesh");
  for (size_t kf = 0; kf < mesh->partner.size(); ++kf) {
    const int pf = mesh->partner[kf];
    if (EToE) EToE[kf] = pf < 0 ? -1 : pf / 4;
    if (EToF) EToF[kf] = pf < 0 ? -1 : pf % 4;
  }
  return DG_OK;
}

int dg_mesh_status(dg_mesh mesh, uint32_t* bits, int reset) {
  if (!mesh) return fail(DG_ERR_INVALID_ARG, "NULL mesh");
  if (!mesh->d.status) return fail(DG_ERR_INVALID_ARG, "the mesh was built with DG_MESH_HOST_ONLY");
  return read_status(mesh->d.status, bits, reset);
}

int dg_gas_create(const dg_gas_desc* desc, dg_gas* out) {
  if (!desc || !out) return fail(DG_ERR_INVALID_ARG, "NULL descriptor or output handle");
  *out = nullptr;
  dg::GasParams p;
  std::memset(&p, 0, sizeof(p));
  p.model = desc->model;
  p.mu = desc->mu;
  p.Pr = desc->Pr;
  if (!(desc->mu >= 0) || !std::isfinite(desc->mu)) return fail(DG_ERR_INVALID_ARG, "mu must be >= 0");
  if (desc->mu > 0 && !(desc->Pr > 0)) return fail(DG_ERR_INVALID_ARG, "Pr must be > 0 when mu > 0");
  if (desc->model == DG_GAS_PERFECT) {
    if (!(desc->gamma > 1) || !(desc->R > 0)) return fail(DG_ERR_INVALID_ARG, "need gamma > 1 and R > 0");
    p.gamma = desc->gamma;
    p.R = desc->R;
    p.cp = desc->gamma * desc->R / (desc->gamma - 1);
    p.kappa = desc->mu > 0 ? desc->mu * p.cp / desc->Pr : 0.0;
  } else if (desc->model == DG_GAS_NASA7) {
    if (desc->nspecies < 1 || desc->nspecies > DG_MAX_SPECIES)
      return fail(DG_ERR_INVALID_ARG, "nspecies must be in 1..8");
    if (!desc->W || !desc->nasa7) return fail(DG_ERR_INVALID_ARG, "NULL W or nasa7");
    if (desc->mu > 0 && !(desc->Sc > 0)) return fail(DG_ERR_INVALID_ARG, "a viscous mixture needs Sc > 0");
    p.Sc = desc->Sc;
    if (!(desc->R_universal > 0)) return fail(DG_ERR_INVALID_ARG, "R_universal must be > 0");
    if (!(desc->newton_tol > 0) || desc->newton_max_it < 1)
      return fail(DG_ERR_INVALID_ARG, "need newton_tol > 0 and newton_max_it >= 1");
    p.ns = desc->nspecies;
    for (int k = 0; k < p.ns; ++k) {
      if (!(desc->W[k] > 0)) return fail(DG_ERR_INVALID_ARG, "molar masses must be > 0");
      p.Rk[k] = desc->R_universal / desc->W[k];
      for (int i = 0; i < 7; ++i) p.a[k][i] = desc->nasa7[7 * k + i];
      const double* a = p.a[k];
      const double fc[6] = {a[5], a[0] - 1.0, a[1] / 2.0, a[2] / 3.0, a[3] / 4.0, a[4] / 5.0};
      for (int j = 0; j < 6; ++j) p.fc[k][j] = p.Rk[k] * fc[j];
      for (int j = 0; j < 7; ++j) {
        const double x = j < 6 ? p.fc[k][j] : p.Rk[k];
        const float hi = (float)x;
        p.fc2[k][j] = make_float2(hi, (float)(x - (double)hi));
      }
    }
    p.newton_tol = desc->newton_tol;
    p.newton_max_it = desc->newton_max_it;
  } else {
    return fail(DG_ERR_INVALID_ARG, "unknown gas model");
  }
  dg_gas g = new (std::nothrow) dg_gas_s();
  if (!g) return fail(DG_ERR_OOM, "host allocation failed");
  g->p = p;
  cudaGetDevice(&g->device);
  cudaError_t e = cudaMalloc((void**)&g->status, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(g->status, 0, sizeof(unsigned));
  if (e != cudaSuccess) {
    cudaFree(g->status);
    delete g;
    return cuda_fail(e, "gas status allocation");
  }
  *out = g;
  return DG_OK;
}

int dg_gas_free(dg_gas gas) {
  if (!gas) return DG_OK;
  cudaFree(gas->status);
  cudaFree(gas->mlp_theta);
  cudaFree(gas->mlp_w1h);
  cudaFree(gas->mlp_w2h);
  delete gas;
  return DG_OK;
}

int dg_gas_status(dg_gas gas, uint32_t* bits, int reset) {
  if (!gas) return fail(DG_ERR_INVALID_ARG, "NULL gas");
  return read_status(gas->status, bits, reset);
}

int dg_rhs(dg_mesh mesh, dg_gas gas, const double* q, double* rhs, double* T_io, const dg_opts* opts,
           void* stream) {
  return run_rhs(mesh, gas, q, rhs, nullptr, T_io, opts, stream, false, 0, 0.0);
}

int dg_rk_stage(dg_mesh mesh, dg_gas gas, int32_t stage, double dt, const double* q_in, double* q_out,
                double* k, double* T_io, const dg_opts* opts, void* stream) {
  return run_rhs(mesh, gas, q_in, q_out, k, T_io, opts, stream, true, stage, dt);
}

int dg_temperature(dg_gas gas, int64_t n, const double* q, double* T_io, int32_t* iters, const dg_opts* opts,
                   void* stream) {
  if (!gas) return fail(DG_ERR_INVALID_ARG, "NULL gas");
  if (gas->p.model != DG_GAS_NASA7) return fail(DG_ERR_INVALID_ARG, "dg_temperature needs a NASA-7 gas");
  if (n < 0) return fail(DG_ERR_INVALID_ARG, "n must be >= 0");
  if (n == 0) return DG_OK;
  if (!q || !T_io) return fail(DG_ERR_INVALID_ARG, "NULL state or temperature");
  if (int rc = check_opts(opts)) return rc;
  const int mode = opts ? opts->t_seed : DG_TSEED_INPUT;
  const double tc = opts ? opts->t_const : 0.0;
  if (mode == DG_TSEED_MLP && !gas->has_mlp) return fail(DG_ERR_INVALID_ARG, "DG_TSEED_MLP needs a trained MLP");
  cudaError_t e = mode == DG_TSEED_MLP
                      ? dg::launch_temperature_mlp(gas, n, q, T_io, iters, 0, (cudaStream_t)stream,
                                                   dg::MixturePrims(), opts ? opts->wait_polls : 0)
                      : dg::launch_temperature(gas->p, n, q, T_io, iters, mode, tc, gas->status, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "temperature kernel");
  return DG_OK;
}

int dg_mixture_energy(dg_gas gas, int64_t n, const double* T, const double* Y, double* e_out, void* stream) {
  if (!gas) return fail(DG_ERR_INVALID_ARG, "NULL gas");
  if (gas->p.model != DG_GAS_NASA7) return fail(DG_ERR_INVALID_ARG, "dg_mixture_energy needs a NASA-7 gas");
  if (n < 0) return fail(DG_ERR_INVALID_ARG, "n must be >= 0");
  if (n == 0) return DG_OK;
  if (!T || !Y || !e_out) return fail(DG_ERR_INVALID_ARG, "NULL pointer");
  cudaError_t e = dg::launch_mixture_energy(gas->p, n, T, Y, e_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "mixture energy kernel");
  return DG_OK;
}

int dg_mlp_set(dg_gas gas, const float* params, const dg_mlp_norm* norm) {
  if (!gas || !params || !norm) return fail(DG_ERR_INVALID_ARG, "NULL gas, params or norm");
  if (gas->p.model != DG_GAS_NASA7) return fail(DG_ERR_INVALID_ARG, "the MLP guess needs a NASA-7 gas");
  if (!(norm->e_scale > 0) || !(norm->T_scale > 0) || !(norm->T_max >= norm->T_min))
    return fail(DG_ERR_INVALID_ARG, "need e_scale > 0, T_scale > 0 and T_max >= T_min");
  cudaError_t e = dg::mlp_set_params(gas, params, *norm);
  if (e != cudaSuccess) return cuda_fail(e, "MLP upload");
  return DG_OK;
}

int dg_mlp_get(dg_gas gas, float* params, dg_mlp_norm* norm) {
  if (!gas) return fail(DG_ERR_INVALID_ARG, "NULL gas");
  if (!gas->has_mlp) return fail(DG_ERR_INVALID_ARG, "the gas has no MLP");
  if (params) {
    cudaError_t e = cudaMemcpy(params, gas->mlp_theta, sizeof(float) * DG_MLP_PARAMS, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "MLP download");
  }
  if (norm) *norm = gas->mlp_norm;
  return DG_OK;
}

int dg_mlp_loss_grad(int64_t n, const float* params, const float* x, const float* t, float* grad, float* loss,
                     void* stream) {
  if (n < 0) return fail(DG_ERR_INVALID_ARG, "n must be >= 0");
  if (n == 0) return DG_OK;
  if (!params || !x || !t || !grad || !loss) return fail(DG_ERR_INVALID_ARG, "NULL pointer");
  cudaError_t e = dg::mlp_loss_grad(n, params, x, t, grad, loss, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "MLP gradient kernel");
  return DG_OK;
}

int dg_mlp_adam_step(int32_t t, float lr, float* params, float* grad, float* m, float* v, void* stream) {
  if (!params || !grad || !m || !v) return fail(DG_ERR_INVALID_ARG, "NULL pointer");
  if (t < 1) return fail(DG_ERR_INVALID_ARG, "the step number t must be >= 1");
  if (!std::isfinite(lr)) return fail(DG_ERR_INVALID_ARG, "lr must be finite");
  cudaError_t e = dg::mlp_adam_step(t, lr, params, grad, m, v, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "Adam kernel");
  return DG_OK;
}

int dg_mlp_train(dg_gas gas, int64_t n, const double* e_dev, const double* Y_dev, const double* T_dev,
                 const float* init, const dg_mlp_train_opts* o, float* history) {
  if (!gas || !o || !init) return fail(DG_ERR_INVALID_ARG, "NULL gas, options or initial parameters");
  if (gas->p.model != DG_GAS_NASA7) return fail(DG_ERR_INVALID_ARG, "the MLP guess needs a NASA-7 gas");
  if (gas->p.ns > 7) return fail(DG_ERR_UNSUPPORTED, "the MLP takes at most 7 mass fractions");
  if (!e_dev || !Y_dev || !T_dev) return fail(DG_ERR_INVALID_ARG, "NULL sample array");
  if (o->epochs < 1 || o->batch < 1 || !(o->lr > 0) || !(o->lr_decay > 0) || n < o->batch)
    return fail(DG_ERR_INVALID_ARG, "need epochs >= 1, 1 <= batch <= n, lr > 0, lr_decay > 0");
  cudaError_t e = dg::mlp_train(gas, n, e_dev, Y_dev, T_dev, *o, init, history);
  if (e != cudaSuccess) return cuda_fail(e, "MLP training");
  return DG_OK;
}

int dg_mlp_guess(dg_gas gas, int64_t n, const double* q, double* T, void* stream) {
  if (!gas) return fail(DG_ERR_INVALID_ARG, "NULL gas");
  if (!gas->has_mlp) return fail(DG_ERR_INVALID_ARG, "the gas has no MLP");
  if (n < 0) return fail(DG_ERR_INVALID_ARG, "n must be >= 0");
  if (n == 0) return DG_OK;
  if (!q || !T) return fail(DG_ERR_INVALID_ARG, "NULL pointer");
  cudaError_t e = dg::launch_temperature_mlp(gas, n, q, T, nullptr, 1, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "MLP guess kernel");
  return DG_OK;
}

}  // extern "C"

namespace dg {

int device_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

int resident_blocks(const void* fn, int threads, size_t dyn_smem, int tmem_cols) {
  cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  int dev = 0, smem_sm = 0, regs_sm = 0, thr_sm = 0, blk_sm = 0, reserved = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  const int warps = (threads + 31) / 32;
  const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;  // allocated per warp in units of 256
  int n = blk_sm > 0 ? blk_sm : 1;
  if (regs_warp > 0) n = std::min(n, regs_sm / (regs_warp * warps));
  n = std::min(n, smem_sm / (int)(dyn_smem + fa.sharedSizeBytes + (size_t)reserved));
  n = std::min(n, thr_sm / (warps * 32));
  if (tmem_cols > 0) n = std::min(n, 512 / tmem_cols);
  return std::max(n, 1);
}

}  // namespace dg
