// Batched form: many independent cases of uneven size and order advanced together,
// one CUDA-graph launch per RK4 step.
//
// The cases are grouped by (order, physics).  Each group's kernels are persistent
// over a device work list of (case, first element) tiles of 25 elements (the 128 rows of
// one tensor-core tile), so one launch per group and pass serves all its cases; a step is
// 5 stages x (primitives pass, BR1 pass per viscous group, right-hand side per group) plus
// a copy of each case's result back into its state buffer, captured once into a graph.
// The block size of each group's kernels (threads per tile, i.e. nodes per thread against
// resident blocks per SM) is chosen at creation by timing the compiled candidates on the
// batch's own cases (the autotuner).  The paper's nearest counterpart is its
// concatenation of outlined calls into fewer, larger kernels (Sec. 4.2.4) and the
// launch-overhead floor it reports (Sec. 5.2).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "dg_tc.cuh"

namespace dg {
namespace {

using mixk::MixedCase;

struct Group {
  int N = 0, phys = 0, epb = 0, nt = 0;  // elements per work item (25), threads per block
  int2* work = nullptr;
  int nwork = 0;
  std::vector<int> cases;
};

// Persistent grid of a kernel: resident blocks per SM x SMs, at most one block per work item.
template <typename K>
int persistent_grid(K kernel, int threads, size_t smem, int tmem_cols, int nwork) {
  return std::max(1, std::min(nwork, resident_blocks((const void*)kernel, threads, smem, tmem_cols) * device_sms()));
}

// Right-hand side + RK stage of a group on the tensor cores (tcgen05), tiles of 25 elements,
// NT threads per block.
template <int N, int NT, int PHYS>
cudaError_t rhs_batched_t(const Group& g, const MixedCase* cases, const MixedOps& mx, const int32_t* fmask, int stage,
                          double a, double b, unsigned* status, cudaStream_t s) {
  using C = tc::Cfg<N, NT>;
  auto kern_fn = tc::rhs_tc_batched<N, NT, PHYS>;
  cudaError_t e = cudaFuncSetAttribute(kern_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  if (e != cudaSuccess) return e;
  const int grid = persistent_grid(kern_fn, NT, C::SMEM, C::TMEM_COLS, g.nwork);
  kern_fn<<<grid, NT, C::SMEM, s>>>(cases, g.work, g.nwork, reinterpret_cast<const uint4*>(mx.tc_rhs), fmask, stage,
                                    a, b, status);
  return cudaGetLastError();
}

// BR1 pass of a group on the tensor cores (tcgen05), tiles of 25 elements, NT threads per block.
template <int N, int NT>
cudaError_t vis_batched_t(const Group& g, const MixedCase* cases, const MixedOps& mx, const int32_t* fmask, int stage,
                          unsigned* status, cudaStream_t s) {
  using C = tc::VCfg<N, NT>;
  auto kern_fn = tc::vis_tc_batched<N, NT>;
  cudaError_t e = cudaFuncSetAttribute(kern_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  if (e != cudaSuccess) return e;
  const int grid = persistent_grid(kern_fn, NT, C::SMEM, C::TMEM_COLS, g.nwork);
  kern_fn<<<grid, NT, C::SMEM, s>>>(cases, g.work, g.nwork, reinterpret_cast<const uint4*>(mx.tc_vis), fmask, stage,
                                    status);
  return cudaGetLastError();
}

// Compiled candidates (threads per 25-element tile) per order; the first is the single-case
// default.  Fewer threads: more resident blocks, more nodes per thread; more threads: one
// node (or face node) per thread and fewer blocks.  Both passes use the same lists.
const std::vector<int>& nt_candidates(int N) {
  static const std::vector<int> c1{128, 256}, c2{256, 128}, c3{256, 512}, c4{448, 896};
  return N == 1 ? c1 : N == 2 ? c2 : N == 3 ? c3 : c4;
}

cudaError_t launch_rhs_group(const Group& g, const MixedCase* cases, const MixedOps& mx, const int32_t* fmask,
                             int stage, double a, double b, unsigned* status, cudaStream_t s) {
  const bool ns = g.phys == kern::NAVIER_STOKES;
#define DG_RHS(NN, TT)                                                                                \
  if (g.N == NN && g.nt == TT)                                                                        \
    return ns ? rhs_batched_t<NN, TT, kern::NAVIER_STOKES>(g, cases, mx, fmask, stage, a, b, status, s) \
              : rhs_batched_t<NN, TT, kern::EULER>(g, cases, mx, fmask, stage, a, b, status, s);
  DG_RHS(1, 128)
  DG_RHS(1, 256)
  DG_RHS(2, 256)
  DG_RHS(2, 128)
  DG_RHS(3, 256)
  DG_RHS(3, 512)
  DG_RHS(4, 448)
  DG_RHS(4, 896)
#undef DG_RHS
  return cudaErrorInvalidValue;
}

cudaError_t launch_vis_group(const Group& g, const MixedCase* cases, const MixedOps& mx, const int32_t* fmask,
                             int stage, unsigned* status, cudaStream_t s) {
#define DG_VIS(NN, TT) \
  if (g.N == NN && g.nt == TT) return vis_batched_t<NN, TT>(g, cases, mx, fmask, stage, status, s);
  DG_VIS(1, 128)
  DG_VIS(1, 256)
  DG_VIS(2, 256)
  DG_VIS(2, 128)
  DG_VIS(3, 256)
  DG_VIS(3, 512)
  DG_VIS(4, 448)
  DG_VIS(4, 896)
#undef DG_VIS
  return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace dg

struct dg_batch_s {
  std::vector<dg_mesh> meshes;
  std::vector<dg::mixk::MixedCase> cases;
  dg::mixk::MixedCase* dcases = nullptr;
  std::vector<double*> owned;  // work state and RK register of every case
  std::vector<dg::Group> rhs, vis;
  int2* prims_work = nullptr;
  int prims_nwork = 0;
  unsigned* status = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  double tune_ms[4][2][4] = {};  // [order-1][physics][candidate] right-hand-side tile timings
  double tune_vis_ms[4][4] = {};
};

namespace {

using dg::fail;
using dg::cuda_fail;

const dg::MeshDev& mdev(const dg_batch_s* b, int N) {
  for (dg_mesh m : b->meshes)
    if (m->d.N == N) return m->d;
  return b->meshes[0]->d;
}

cudaError_t build_work(dg::Group& g, const dg_batch_s* b) {
  std::vector<int2> w;
  for (int ci : g.cases)
    for (int e0 = 0; e0 < b->cases[ci].K; e0 += g.epb) w.push_back(make_int2(ci, e0));
  cudaFree(g.work);
  g.work = nullptr;
  g.nwork = (int)w.size();
  cudaError_t e = cudaMalloc((void**)&g.work, sizeof(int2) * std::max<size_t>(w.size(), 1));
  if (e == cudaSuccess && !w.empty())
    e = cudaMemcpy(g.work, w.data(), sizeof(int2) * w.size(), cudaMemcpyHostToDevice);
  return e;
}

cudaError_t launch_prims(dg_batch_s* b, int stage, cudaStream_t s) {
  const int grid = std::min(b->prims_nwork, dg::device_sms() * 8);
  dg::mixk::prims_batched<<<std::max(grid, 1), 256, 0, s>>>(b->dcases, b->prims_work, b->prims_nwork, stage,
                                                             b->status);
  return cudaGetLastError();
}

cudaError_t launch_stage(dg_batch_s* b, int stage, cudaStream_t s) {
  cudaError_t e = launch_prims(b, stage, s);
  for (const dg::Group& g : b->vis)
    if (e == cudaSuccess) {
      const dg::MeshDev& m = mdev(b, g.N);
      e = dg::launch_vis_group(g, b->dcases, m.mx, m.fmask, stage, b->status, s);
    }
  for (const dg::Group& g : b->rhs)
    if (e == cudaSuccess) {
      const dg::MeshDev& m = mdev(b, g.N);
      e = dg::launch_rhs_group(g, b->dcases, m.mx, m.fmask, stage, dg::kRK4A[stage], dg::kRK4B[stage], b->status, s);
    }
  return e;
}

// Average ms of `reps` launches of f on stream s (after one warm-up launch).
template <typename F>
double time_launches(F f, cudaStream_t s, int reps = 3) {
  cudaEvent_t a, z;
  cudaEventCreate(&a);
  cudaEventCreate(&z);
  f();
  cudaEventRecord(a, s);
  for (int i = 0; i < reps; ++i) f();
  cudaEventRecord(z, s);
  cudaEventSynchronize(z);
  float ms = 0;
  cudaEventElapsedTime(&ms, a, z);
  cudaEventDestroy(a);
  cudaEventDestroy(z);
  return ms / reps;
}

void free_batch(dg_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (auto& g : b->rhs) cudaFree(g.work);
  for (auto& g : b->vis) cudaFree(g.work);
  for (double* p : b->owned) cudaFree(p);
  cudaFree(b->prims_work);
  cudaFree(b->dcases);
  cudaFree(b->status);
  delete b;
}

}  // namespace

extern "C" {

int dg_batch_create(const dg_batch_case* in, int32_t ncases, int32_t flags, dg_batch* out) {
  if (!in || !out || ncases < 1) return fail(DG_ERR_INVALID_ARG, "need cases and an output handle");
  *out = nullptr;
  for (int i = 0; i < ncases; ++i) {
    const dg_batch_case& c = in[i];
    if (!c.mesh || !c.gas || !c.q_dev) return fail(DG_ERR_INVALID_ARG, "case " + std::to_string(i) + ": NULL field");
    if (!c.mesh->d.ops) return fail(DG_ERR_INVALID_ARG, "case " + std::to_string(i) + ": host-only mesh");
    if (c.mesh->d.av.eps0 > 0)
      return fail(DG_ERR_UNSUPPORTED, "case " + std::to_string(i) + ": artificial viscosity runs in the FP64 form");
    if (c.mesh->d.oi_q > 0)
      return fail(DG_ERR_UNSUPPORTED, "case " + std::to_string(i) + ": over-integration runs in the FP64 form");
    if (c.mesh->d.inflow_faces > 0 && c.mesh->d.inflow_nvar != 5)
      return fail(DG_ERR_INVALID_ARG, "case " + std::to_string(i) +
                                          ": the mesh has inflow faces: set the inflow state with dg_mesh_set_inflow");
    if (c.gas->p.model != DG_GAS_PERFECT)
      return fail(DG_ERR_UNSUPPORTED, "case " + std::to_string(i) + ": the batched form needs a perfect gas");
    if (!std::isfinite(c.dt)) return fail(DG_ERR_INVALID_ARG, "case " + std::to_string(i) + ": dt must be finite");
    for (int j = 0; j < i; ++j)
      if (in[j].mesh->d.N == c.mesh->d.N &&
          (in[j].mesh->ops.Dr != c.mesh->ops.Dr || in[j].mesh->ops.LIFT != c.mesh->ops.LIFT))
        return fail(DG_ERR_INVALID_ARG, "cases of one order must share their reference operators");
  }
  dg_batch_s* b = new dg_batch_s();
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < ncases && e == cudaSuccess; ++i) {
    const dg::MeshDev& m = in[i].mesh->d;
    const dg::GasParams& gp = in[i].gas->p;
    const size_t n = (size_t)5 * m.K * m.Np;
    double *work = nullptr, *k = nullptr;
    e = cudaMalloc((void**)&work, sizeof(double) * n);
    if (e == cudaSuccess) b->owned.push_back(work);
    if (e == cudaSuccess) e = cudaMalloc((void**)&k, sizeof(double) * n);
    if (e == cudaSuccess) b->owned.push_back(k);
    if (e != cudaSuccess) break;
    dg::mixk::MixedCase c = dg::make_mixed_case(m, gp, in[i].q_dev, work, k, in[i].dt);
    b->cases.push_back(c);
    b->meshes.push_back(in[i].mesh);
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->dcases, sizeof(dg::mixk::MixedCase) * ncases);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->dcases, b->cases.data(), sizeof(dg::mixk::MixedCase) * ncases, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->status, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(b->status, 0, sizeof(unsigned));
  // primitives pass work list
  if (e == cudaSuccess) {
    std::vector<int2> pw;
    for (int i = 0; i < ncases; ++i)
      for (int n0 = 0; n0 < b->cases[i].K * b->cases[i].Np; n0 += dg::mixk::PRIMS_CHUNK) pw.push_back(make_int2(i, n0));
    b->prims_nwork = (int)pw.size();
    e = cudaMalloc((void**)&b->prims_work, sizeof(int2) * pw.size());
    if (e == cudaSuccess) e = cudaMemcpy(b->prims_work, pw.data(), sizeof(int2) * pw.size(), cudaMemcpyHostToDevice);
  }
  // groups with their default tiles
  if (e == cudaSuccess) {
    std::map<std::pair<int, int>, dg::Group> rg;
    std::map<int, dg::Group> vg;
    for (int i = 0; i < ncases; ++i) {
      const int N = b->cases[i].K ? in[i].mesh->d.N : 0;
      const int phys = in[i].gas->p.mu > 0 ? dg::kern::NAVIER_STOKES : dg::kern::EULER;
      dg::Group& g = rg[{N, phys}];
      g.N = N;
      g.phys = phys;
      g.epb = dg::tc::Cfg<1>::E;
      g.nt = dg::nt_candidates(N)[0];
      g.cases.push_back(i);
      if (phys == dg::kern::NAVIER_STOKES) {
        dg::Group& v = vg[N];
        v.N = N;
        v.phys = phys;
        v.epb = dg::tc::VCfg<1>::E;
        v.nt = dg::nt_candidates(N)[0];
        v.cases.push_back(i);
      }
    }
    for (auto& kv : rg) b->rhs.push_back(kv.second);
    for (auto& kv : vg) b->vis.push_back(kv.second);
    for (auto& g : b->rhs)
      if (e == cudaSuccess) e = build_work(g, b);
    for (auto& g : b->vis)
      if (e == cudaSuccess) e = build_work(g, b);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  // autotune: time each group's compiled block sizes on stage 0 (reads the cases' states, writes
  // only work buffers) and keep the fastest
  if (e == cudaSuccess && (flags & DG_BATCH_AUTOTUNE)) {
    e = launch_stage(b, 0, b->cap);
    for (auto& g : b->vis) {
      double best = 1e300;
      int best_nt = g.nt;
      const auto& cand = dg::nt_candidates(g.N);
      for (size_t ci = 0; ci < cand.size() && e == cudaSuccess; ++ci) {
        g.nt = cand[ci];
        const dg::MeshDev& m = mdev(b, g.N);
        const double ms =
            time_launches([&] { return dg::launch_vis_group(g, b->dcases, m.mx, m.fmask, 0, b->status, b->cap); }, b->cap);
        b->tune_vis_ms[g.N - 1][ci] = ms;
        if (ms < best) {
          best = ms;
          best_nt = cand[ci];
        }
      }
      g.nt = best_nt;
    }
    for (auto& g : b->rhs) {
      double best = 1e300;
      int best_nt = g.nt;
      const auto& cand = dg::nt_candidates(g.N);
      for (size_t ci = 0; ci < cand.size() && e == cudaSuccess; ++ci) {
        g.nt = cand[ci];
        const dg::MeshDev& m = mdev(b, g.N);
        const double ms = time_launches(
            [&] {
              return dg::launch_rhs_group(g, b->dcases, m.mx, m.fmask, 0, dg::kRK4A[0], dg::kRK4B[0], b->status, b->cap);
            },
            b->cap);
        b->tune_ms[g.N - 1][g.phys == dg::kern::NAVIER_STOKES][ci] = ms;
        if (ms < best) {
          best = ms;
          best_nt = cand[ci];
        }
      }
      g.nt = best_nt;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->cap);
    if (e == cudaSuccess) e = cudaMemset(b->status, 0, sizeof(unsigned));
  }
  // capture one RK4 step: 5 stages, then each case's result (stage 4 writes q[1]) back into q[0]
  if (e == cudaSuccess) {
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    for (int st = 0; st < 5 && e == cudaSuccess; ++st) e = launch_stage(b, st, b->cap);
    for (int i = 0; i < ncases && e == cudaSuccess; ++i) {
      const size_t n = (size_t)5 * b->cases[i].K * b->cases[i].Np;
      e = cudaMemcpyAsync(b->cases[i].q[0], b->cases[i].q[1], sizeof(double) * n, cudaMemcpyDeviceToDevice, b->cap);
    }
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
  }
  if (e != cudaSuccess) {
    free_batch(b);
    return cuda_fail(e, "batch creation");
  }
  *out = b;
  return DG_OK;
}

int dg_batch_step(dg_batch b, int32_t steps, void* stream) {
  if (!b) return fail(DG_ERR_INVALID_ARG, "NULL batch");
  if (steps < 0) return fail(DG_ERR_INVALID_ARG, "steps must be >= 0");
  for (int i = 0; i < steps; ++i) {
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  }
  return DG_OK;
}

int dg_batch_tiles(dg_batch b, int32_t* rhs_tiles, int32_t* viscous_tiles, double* rhs_tune_ms) {
  if (!b) return fail(DG_ERR_INVALID_ARG, "NULL batch");
  if (rhs_tiles)
    for (int i = 0; i < 8; ++i) rhs_tiles[i] = 0;
  if (viscous_tiles)
    for (int i = 0; i < 4; ++i) viscous_tiles[i] = 0;
  for (const auto& g : b->rhs)
    if (rhs_tiles) rhs_tiles[(g.N - 1) * 2 + (g.phys == dg::kern::NAVIER_STOKES)] = g.nt;
  for (const auto& g : b->vis)
    if (viscous_tiles) viscous_tiles[g.N - 1] = g.nt;
  if (rhs_tune_ms) std::memcpy(rhs_tune_ms, b->tune_ms, sizeof(b->tune_ms));
  return DG_OK;
}

int dg_batch_status(dg_batch b, uint32_t* bits, int reset) {
  if (!b || !bits) return fail(DG_ERR_INVALID_ARG, "NULL batch or bits");
  cudaError_t e = cudaDeviceSynchronize();
  unsigned v = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&v, b->status, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && reset) e = cudaMemset(b->status, 0, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_fail(e, "batch status");
  *bits = v;
  return DG_OK;
}

int dg_batch_free(dg_batch b) {
  if (!b) return DG_OK;
  cudaDeviceSynchronize();
  free_batch(b);
  return DG_OK;
}

}  // extern "C"
