// Internal declarations of libdg (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dg.h"

namespace dg {

// ---- errors (thread-local message, see dg_last_error) -----------------------
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

// ---- host-side builders -----------------------------------------------------
struct RefOps {
  int N = 0, Np = 0, Nfp = 0;
  std::vector<double> Dr, Ds, Dt;  // [Np][Np] row-major
  std::vector<double> LIFT;        // [Np][4 Nfp]
  std::vector<int32_t> Fmask;      // [4][Nfp]
  std::vector<double> modal;       // [Np][Np]: orthonormal (PKDO) coefficients from nodal values,
                                   // the ntop modes of total degree N in the last rows
  int ntop = 0;
  std::vector<double> wq;          // [Np]: integral of each nodal basis function over the element
};

// Reference operators of order N on the given nodes (refops.cpp).
bool build_ref_ops(int N, const double* nodes, RefOps& out, std::string& err);

// Over-integration of the volume term (refops.cpp): the Stroud conical-product rule with q
// Gauss-Jacobi points per collapsed direction on the reference tetrahedron, the nodal basis at its
// points and the weak-form operators M^-1 D_a^T.
struct OverintOps {
  int q = 0, Ng = 0;                // points per direction, q^3 points
  std::vector<double> rst, w;       // [Ng][3] points, [Ng] weights (point (k q + j) q + i of (a_i, b_j, c_k))
  // sum-factorised form: the orthonormal modes psi_pqr = A_p(a) B_pq(b) C_pqr(c) at the rule's
  // collapsed coordinates (modes in (p, q, r) order, p outermost; pq pairs in (p, q) order); the
  // weighted copies carry half the 1-D Gauss-Jacobi weight each, so that their product is w_g
  std::vector<double> A, Aw;        // [N+1][q]: A_p(a_i)
  std::vector<double> B, Bw;        // [(N+1)(N+2)/2][q]: B_pq(b_j)
  std::vector<double> C, Cw;        // [Np][q]: C_pqr(c_k)
  std::vector<double> VinvT;        // [Np(j)][Np(n)]: (V_o^-1)[n][j], nodal values -> mode n
  std::vector<double> VoT;          // [Np(n)][Np(i)]: V_o[i][n], modes -> nodal values
  // the modal derivative matrices Dh_a = V_o^-1 D_a V_o by column, zeros left out, the columns in
  // the order Dh_col (longest first): entries Dh_ptr[s] .. Dh_ptr[s+1] - 1 hold Dh_a[m][n] of
  // column n = Dh_col[s] in Dh_val, with a Np + m in Dh_idx
  std::vector<int> Dh_ptr, Dh_idx, Dh_col;
  std::vector<double> Dh_val;
};
bool tet_quadrature(int q, std::vector<double>& rst, std::vector<double>& w, std::string& err);
bool build_overint_ops(int N, const double* nodes, int q, OverintOps& out, std::string& err);

// Affine geometric factors, geo[K][DG_GEO_STRIDE] (mesh.cpp).
bool build_geometry(int K, const double* verts, std::vector<double>& geo, std::string& err);

// Periodic face-node connectivity vmapP[K][4 Nfp] (mesh.cpp).
// face_bc [K][4] (may be null): DG_BC_* code of the faces without a partner; their face nodes
// get vmapP = -code.
// partner_out (optional) receives the face pairing [4K]: 4 k2 + f2, -1 at boundary faces.
bool build_connectivity(int K, const double* verts, const double period[3], const RefOps& ops,
                        const double* ref_nodes, const int32_t* face_bc, std::vector<int32_t>& vmapP,
                        std::string& err, std::vector<int>* partner_out = nullptr);

// The same from a face pairing given by the caller (EToE / EToF [K][4], -1 for a face without a
// partner; the pairing must be symmetric).
bool build_connectivity_from_faces(int K, const double* verts, const double period[3], const RefOps& ops,
                                   const double* ref_nodes, const int32_t* face_bc, const int32_t* EToE,
                                   const int32_t* EToF, std::vector<int32_t>& vmapP, std::string& err,
                                   std::vector<int>& partner);
// Checks of caller-supplied tables (mesh.cpp): a vmapP (range, one partner face per face, coincident
// partner nodes modulo the period, symmetry, boundary codes as in face_bc; partner [4K] receives the
// face pairing), global vertex numbers against the pairing, reference operators (finite, D
// annihilates constants, Fmask nodes on their faces), geometric factors (finite, J > 0, unit
// normals, Fscale > 0).
bool check_connectivity(int K, const double* verts, const double period[3], const RefOps& ops,
                        const double* ref_nodes, const int32_t* face_bc, const int32_t* vmapP,
                        std::vector<int>& partner, std::string& err);
bool check_vertex_numbers(int K, const int32_t* EToV, const std::vector<int>& partner, std::string& err);
bool check_ref_ops(int N, const double* ref_nodes, const double* Dr, const double* Ds, const double* Dt,
                   const double* LIFT, const int32_t* Fmask, std::string& err);
bool check_geometry(int K, const double* geo, std::string& err);

// ---- device-side parameter blocks -------------------------------------------
struct GasParams {  // passed to kernels by value
  int model;        // DG_GAS_PERFECT / DG_GAS_NASA7
  int ns;           // species (NASA-7), 0 for a perfect gas
  double gamma, R, mu, Pr, kappa, cp;
  double Rk[DG_MAX_SPECIES];
  double a[DG_MAX_SPECIES][7];
  // NASA-7: species k's share of the internal-energy quintic per unit mass fraction,
  // e_k(T) = sum_j fc[k][j] T^j = R_k (a6 + (a1 - 1) T + a2/2 T^2 + a3/3 T^3 + a4/4 T^4 + a5/5 T^5)
  double fc[DG_MAX_SPECIES][6];
  // the same coefficients and R_k as float pairs (hi = the value rounded to FP32, lo = the rest
  // rounded to FP32), for the mixed-precision form's fold on the FP32 pipe: [k][0..5] = fc[k][j],
  // [k][6] = R_k
  float2 fc2[DG_MAX_SPECIES][7];
  double newton_tol;
  int newton_max_it;
  double Sc;        // NASA-7 with viscosity: Schmidt number, rho D = mu / Sc
};

// Split-BF16 operator tables of the mixed-precision path (built at upload): three terms
// (x = hi + mid + lo, each bf16), each the image of the operator in the UMMA K-major
// shared-memory layout that the tcgen05 kernels copy in as is.
struct MixedOps {
  unsigned char* tc_rhs = nullptr;  // tcgen05 operator table: 3 BF16 terms of [-Dr | -Ds | -Dt | LIFT]
                                    // in the UMMA K-major layout (chunks of round16(Np) columns)
  unsigned char* tc_vis = nullptr;  // tcgen05 BR1 table: rows (a, i), [D_a | 1/2 sum_f c_fa LIFT_f]
};

// Artificial-viscosity parameters (eps0 > 0: on).
struct AvParams {
  double eps0, s0, kappa;
};

// Boundary data passed to the FP64 kernels by value: the conserved state of DG_BC_INFLOW faces
// and, for a mixture, (1/rho, p, c) of that state at its temperature T_in (the root of
// e(T) = e_in, solved on the host before each right-hand side of a NASA-7 gas).
struct BcParams {
  double q_in[5 + DG_MAX_SPECIES];
  double prim_in[3];
  double T_in;
};

struct MeshDev {
  int K = 0, N = 0, Np = 0, Nfp = 0;
  int boundary_faces = 0;     // faces carrying a DG_BC_* code
  int inflow_faces = 0;       // of which DG_BC_INFLOW
  int inflow_nvar = 0;        // 0 until dg_mesh_set_inflow
  BcParams bc{};
  // artificial viscosity (dg_mesh_set_av): parameters, modal-analysis matrix, element viscosity
  // [K] and the flux eps grad q_v along x_d, [(5 d + v)][K][Np]
  AvParams av{};
  int ntop = 0;
  double* modal = nullptr;
  double* av_eps = nullptr;
  int* av_list = nullptr;      // [1 + K]: the count, then the elements with eps > 0 (the last indicator pass's)
  double* av_sig = nullptr;
  double* mix_fv = nullptr;  // viscous flux of a mixture, [9 + 3 DG_MAX_SPECIES][K][Np] (on first use)
  MixedOps mx;
  double* ops = nullptr;       // Dr | Ds | Dt | LIFT, row-major
  int32_t* fmask = nullptr;    // [4][Nfp]
  double* geo = nullptr;       // [K][DG_GEO_STRIDE]
  int32_t* vmapP = nullptr;    // [K][4 Nfp]
  double* scratch = nullptr;   // 80 B per node: FP64 form [9][K][Np] viscous flux (BR1 pass 1 output);
                               // mixed form node records (dg_mixed.cuh NodeTables) or mixture tables
  float* geo32 = nullptr;      // [K][DG_GEO_STRIDE] float copy of geo (mixed form)
  unsigned* status = nullptr;  // device status word
  double* wq = nullptr;        // [Np] reference quadrature weights (mass-matrix row sums)
  double* diag = nullptr;      // per-block partials of the global reductions (k_diag.cu)
  double* prim = nullptr;      // FP64 form, perfect gas: [3][K][Np] (1/rho, p, c) of the state being
                               // differentiated, written by the primitives pass before each stage
  // over-integration (dg_mesh_set_overint; oi_q = 0: off): the sum-factorised tables of
  // OverintOps, A | Aw | B | Bw | C | Cw | V_o^-T | V_o^T | Dh_val | Dh_ptr | Dh_idx | Dh_col (the
  // last three as doubles), with oi_nnz entries in Dh
  double* oi_tab = nullptr;
  int oi_q = 0, oi_ng = 0, oi_nnz = 0;
};

// LSRK4 coefficients (Carpenter & Kennedy 1994, five stages, 2N storage).
extern const double kRK4A[5];
extern const double kRK4B[5];

// ---- kernel launchers (kernels_dg.cu, kernels_thermo.cu) ------------------------
// Elements [begin, end) of a launch; end < 0: to the mesh's last element.
struct ElemRange {
  int begin = 0, end = -1;
};
// Right-hand side (rk == false: out = rhs) or fused RK stage (rk == true:
// k <- a k + dt rhs, out = q + b k).  T (may be null for a perfect gas) holds
// the node temperatures of a mixture.  r: the elements evaluated (perfect gas; a mixture
// is always evaluated whole).
cudaError_t launch_rhs(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k,
                       const double* T, bool rk, double a, double b, double dt, cudaStream_t s,
                       ElemRange r = ElemRange());
// Artificial viscosity (k_av.cu): element viscosities of q into eps [K]; the flux eps grad q into
// m.av_sig (from m.av_eps); the right-hand side / RK stage with that flux added.
// list (may be null): m.av_list, refilled with the elements whose eps > 0 for launch_av_flux.
// fp32: the arithmetic in FP32 (the mixed-precision form), else FP64; eps and sigma stay FP64 arrays.
cudaError_t launch_av_sensor(const MeshDev& m, const double* q, double* eps, cudaStream_t s, int* list = nullptr,
                             bool fp32 = false);
// Over-integrated weak-form Euler or Navier-Stokes right-hand side / RK stage of a perfect gas
// (k_oi.cu; Navier-Stokes reads the BR1 viscous flux in m.scratch, artificial viscosity the flux of
// the AV pass in m.av_sig), and whether its tables and one element's work for Ng points fit in a
// block's shared memory at order N.
cudaError_t launch_rhs_overint(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k,
                               bool rk, double a, double b, double dt, cudaStream_t s);
bool overint_fits(int N, int q, int nnz, bool visc, bool av);
cudaError_t launch_av_flux(const MeshDev& m, const GasParams& g, const double* q, cudaStream_t s, bool fp32 = false);
// Mixture with viscosity (k_mixns.cu): BR1 gradients of (rho, rho u, T, Y_k) and the viscous
// flux with species diffusion into m.mix_fv; the right-hand side / RK stage that subtracts it.
cudaError_t launch_viscous_mixture(const MeshDev& m, const GasParams& g, const double* q, const double* T,
                                   cudaStream_t s);
cudaError_t launch_rhs_mixture_ns(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k,
                                  const double* T, bool rk, double a, double b, double dt, cudaStream_t s);
cudaError_t launch_rhs_av(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k, bool rk,
                          double a, double b, double dt, cudaStream_t s);
// Mixed-precision path: primitives pass (k_mixed.cu); operator tables, tensor-core right-hand
// side / RK stage and its BR1 pass (k_tc.cu).
void free_mixed_ops(MeshDev& m);
cudaError_t launch_prims_mixed(const MeshDev& m, const GasParams& g, const double* q, cudaStream_t s);
cudaError_t build_tc_ops(MeshDev& m, const RefOps& ops);
// wait_polls: polls per bounded mbarrier wait (0 = the default bound; a small value is a test aid
// that makes the waits run out).
cudaError_t launch_rhs_tc(const MeshDev& m, const GasParams& g, const double* q, double* out, double* k, bool rk,
                          double a, double b, double dt, cudaStream_t s, int wait_polls = 0);
cudaError_t launch_viscous_tc(const MeshDev& m, const GasParams& g, const double* q, cudaStream_t s,
                              int wait_polls = 0);
// BR1 pass 1: viscous flux of a perfect gas into m.scratch, for the elements r.
cudaError_t launch_viscous_flux(const MeshDev& m, const GasParams& g, const double* q, cudaStream_t s,
                                ElemRange r = ElemRange());
// Per-node (1/rho, p, c) of a perfect-gas state into m.prim (k_ns.cu); the FP64 viscous and
// right-hand-side kernels of the perfect gas read them.
cudaError_t launch_prims_fp64(const MeshDev& m, const GasParams& g, const double* q, cudaStream_t s,
                              ElemRange r = ElemRange());
// Global reductions (k_diag.cu): a fixed grid of kDiagBlocks blocks writes per-block partials
// into MeshDev::diag, one block combines them in a fixed order.
constexpr int kDiagBlocks = 512, kDiagThreads = 256, kDiagMaxV = 5 + DG_MAX_SPECIES;
constexpr size_t kDiagPartialBytes = sizeof(double) * kDiagBlocks * kDiagMaxV;
// Outputs of the mixed-precision form that the temperature solve also writes (rec null: none):
// the node records [n][4] float4 {rho_hi, rho u, rho v, rho w}, {rho E, p_hi, p_lo, c},
// {rho Y_1..4}, {rho Y_5..8}; rho <= 0 or p <= 0 sets DG_STATUS_NONPHYSICAL in *status.
struct MixturePrims {
  float4* rec = nullptr;      // mixed form: the node records
  float4* lo = nullptr;       // mixed form: [n] low halves of momentum and energy
  double* prim = nullptr;     // FP64 form: [3][n] 1/rho, p, c at the converged temperature
  unsigned* status = nullptr;
};
// The mesh scratch's mixture tables (k_mixed.cu).
MixturePrims mixture_prims_out(const MeshDev& m);
// Mixture temperature (Newton).  seed_mode: DG_TSEED_*; nvar = 5 + ns; q is [nvar][n].
cudaError_t launch_temperature(const GasParams& g, int64_t n, const double* q, double* T, int32_t* iters,
                               int seed_mode, double t_const, unsigned* status, cudaStream_t s,
                               const MixturePrims& mp = MixturePrims());
cudaError_t launch_mixture_energy(const GasParams& g, int64_t n, const double* T, const double* Y, double* e,
                                  cudaStream_t s);

// SMs of the current device.
int device_sms();
// Blocks of kernel fn (threads per block, dynamic shared memory, TMEM columns allocated per
// block) resident on one SM at once, from its registers, shared memory, threads and tensor
// memory (512 columns per SM) against the SM's limits; sets the kernel's shared memory
// carveout to the maximum.  A persistent kernel's grid is this times device_sms().
int resident_blocks(const void* fn, int threads, size_t dyn_smem, int tmem_cols = 0);

}  // namespace dg

namespace dg {
// Event pairs bracketing kernel launches, resolved lazily (dg_mesh_kernel_times).
struct KernelTimer {
  bool enabled = false;
  std::vector<cudaEvent_t> pool;                                // idle events
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[DG_NUM_KERNELS];
  double ms[DG_NUM_KERNELS] = {};
  int64_t count[DG_NUM_KERNELS] = {};
};
}  // namespace dg

struct dg_mesh_s {
  dg::MeshDev d;
  dg::KernelTimer timer;
  dg::RefOps ops;
  std::vector<int32_t> vmapP;
  std::vector<double> geo;
  std::vector<int> partner;  // [4 K]: 4 k2 + f2 of each face's partner, -1 at boundary faces
  std::vector<double> ref_nodes;  // [Np][3] reference nodes given at upload
  int device = 0;
};

struct dg_gas_s {
  dg::GasParams p;
  unsigned* status = nullptr;
  int device = 0;
  // learned temperature guess
  bool has_mlp = false;
  float* mlp_theta = nullptr;  // [DG_MLP_PARAMS] fp32
  void* mlp_w1h = nullptr;     // fp16 [64][16]
  void* mlp_w2h = nullptr;     // fp16 [64][64]
  dg_mlp_norm mlp_norm{};
};

namespace dg {
// k_mlp.cu
// wait_polls: polls per mbarrier wait of the inference MMAs (0 = the default bound).
cudaError_t launch_temperature_mlp(dg_gas gas, int64_t n, const double* q, double* T, int32_t* iters, int guess_only,
                                   cudaStream_t s, const MixturePrims& mp = MixturePrims(), int wait_polls = 0);
cudaError_t mlp_set_params(dg_gas gas, const float* theta_host, const dg_mlp_norm& nrm);
cudaError_t mlp_loss_grad(int64_t n, const float* theta, const float* X, const float* t, float* grad, float* loss,
                          cudaStream_t s);
// One Adam step (step number t >= 1) on the DG_MLP_PARAMS parameters; zeroes grad.
cudaError_t mlp_adam_step(int t, float lr, float* theta, float* grad, float* m, float* v, cudaStream_t s);
cudaError_t mlp_train(dg_gas gas, int64_t n, const double* e_dev, const double* Y_dev, const double* T_dev,
                      const dg_mlp_train_opts& o, const float* init_host, float* history);
}  // namespace dg
