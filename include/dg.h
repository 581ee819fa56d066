/*
 * dg.h - C ABI of libdg: the nodal discontinuous-Galerkin right-hand side and
 * low-storage RK4 stage for compressible (multi-species, viscous) flow on
 * tetrahedral meshes, on one GB300 GPU (sm_103a).
 *
 * Method (arXiv 2512.17101, MIRGE-Com):
 *   - DOFs are local to each element and stored as an array per field, the
 *     element-major nodal layout of Sec. 1, Fig. 1;
 *   - nodal DG on tetrahedra (Sec. 1) with full assembly of the reference
 *     operators (Sec. 5.2); Euler equations with a Lax-Friedrichs flux
 *     (Sec. 5.2); compressible Navier-Stokes (Sec. 5.3) with BR1 gradients;
 *     perfect gas gamma = 1.4 (Sec. 5.3) or a multi-species NASA-7 mixture
 *     (Sec. 4, Sec. 5) whose temperature comes from a per-node Newton solve;
 *   - explicit fourth-order Runge-Kutta (Sec. 5.2), here the five-stage
 *     2N-storage scheme of Carpenter & Kennedy.
 * The paper names these pieces without formulas; the library implements the
 * textbook forms (Hesthaven & Warburton) that its Sec. 1 cites.
 *
 * Conventions shared by all calls
 *   - State q is float64 [V][K][Np], node index fastest ("field, element,
 *     node"), with V = 5 + nspecies: rho, rho u, rho v, rho w, rho E, rho Y_k.
 *     The right-hand side, the RK register k and the stage output use the
 *     same layout.  Temperature fields are float64 [K][Np].
 *   - Reference tetrahedron: vertices (-1,-1,-1), (1,-1,-1), (-1,1,-1),
 *     (-1,-1,1); element vertex m is the image of reference vertex m.
 *   - Pointers named *_dev are device pointers owned by the caller; the
 *     library never frees or retains them beyond the call.  Pointers named
 *     *_host are host pointers read during the call only.
 *   - Calls that take a stream enqueue work asynchronously on it (a
 *     cudaStream_t passed as void*; NULL = the legacy default stream) and
 *     return after launching.  Errors found on the device (non-physical
 *     state, Newton without convergence) are recorded in a status word of
 *     the handle and read with dg_mesh_status / dg_gas_status.
 *   - Every call returns DG_OK (0) or a negative DG_ERR_* code; the message
 *     of the last error on the calling thread is dg_last_error().  The
 *     library never prints, exits or traps.
 */
#ifndef DG_H_
#define DG_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define DG_OK 0
#define DG_ERR_INVALID_ARG (-1)
#define DG_ERR_CUDA (-2)
#define DG_ERR_NO_CONVERGENCE (-3)
#define DG_ERR_NONPHYSICAL (-4)
#define DG_ERR_TIMEOUT (-5)
#define DG_ERR_OOM (-6)
#define DG_ERR_UNSUPPORTED (-7)

/* bits of the device status word (dg_mesh_status / dg_gas_status) */
#define DG_STATUS_NONPHYSICAL 1u      /* rho <= 0 or p <= 0 met at some node */
#define DG_STATUS_NO_CONVERGENCE 2u   /* a Newton temperature solve hit its cap */
#define DG_STATUS_TIMEOUT 4u          /* a tensor-core kernel's wait on its own MMA completion hit
                                         its iteration bound; that kernel stopped early and its
                                         output is incomplete */

/* ---- limits -------------------------------------------------------------- */
#define DG_MAX_ORDER 4
#define DG_MAX_SPECIES 8
#define DG_MAX_OVERINT_POINTS 12   /* Gauss-Jacobi points per collapsed direction          */
#define DG_OVERINT_DEFAULT (-1)    /* dg_mesh_set_overint: ceil(3N/2) points per direction */

typedef struct dg_mesh_s* dg_mesh;
typedef struct dg_gas_s* dg_gas;

/* ---- mesh ---------------------------------------------------------------- */
typedef struct {
  int32_t K;                 /* number of tetrahedra, >= 1                        */
  int32_t N;                 /* polynomial order, 1..DG_MAX_ORDER                 */
  const double* ref_nodes;   /* host [Np][3]: (r,s,t) of the reference nodes; the  */
                             /* face nodes of each face must match those of the   */
                             /* neighbouring face (e.g. equispaced lattice)        */
  const double* vertices;    /* host [K][4][3]: vertex coordinates per element,   */
                             /* unwrapped across periodic seams; positive volume  */
  double period[3];          /* periodic box lengths; 0 = not periodic along it    */
  int32_t flags;             /* DG_MESH_* bits                                     */
  const int32_t* face_bc;    /* host [K][4] or NULL: DG_BC_* code of each face that */
                             /* has no partner, 0 on paired faces (face f has the   */
                             /* vertex triple 012, 013, 123, 023 for f = 0..3)      */
  /* Optional tables of the caller (Sec. 1 Fig. 1 and Sec. 4.1.2: element-local arrays plus
   * connectivity data).  NULL: the library builds the table, as described at dg_mesh_upload.
   * Every table given is checked on the host and copied; a malformed one is DG_ERR_INVALID_ARG. */
  const int32_t* EToV;       /* host [K][4]: global vertex numbers (periodic images     */
                             /* share a number); checked against the face pairing:     */
                             /* paired faces have the same three vertex numbers         */
  const int32_t* EToE;       /* host [K][4] with EToF: the element and face (0..3)       */
  const int32_t* EToF;       /* paired with each face, -1 in EToE for a face without a  */
                             /* partner (which needs a face_bc code); must be symmetric */
  const int32_t* vmapP;      /* host [K][4 Nfp]: flat node index k2 Np + n2 of the      */
                             /* partner of each face node, -code at boundary faces;     */
                             /* checked for range, symmetry and coincident positions    */
                             /* (modulo the period), and against EToE / EToF if given   */
  const double* Dr;          /* host [Np][Np] row-major, with Ds, Dt, LIFT and Fmask:    */
  const double* Ds;          /* all five or none; D must annihilate constants and the   */
  const double* Dt;          /* Fmask nodes must lie on their faces of the reference    */
  const double* LIFT;        /* tetrahedron (ref_nodes); LIFT [Np][4 Nfp]                */
  const int32_t* Fmask;      /* [4][Nfp]                                                  */
  const double* geo;         /* host [K][DG_GEO_STRIDE]: geometric factors (finite,       */
                             /* J > 0, unit normals, Fscale > 0)                          */
} dg_mesh_desc;

/* Boundary conditions of faces without a partner (Sec. 5.3-5.4 run wall-bounded and inflow /
 * outflow cases; the paper does not write out their treatment).  Ghost-state reading: at a
 * boundary face node the exterior trace q+ is built from the interior trace q- and the outward
 * unit normal n and fed to the same numerical fluxes as an interior face:
 *   DG_BC_SLIP_WALL   q+ = (rho, m - 2 (m.n) n, rho E): mirror state; with viscosity the wall
 *                     is shear-free and adiabatic: traction t+ = 2 (n.t-) n - t-, energy flux
 *                     e+ = -e- (t = tau n, e = n.(u.tau + kappa grad T));
 *   DG_BC_NOSLIP_WALL q+ = (rho, -m, rho E); viscous t+ = t-, e+ = -e- (adiabatic, no work);
 *   DG_BC_INFLOW      q+ = the state set by dg_mesh_set_inflow (supersonic inflow);
 *   DG_BC_OUTFLOW     q+ = q- (supersonic outflow).
 * BR1 exterior values are w(q+); away from walls the viscous exterior flux is the interior one.
 * Meshes with boundary faces run with a perfect gas (Euler or Navier-Stokes) in the FP64, the
 * mixed-precision and the batched forms (the last two with ghost node records), and with an
 * NASA-7 mixture in the FP64 form (inviscid or viscous) and the mixed-precision form (inviscid):
 * species densities are carried like the density; a wall or outflow ghost keeps the node's
 * internal energy and so its temperature, p and c; an inflow ghost takes p and c of q_in at its
 * own temperature.
 * In the vmapP of dg_mesh_connectivity a boundary face node holds -code. */
#define DG_BC_SLIP_WALL 1
#define DG_BC_NOSLIP_WALL 2
#define DG_BC_INFLOW 3
#define DG_BC_OUTFLOW 4

/* Build the host-side tables only (no device memory, no CUDA call).  Such a
 * mesh answers dg_mesh_info / dg_mesh_operators / dg_mesh_connectivity and is
 * rejected by the compute calls.  Lets the host logic be checked without a GPU. */
#define DG_MESH_HOST_ONLY 1

/* Uploads the mesh: the element-local arrays and connectivity data of the paper's problem
 * statement (Sec. 1 Fig. 1; Sec. 4.1.2 / Sec. 4.3 connectivity and indirect gather).  Tables the
 * caller does not give are built: the reference operators (Dr, Ds, Dt, LIFT = M^-1 E, Fmask) from
 * the reference nodes, the affine geometric factors (inverse Jacobian, unit outward normals,
 * Fscale = face area / (2 J)) from the vertices, and vmapP from the caller's EToE / EToF (face
 * nodes matched by coordinates under each pair's periodic shift) or, without them, with the faces
 * paired by centroid modulo the period.  The quadrature weights, the modal matrix of the shock
 * sensor and the tensor-core operator tables always come from the reference nodes and the
 * (given or built) operators.  Then copies them to the current device together with
 * per-node scratch: the viscous flux (9 doubles per node), the FP64 form's primitives
 * (1/rho, p, c: 3 doubles per node) and the partials of the global reductions.  Sec. 1
 * Fig. 1 (element-local arrays), Sec. 4.1.2 / Sec. 4.3 (connectivity, indirect gather).
 * Every face must find exactly one partner, or carry a DG_BC_* code in face_bc;
 * a paired face must carry 0; otherwise DG_ERR_INVALID_ARG.  Allocates device
 * memory (cudaMalloc); *out owns it.  The scratch is the mesh's: calls on one mesh from
 * several streams or host threads at once race on it and must be serialised (a state
 * per stream needs a mesh per stream). */
int dg_mesh_upload(const dg_mesh_desc* desc, dg_mesh* out);
int dg_mesh_free(dg_mesh mesh);

/* Sets the conserved state q_in[nvar] (host; nvar = 5 for a perfect gas, 5 + species for a
 * NASA-7 mixture) that DG_BC_INFLOW faces impose.  Required before a right-hand side on a mesh
 * with inflow faces (DG_ERR_INVALID_ARG otherwise, or when nvar differs from the gas's).  With a
 * mixture, each right-hand side first solves the state's temperature on the host (Newton on
 * e(T) = E/rho - |u|^2/2 from 1000 K to the gas's tolerance); a solve that does not reach a
 * positive T with a positive cv makes that call fail with DG_ERR_INVALID_ARG before any launch.
 * Errors: DG_ERR_INVALID_ARG (NULL, nvar outside 5..5+DG_MAX_SPECIES, rho <= 0 or non-finite). */
int dg_mesh_set_inflow(dg_mesh mesh, const double* q_in, int32_t nvar);

/* ---- shock capturing: artificial viscosity ------------------------------------------------
 * Sec. 5.3 stabilises its shock cases with artificial viscosity (among others) without writing
 * it out; the method here is the sub-cell shock capturing of Persson and Peraire (2006).  Per
 * element, the smoothness indicator of the density, S = (energy of its orthonormal modes of total
 * degree N) / (its total energy), s = log10 S, sets the viscosity eps = 0 (s < s0 - kappa),
 * eps0 (s > s0 + kappa), eps0/2 (1 + sin(pi (s - s0) / (2 kappa))) in between; the right-hand
 * side gains div(eps grad q) on every conserved variable with BR1 central fluxes in both passes
 * (at boundary faces the gradient pass takes the ghost state and the exterior flux is the
 * interior one).  A perfect gas (Euler or Navier-Stokes) in the FP64 form, and in the
 * mixed-precision form: there the indicator and the flux sigma are formed in FP64 as above and the
 * tensor-core right-hand side subtracts sigma (in FP32, only in elements with eps > 0) and adds its
 * central face flux.  The batched form and the mixture reject a mesh with it on
 * (DG_ERR_UNSUPPORTED). */
typedef struct {
  double eps0;   /* maximum viscosity, >= 0; 0 turns the term off                            */
  double s0;     /* indicator threshold, log10 scale (e.g. -4 log10 N)                       */
  double kappa;  /* half width of the ramp, > 0                                              */
} dg_av_params;
/* Turns artificial viscosity on (params->eps0 > 0) or off (NULL or eps0 = 0) for later dg_rhs /
 * dg_rk_stage calls on the mesh; the first call that turns it on allocates 15 doubles per node
 * and one per element of device scratch (cudaMalloc; the mesh owns it).  Errors:
 * DG_ERR_INVALID_ARG (host-only mesh, eps0 < 0, kappa <= 0, non-finite), DG_ERR_CUDA, DG_ERR_OOM. */
int dg_mesh_set_av(dg_mesh mesh, const dg_av_params* params);
/* eps_dev [K] (device, caller-owned) <- the element viscosities of the state q_dev (device
 * [V][K][Np]; its density is read) under the mesh's parameters.  Asynchronous on stream. */
int dg_av_viscosity(dg_mesh mesh, const double* q_dev, double* eps_dev, void* stream);

/* ---- shock capturing: over-integration ------------------------------------------------------
 * Sec. 5.3 also names over-integration among the stabilisations of its shock cases, without
 * writing it out.  Reading: the Euler right-hand side in weak form, with the volume integral of
 * each test function's gradient against the flux taken by a quadrature rule finer than the
 * nodes, so that the flux of the interpolated state is integrated, not its nodal interpolant:
 *   rhs = sum_a M^-1 (I D_a)^T W F_a(I q) - LIFT(Fscale f*),  F_a = sum_d (dr_a/dx_d) F_d,
 * I the nodal basis at the rule's points, W its weights, f* the pointwise Lax-Friedrichs flux of
 * the face-node traces (the ghost states at boundary faces).  The rule is the Stroud conical
 * product on the collapsed cube: q Gauss-Jacobi points per direction for the weights 1, (1 - b),
 * (1 - c)^2, so q^3 points with positive weights, exact for total degree 2q - 1; ceil(3N/2)
 * points integrate degree 3N - 1, a degree-N field's quadratic fluxes against the test
 * functions' gradients.  Navier-Stokes: the whole flux G = F - Fv is integrated on the rule, with
 * the nodal BR1 viscous flux Fv of the first pass interpolated to the points.  Fv is a degree-N
 * field, so from q = N + 1 on the rule integrates that part exactly and it equals the collocated
 * weak-form term; the library applies it in that exact form on the nodes.  The face flux gains
 * minus the central viscous flux with the walls' exterior viscous fluxes, as in the collocated
 * form. */

/* Host only (no CUDA call): the rule with q points per direction (1..DG_MAX_OVERINT_POINTS) on the
 * reference tetrahedron, rst_host[q^3][3] and w_host[q^3] (caller-owned); point (k q + j) q + i
 * is the image of (a_i, b_j, c_k) under r = (1+a)(1-b)(1-c)/4 - 1, s = (1+b)(1-c)/2 - 1, t = c.
 * Errors: DG_ERR_INVALID_ARG (NULL, q out of range). */
int dg_tet_quadrature(int32_t q, double* rst_host, double* w_host);

/* Over-integration for later dg_rhs / dg_rk_stage calls on the mesh: q points per direction,
 * DG_OVERINT_DEFAULT for ceil(3N/2), 0 for the collocated strong form again.  Builds the
 * sum-factorised tables in long double from the mesh's reference nodes (the collapsed-coordinate
 * factors of the orthonormal modes at the rule's 1-D points, with and without the weights, V_o^-1,
 * V_o and the modal derivative matrices V_o^-1 D_a V_o by column, their structural zeros left
 * out) and copies them to the device (cudaMalloc; the mesh owns them).  Right-hand sides with it
 * on run in the FP64 form with a perfect gas (Euler or Navier-Stokes), periodic or with boundary
 * faces, over the whole mesh, with or without artificial viscosity (whose flux sigma =
 * eps grad_h q, a degree-N field, is integrated with G, and whose central face flux joins n.G*).
 * The viscous and AV fluxes, degree-N nodal fields, take their exact weak form, which the rule
 * reproduces from q = N + 1 on: below that a viscous or AV right-hand side is DG_ERR_UNSUPPORTED.
 * The mixed-precision and batched forms, a mixture, element ranges and prims_given are
 * DG_ERR_UNSUPPORTED too, and so is a viscous or AV right-hand side whose larger per-element work
 * does not fit at this point count.  Errors:
 * DG_ERR_INVALID_ARG (host-only mesh, q below -1 or above DG_MAX_OVERINT_POINTS, a table
 * construction that fails its own checks), DG_ERR_UNSUPPORTED (the tables and one element's Euler
 * work do not fit in a block's shared memory), DG_ERR_CUDA, DG_ERR_OOM. */
int dg_mesh_set_overint(dg_mesh mesh, int32_t q);

/* ---- partitioned meshes: halo exchange support -------------------------------------------
 * A partition of a mesh over several processes (the paper's multi-GPU runs exchange face data
 * between ranks, Sec. 5.4) is uploaded as its owned elements followed by copies of their face
 * neighbours owned elsewhere (halo elements, whose outer faces carry DG_BC_OUTFLOW); before each
 * right-hand side the halo copies are refreshed from their owners, and for Navier-Stokes the
 * viscous flux is computed, its halo refreshed, and then used (dg_opts.viscous_given).  These
 * entry points move the data; the transport between processes is the caller's. */
/* dst [V][n][Np] <- src [V][K][Np] at the elements elems_dev[n] (device int32, each in [0, K);
 * an entry outside that range is skipped: its slot of dst is left as it was).  Asynchronous on
 * stream; n = 0 does nothing.  Errors: DG_ERR_INVALID_ARG (NULL with n > 0, V < 1, Np < 1, K < 1). */
int dg_gather_elements(const double* src_dev, int32_t V, int64_t K, int32_t Np, const int32_t* elems_dev,
                       int32_t n, double* dst_dev, void* stream);
/* dst [V][K][Np] at the elements elems_dev[n] <- src [V][n][Np]; same rules as the gather. */
int dg_scatter_elements(const double* src_dev, int32_t V, int64_t K, int32_t Np, const int32_t* elems_dev,
                        int32_t n, double* dst_dev, void* stream);
/* The BR1 viscous flux of q (perfect gas, FP64 form) into the mesh's buffer (after the per-node
 * primitives 1/rho, p, c of q into the mesh's own primitives buffer), and that buffer's device
 * address and layout ([9][K][Np]: tau_xx, tau_yy, tau_zz, tau_xy, tau_xz, tau_yz, E_x, E_y, E_z),
 * valid while the mesh lives. */
int dg_viscous_flux(dg_mesh mesh, dg_gas gas, const double* q_dev, void* stream);
/* The pieces of a stage that a partition schedules around its halo exchanges (its interior
 * elements first, while the exchange is in flight; the rest after it; Sec. 4.6.1), FP64 form,
 * perfect gas, asynchronous on stream:
 * dg_primitives: (1/rho, p, c) of q at the nodes of elements [elem_begin, elem_end) into the
 * mesh's primitives buffer (DG_STATUS_NONPHYSICAL where rho <= 0 or p <= 0 there);
 * dg_viscous_flux_range: the BR1 viscous flux of the elements [elem_begin, elem_end) into the
 * mesh's buffer (the other elements' entries are left as they were), from the primitives already
 * in the primitives buffer, which must hold those of q at these elements' nodes and at their face
 * neighbours' nodes.  A stage then follows with dg_opts.viscous_given, prims_given and the element
 * range.  Errors: as dg_viscous_flux (dg_primitives: a perfect gas), and DG_ERR_INVALID_ARG
 * unless 0 <= elem_begin <= elem_end <= K. */
int dg_primitives(dg_mesh mesh, dg_gas gas, const double* q_dev, int32_t elem_begin, int32_t elem_end,
                  void* stream);
int dg_viscous_flux_range(dg_mesh mesh, dg_gas gas, const double* q_dev, int32_t elem_begin, int32_t elem_end,
                          void* stream);
int dg_mesh_viscous_buffer(dg_mesh mesh, double** fv_dev);

/* ---- global reductions: conservation integrals and the stability rate -------------------------
 * The two reductions a distributed run needs beside the halo exchange: the integrals of the
 * conserved variables (conservation diagnostics) and the largest stability rate, from which the
 * caller takes the time step dt = CFL / rate.  Both reduce over the first K_count elements of the
 * mesh (a partition's owned elements come first), run a fixed grid whose partials are combined in
 * a fixed order (bitwise reproducible), write device memory and are asynchronous on stream; the
 * caller combines the values of several ranks (sum, max).  The paper fixes neither: the
 * definitions are stated with each call.  Errors: DG_ERR_INVALID_ARG (NULL pointers, a host-only
 * mesh, K_count outside [0, K], nvar outside 1..5+DG_MAX_SPECIES). */
/* out_dev[v] <- integral of q_v over the first K_count elements, v < nvar:
 * sum_e J_e sum_i w_i q[v][e][i], w_i the integral of the i-th nodal basis function over the
 * reference tetrahedron (exact for the element's polynomial).  q_dev [>= nvar][K][Np]. */
int dg_integrals(dg_mesh mesh, const double* q_dev, int32_t nvar, int64_t K_count, double* out_dev, void* stream);
/* out_dev[0] <- max over the first K_count elements and their nodes of
 *   (N+1)^2/2 F_e (|u| + c) + (N+1)^4/4 F_e^2 nu,   F_e = max over the element's faces of Fscale,
 *   nu = (mu / rho) max(4/3, gamma / Pr) (0 for an inviscid gas),
 * the nodal-DG step estimate (advective (N+1)^2/h, diffusive (N+1)^4/h^2, 1/h read as F_e/2);
 * 0 for K_count = 0.  A node with rho <= 0 or p <= 0 gives +infinity and sets
 * DG_STATUS_NONPHYSICAL in the mesh status.  q_dev [5][K][Np]; perfect gas only
 * (DG_ERR_UNSUPPORTED otherwise). */
int dg_max_rate(dg_mesh mesh, dg_gas gas, const double* q_dev, int64_t K_count, double* out_dev, void* stream);

/* Sizes of an uploaded mesh. Any pointer may be NULL. */
int dg_mesh_info(dg_mesh mesh, int32_t* K, int32_t* N, int32_t* Np, int32_t* Nfp);

/* Copies the library's reference operators to host buffers (any may be NULL):
 * Dr/Ds/Dt [Np][Np] row-major, LIFT [Np][4 Nfp], Fmask [4][Nfp]. Test aid. */
int dg_mesh_operators(dg_mesh mesh, double* Dr_host, double* Ds_host, double* Dt_host,
                      double* LIFT_host, int32_t* Fmask_host);

/* Copies the neighbour map vmapP [K][4 Nfp] (flat node index k2 Np + n2 of the
 * partner of each face node) and per-element geometry to host buffers (any may
 * be NULL).  geo_host is [K][DG_GEO_STRIDE]. Test aid. */
#define DG_GEO_STRIDE 26 /* rx ry rz sx sy sz tx ty tz | (nx ny nz Fscale) x 4 faces | J */
int dg_mesh_connectivity(dg_mesh mesh, int32_t* vmapP_host, double* geo_host);

/* Copies the face pairing EToE, EToF [K][4] (element and face of each face's partner, -1 in both
 * for a face without one) to host buffers (either may be NULL). */
int dg_mesh_face_pairs(dg_mesh mesh, int32_t* EToE_host, int32_t* EToF_host);

/* Reads (and with reset != 0 clears) the device status word of the mesh, after
 * synchronising the device.  *bits receives DG_STATUS_* bits. */
int dg_mesh_status(dg_mesh mesh, uint32_t* bits, int reset);

/* ---- per-kernel timing (CUDA events on the launch stream) ------------------ */
#define DG_KERNEL_VISCOUS 0     /* BR1 gradient + viscous flux pass            */
#define DG_KERNEL_RHS 1         /* fused right-hand side (+ RK stage)          */
#define DG_KERNEL_TEMPERATURE 2 /* Newton temperature solve inside dg_rhs/stage */
#define DG_KERNEL_PRIMS 3       /* per-node primitives pass (1/rho, p, c; mixed form: + T, records) */
#define DG_KERNEL_AV 4          /* artificial viscosity: indicator + flux passes  */
#define DG_NUM_KERNELS 5

/* With enable != 0, every later dg_rhs / dg_rk_stage on this mesh brackets each
 * of its kernel launches with CUDA events recorded on the launch stream (the
 * events are created by the library).  Timing adds two event records per
 * launch and nothing else. */
int dg_mesh_set_timing(dg_mesh mesh, int enable);

/* Waits for the recorded events and returns, per DG_KERNEL_* id, the summed
 * device time in milliseconds (ms_host[DG_NUM_KERNELS]) and the number of
 * launches (launches_host[DG_NUM_KERNELS]) since the last reset; reset != 0
 * clears the totals. */
int dg_mesh_kernel_times(dg_mesh mesh, double* ms_host, int64_t* launches_host, int reset);

/* ---- gas ----------------------------------------------------------------- */
/* A NASA-7 mixture with mu > 0 (FP64 form) carries viscosity, heat conduction
 * and species diffusion (the paper's viscous multi-species flows, Sec. 4-5, name no transport
 * model; reading): constant mu, Stokes hypothesis; kappa = mu cp_mix(T, Y) / Pr; Fickian
 * diffusion at the Schmidt number Sc with the zero-sum correction,
 * J_k = -(mu / Sc) (grad Y_k - Y_k sum_j grad Y_j); heat flux q = -kappa grad T + sum_k h_k J_k;
 * BR1 central fluxes on (rho, rho u, T, Y_k).  At boundary faces the gradient pass takes the
 * ghost state's values (the node's own T and Y at walls and outflow, the inflow state's at
 * inflow); walls are adiabatic (the energy flux holds the enthalpy diffusion too) and impermeable
 * (the species rows' exterior normal flux is minus the interior one), a slip wall shear-free.  The
 * mesh allocates 33 doubles per node for its viscous flux on the first such call. */
#define DG_GAS_PERFECT 0
#define DG_GAS_NASA7 1

typedef struct {
  int32_t model;             /* DG_GAS_PERFECT or DG_GAS_NASA7                     */
  double gamma;              /* perfect gas: ratio of specific heats               */
  double R;                  /* perfect gas: gas constant (T = p / (rho R))       */
  double mu;                 /* dynamic viscosity; 0 = inviscid (Euler)            */
  double Pr;                 /* Prandtl number: kappa = mu cp / Pr                 */
  int32_t nspecies;          /* NASA-7: 1..DG_MAX_SPECIES (state V = 5 + nspecies) */
  const double* W;           /* NASA-7: host [nspecies] molar masses               */
  const double* nasa7;       /* NASA-7: host [nspecies][7] coefficients a1..a7     */
  double R_universal;        /* NASA-7: R_k = R_universal / W_k                    */
  double newton_tol;         /* NASA-7: stop at |dT| < tol (K), e.g. 1e-10         */
  int32_t newton_max_it;     /* NASA-7: iteration cap, e.g. 50                     */
  double Sc;                 /* NASA-7 with mu > 0: Schmidt number of the species  */
                             /* diffusion, rho D = mu / Sc (> 0)                   */
} dg_gas_desc;

/* Perfect gas (Sec. 5.3): p = (gamma-1)(rho E - rho |u|^2 / 2).
 * NASA-7 mixture (Sec. 4, Sec. 5 multi-species): cp_k/R_k = a1 + a2 T + ... + a5 T^4,
 * h_k/R_k = a1 T + a2 T^2/2 + ... + a5 T^5/5 + a6, e = sum_k Y_k (h_k - R_k T),
 * p = rho R_mix T, c^2 = (cp/cv) p / rho.  Viscous mixtures are unsupported. */
int dg_gas_create(const dg_gas_desc* desc, dg_gas* out);
int dg_gas_free(dg_gas gas);
int dg_gas_status(dg_gas gas, uint32_t* bits, int reset);

/* ---- options --------------------------------------------------------------- */
#define DG_PREC_FP64 0   /* every step in float64                                   */
/* D and LIFT contractions on tensor cores as split-fp16 products (x = hi + lo,
 * three products, fp32 accumulation), pointwise fluxes in fp32; pressure,
 * pressure/state differences that would cancel, and the RK update in fp64.
 * Perfect gas only; error vs the fp64 form is reported by the tests. */
#define DG_PREC_MIXED 1
#define DG_TSEED_INPUT 0 /* Newton starts from T_io                                  */
#define DG_TSEED_CONST 1 /* Newton starts from opts.t_const                           */
#define DG_TSEED_MLP 2   /* Newton starts from the gas's trained MLP guess            */

typedef struct {
  int32_t precision;      /* DG_PREC_*                                               */
  int32_t t_seed;         /* DG_TSEED_*                                              */
  double t_const;         /* constant Newton seed for DG_TSEED_CONST                 */
  int32_t viscous_given;  /* FP64 Navier-Stokes: != 0 uses the viscous flux already   */
                          /* in the mesh's buffer (dg_viscous_flux, then a halo       */
                          /* exchange) instead of computing it                        */
  int32_t wait_polls;     /* tensor-core kernels (mixed form, MLP guess): polls of    */
                          /* each bounded wait for an MMA completion; 0 = the default  */
                          /* bound.  A test aid: a small value makes the waits run    */
                          /* out, which the kernels report as DG_STATUS_TIMEOUT (the  */
                          /* output is then incomplete) and return without hanging    */
  int32_t elem_range;     /* FP64 form, perfect gas, no artificial viscosity: != 0    */
  int32_t elem_begin;     /* evaluates the right-hand side / stage of the elements    */
  int32_t elem_end;       /* [elem_begin, elem_end) only (0 <= elem_begin <= elem_end */
                          /* <= K; an empty range does nothing); the other elements'  */
                          /* outputs (and RK register) are left as they were.  The    */
                          /* primitives of every node (and,                           */
                          /* without viscous_given, the viscous flux of every         */
                          /* element) are still computed, unless prims_given.  A      */
                          /* partition evaluates its interior elements while a halo   */
                          /* exchange is in flight and the rest after it (parts run   */
                          /* as soon as their inputs are there, Sec. 4.6.1).  Other   */
                          /* forms: DG_ERR_UNSUPPORTED                                */
  int32_t prims_given;    /* FP64 form, perfect gas: != 0 skips the primitives pass:  */
                          /* the mesh's primitives buffer already holds those of q    */
                          /* at every node the call reads (dg_primitives).  Other     */
                          /* forms: DG_ERR_UNSUPPORTED                                */
  int32_t reserved[2];
} dg_opts;                /* NULL = defaults: DG_PREC_FP64, DG_TSEED_INPUT          */

/* ---- the hot path ------------------------------------------------------------ */

/* Semi-discrete right-hand side rhs = dq/dt (strong form) of the nodal DG discretisation that
 * MIRGE-Com evaluates (Sec. 1 and Fig. 1: element-local DOF arrays; Sec. 4.2.2 / Sec. 5.2: the
 * reference-operator contractions of the full assembly; Sec. 4.3: the indirect face gather;
 * Sec. 5.2 Euler, Sec. 5.3 Navier-Stokes):
 *   rhs = -sum_d dG_d/dx_d + LIFT( Fscale * (n.G(q-) - G*) ),  G = F_euler - F_viscous,
 * with the pointwise Lax-Friedrichs flux for F_euler and, when mu > 0, BR1
 * central fluxes for the gradients of (rho, rho u, T) and for F_viscous.
 * q_dev, rhs_dev: [V][K][Np]; they must not overlap.  T_io_dev: [K][Np],
 * required for a NASA-7 gas (Newton seed in, temperature out), ignored (may be
 * NULL) for a perfect gas.  The mesh's scratch buffer is used for the viscous
 * flux, so calls on one mesh must not overlap in time. */
int dg_rhs(dg_mesh mesh, dg_gas gas, const double* q_dev, double* rhs_dev, double* T_io_dev,
           const dg_opts* opts, void* stream);

/* Stage s (0..4) of the explicit fourth-order Runge-Kutta time stepping of the paper's runs
 * (Sec. 5.2, the MFEM comparison advances the DG discretisation with explicit fourth-order
 * Runge-Kutta), here the five-stage 2N-storage RK4 of Carpenter & Kennedy (1994):
 *   k <- a_s k + dt rhs(q_in),   q_out <- q_in + b_s k.
 * The right-hand side and the update are fused; k_dev is updated in place
 * (a_0 = 0, so its content is ignored at s = 0).  q_out_dev must not overlap
 * q_in_dev (neighbour traces of q_in are read while q_out is written). */
int dg_rk_stage(dg_mesh mesh, dg_gas gas, int32_t stage, double dt, const double* q_in_dev,
                double* q_out_dev, double* k_dev, double* T_io_dev, const dg_opts* opts, void* stream);

/* The coefficients a_s, b_s (s = 0..4) used by dg_rk_stage (host arrays of 5). */
int dg_lsrk4_coefficients(double* a_host, double* b_host);

/* Per-node temperature of a NASA-7 mixture from the conserved state, the pointwise solve of the
 * paper's multi-species model (Sec. 4: the compressible multispecies flow example; Sec. 5:
 * MIRGE-Com's reactive mixture viscous flows):
 * e = rho E / rho - |u|^2/2, Y_k = rho Y_k / rho, Newton T <- T - (e(T) - e)/cv(T)
 * from the seed (T_io or opts.t_const) until |dT| < newton_tol.  n nodes;
 * q_dev: [V][n] (V = 5 + nspecies); T_io_dev: [n]; iters_dev (nullable):
 * int32 [n] Newton updates taken.  Nodes that reach newton_max_it set
 * DG_STATUS_NO_CONVERGENCE in the gas status. */
int dg_temperature(dg_gas gas, int64_t n, const double* q_dev, double* T_io_dev, int32_t* iters_dev,
                   const dg_opts* opts, void* stream);

/* Mixture internal energy e(T, Y) per node (the inverse of dg_temperature's
 * solve): n nodes, T_dev [n], Y_dev [nspecies][n], e_dev [n]. */
int dg_mixture_energy(dg_gas gas, int64_t n, const double* T_dev, const double* Y_dev, double* e_dev,
                      void* stream);

/* ---- learned temperature guess (no counterpart in the paper) ------------------------
 * An 8 -> 64 -> 64 -> 1 tanh MLP maps x = ((e - e_mean)/e_scale, Y_1..Y_7) to
 * (T - T_mean)/T_scale; its guess (clamped to [T_min, T_max]) seeds the FP64
 * Newton solve, which still decides the result (same |dT| < tol) and its
 * fallback.  Inference uses FP16 operands with FP32 accumulation on the tensor
 * cores; training runs the library's own FP32 forward/backward and Adam kernels.
 * Parameters, float, flat: W1 [64][8] | b1 [64] | W2 [64][64] | b2 [64] | W3 [64] | b3. */
#define DG_MLP_PARAMS 4801

typedef struct {
  double e_mean, e_scale;    /* input 0 = (e - e_mean) / e_scale                    */
  double T_mean, T_scale;    /* T = T_mean + T_scale * output                        */
  double T_min, T_max;       /* clamp of the guess                                   */
} dg_mlp_norm;

typedef struct {
  int32_t epochs;            /* passes over the samples                              */
  int32_t batch;             /* samples per Adam step (full batches are used)        */
  float lr;                  /* Adam step size (beta1 0.9, beta2 0.999, eps 1e-8)    */
  float lr_decay;            /* step size multiplier per epoch                        */
} dg_mlp_train_opts;

/* Attach (or replace) the gas's MLP: params_host [DG_MLP_PARAMS] and its normalisation. */
int dg_mlp_set(dg_gas gas, const float* params_host, const dg_mlp_norm* norm);
/* Copy the gas's MLP parameters and normalisation to the host (either may be NULL). */
int dg_mlp_get(dg_gas gas, float* params_host, dg_mlp_norm* norm);

/* Batch loss and gradient: loss += mean_i (y_i - t_i)^2 and grad += its gradient
 * with respect to params_dev, for x_dev [n][8], t_dev [n] (normalised), all float
 * device arrays; grad_dev [DG_MLP_PARAMS] and loss_dev [1] accumulate (the caller
 * zeroes them).  The training step's kernel, exposed for gradient checks. */
int dg_mlp_loss_grad(int64_t n, const float* params_dev, const float* x_dev, const float* t_dev, float* grad_dev,
                     float* loss_dev, void* stream);

/* One Adam update of the training loop (Kingma & Ba 2015, Algorithm 1, with beta1 = 0.9,
 * beta2 = 0.999, eps = 1e-8), exposed for checks: elementwise over the DG_MLP_PARAMS float device
 * arrays, with g = grad,
 *   m <- beta1 m + (1 - beta1) g,   v <- beta2 v + (1 - beta2) g^2,
 *   params <- params - lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps),
 * then grad <- 0 (the next batch accumulates into it).  t >= 1 is the step number (the bias
 * corrections are formed in FP64, the update in FP32).  Asynchronous on stream.  Errors:
 * DG_ERR_INVALID_ARG (NULL, t < 1, non-finite lr). */
int dg_mlp_adam_step(int32_t t, float lr, float* params_dev, float* grad_dev, float* m_dev, float* v_dev,
                     void* stream);

/* Train the gas's MLP on n samples (e_dev [n], Y_dev [nspecies][n], T_dev [n],
 * float64 device arrays; T typically from dg_temperature), starting from
 * init_params_host, with the normalisation taken from the samples' means and
 * standard deviations.  Synchronous; allocates its work buffers.  The mean loss
 * of each epoch goes to loss_history_host [epochs] (nullable). */
int dg_mlp_train(dg_gas gas, int64_t n, const double* e_dev, const double* Y_dev, const double* T_dev,
                 const float* init_params_host, const dg_mlp_train_opts* opts, float* loss_history_host);

/* The MLP's temperature guess alone (no Newton) for the state q_dev [V][n]. */
int dg_mlp_guess(dg_gas gas, int64_t n, const double* q_dev, double* T_dev, void* stream);

/* ---- allocation-free stage (no counterpart in the paper) --------------------------
 * For callers that cannot call cudaMalloc: code whose device memory is owned by
 * another allocator (a host framework's memory pool that has reserved the
 * device, an arena with a fixed budget), or loops where an allocation's implicit
 * device synchronisation is not acceptable.  Such a caller allocates the tables
 * and buffers itself, fills the tables from a DG_MESH_HOST_ONLY mesh
 * (dg_mesh_operators, dg_mesh_connectivity; no CUDA call is made to build it),
 * and calls dg_rk_stage_noalloc, which allocates nothing: the viscous-flux
 * scratch of the BR1 pass lives in a static device array of
 * DG_STATIC_SCRATCH_NODES * 9 doubles (36 MiB).  With CUDA's default lazy module
 * loading that array is committed on a device when the first call there loads
 * the code module that holds it, and it stays until the process exits (or the
 * context is reset); make that first call before the caller's allocator reserves
 * the device's memory, or it can fail with DG_ERR_CUDA (out of memory). */
#define DG_STATIC_SCRATCH_NODES (1 << 19) /* largest K * Np accepted */

typedef struct {
  int32_t K;                 /* tetrahedra                                            */
  int32_t N;                 /* order, 1..DG_MAX_ORDER                                 */
  const double* ops_dev;     /* [3 Np Np + Np 4 Nfp]: Dr | Ds | Dt | LIFT, row-major  */
  const int32_t* fmask_dev;  /* [4][Nfp]                                               */
  const double* geo_dev;     /* [K][DG_GEO_STRIDE]                                     */
  const int32_t* vmapP_dev;  /* [K][4 Nfp]; boundary face nodes hold -code for          */
                             /* DG_BC_SLIP_WALL, DG_BC_NOSLIP_WALL or DG_BC_OUTFLOW     */
} dg_mesh_tables;

/* Same stage as dg_rk_stage for a viscous perfect gas (gas->model ==
 * DG_GAS_PERFECT, gas->mu > 0): k <- a_s k + dt rhs(q_in), q_out <- q_in + b_s k,
 * with the same kernels, on caller-owned tables and buffers.  status_dev: one
 * uint32 in device memory that receives DG_STATUS_* bits (atomic OR; the
 * caller clears it).  Periodic faces and wall and outflow boundary faces are
 * supported; there is no inflow state here, so a face coded DG_BC_INFLOW gets a
 * zero ghost density, which sets DG_STATUS_NONPHYSICAL (the tables are device
 * memory and are not read on the host).  Rejects K * Np > DG_STATIC_SCRATCH_NODES
 * with DG_ERR_INVALID_ARG.  Each call looks up the static array's device address
 * in the current context (cudaGetSymbolAddress); the first call on a device
 * loads the code module (see above) and must come before any stream capture.  Every
 * call shares the one array and leaves its content behind; the stage writes all
 * of it that it reads, so nothing needs clearing, but calls that overlap in time
 * on the GPU (other streams, other host threads) race on it and must be
 * serialised. */
int dg_rk_stage_noalloc(const dg_mesh_tables* tables, const dg_gas_desc* gas, int32_t stage, double dt,
                        const double* q_in_dev, double* q_out_dev, double* k_dev, uint32_t* status_dev,
                        void* stream);

/* ---- batched form: many uneven cases, one graph launch per RK4 step --------------------
 * Cases of orders 1..4, Euler or Navier-Stokes (perfect gas), any sizes, periodic or with
 * boundary faces (the inflow state set where a mesh has inflow faces), advanced together in the
 * mixed-precision form (DG_PREC_MIXED).  Cases are grouped by
 * (order, physics); each group's kernels are persistent over a device work list of
 * (case, element tile) items, so a stage costs one launch per group and pass, and
 * a whole RK4 step (5 stages, then each case's result copied back into its state)
 * is captured once into a CUDA graph.  With DG_BATCH_AUTOTUNE the tile size of
 * each group (elements per block) is chosen at creation by timing the compiled
 * candidates on the batch's own cases.  The paper's nearest counterpart is its
 * concatenation of outlined calls into fewer kernels (Sec. 4.2.4) and the
 * launch-overhead floor of small cases (Sec. 5.2). */
typedef struct dg_batch_s* dg_batch;

typedef struct {
  dg_mesh mesh;    /* uploaded mesh (its tables and scratch are used by the batch)     */
  dg_gas gas;      /* perfect gas, inviscid or viscous                                  */
  double dt;       /* the case's time step                                              */
  double* q_dev;   /* [5][K][Np] state, advanced in place by dg_batch_step               */
} dg_batch_case;

#define DG_BATCH_AUTOTUNE 1

/* Creates the batch: allocates a work state and an RK register per case, builds the
 * work lists, tunes the tiles (flag), and captures the step graph.  Meshes of one
 * order must share their reference operators; each mesh belongs to one case, and
 * the meshes, gases and states must outlive the batch.  Synchronous. */
int dg_batch_create(const dg_batch_case* cases, int32_t ncases, int32_t flags, dg_batch* out);

/* Advances every case by `steps` RK4 steps: `steps` graph launches on `stream`. */
int dg_batch_step(dg_batch batch, int32_t steps, void* stream);

/* Chosen block sizes (threads per 25-element tensor-core tile): rhs_tiles_host [4][2]
 * (order, physics 0 = Euler / 1 = NS; 0 where the batch has no such group),
 * viscous_tiles_host [4]; rhs_tune_ms_host [4][2][4] the timings of the candidates (any
 * pointer may be NULL). */
int dg_batch_tiles(dg_batch batch, int32_t* rhs_tiles_host, int32_t* viscous_tiles_host, double* rhs_tune_ms_host);

/* DG_STATUS_* bits of the batch's cases (non-physical states, a tensor-core wait that timed out),
 * after synchronising the device; reset != 0 clears them. */
int dg_batch_status(dg_batch batch, uint32_t* bits, int reset);
/* Frees the batch's device memory and CUDA graph (the cases' meshes, gases and states stay the
 * caller's). NULL is a no-op. */
int dg_batch_free(dg_batch batch);

/* ---- tensor-product hexahedra ---------------------------------------------------------------
 * Nodal DG on a periodic box of axis-aligned hexahedra with tensor-product nodes, the element
 * type of the paper's timed runs (Sec. 5.2-5.4, "tensor product elements"); Euler and
 * Navier-Stokes equations of a perfect gas in FP64, the same local Lax-Friedrichs flux,
 * BR1 central fluxes and fused LSRK4 stage as the tetrahedral path.  Collocated nodal spectral-element DG: quadrature weights w_i = integral of the
 * 1-D Lagrange basis through the node set, D[i][j] = l_j'(x_i), diagonal mass,
 *   rhs = - sum_d (2/h_d) D_d F_d + sum over the faces of a node (2/h_d) / w_end (n.F- - n.F*),
 * applied by sum factorisation.  State layout [5][K][(N+1)^3], node index i + (N+1)(j + (N+1)k)
 * (i along x fastest), element index ex + nx (ey + ny ez); element (ex, ey, ez) spans
 * [ex h_x, (ex+1) h_x] x ... with h = L / n. */
typedef struct dg_hex_mesh_s* dg_hex_mesh;
typedef struct {
  int32_t n[3];            /* hexahedra per direction, >= 1                                   */
  double L[3];             /* box lengths, > 0                                                */
  int32_t N;               /* order, 1..DG_MAX_ORDER                                          */
  const double* nodes1d;   /* host [N+1]: the 1-D node set, ascending, first -1 and last 1
                              (copied; Gauss-Lobatto-Legendre points in the workloads)        */
  int32_t bc[6];           /* DG_BC_* code of the box faces x-, x+, y-, y+, z-, z+; 0 on both
                              faces of an axis: periodic along it (ghost states as for the
                              tetrahedral path, with n = -e_axis or +e_axis)                  */
} dg_hex_desc;
/* Builds the 1-D operators on the host and uploads them.  Errors: DG_ERR_INVALID_ARG (sizes,
 * node set), DG_ERR_CUDA. */
int dg_hex_mesh_create(const dg_hex_desc* desc, dg_hex_mesh* out);
int dg_hex_mesh_free(dg_hex_mesh mesh);
/* Host copies of the library's 1-D operators: D_host [N+1][N+1] row-major, w_host [N+1]
 * (either may be NULL). */
int dg_hex_operators(dg_hex_mesh mesh, double* D_host, double* w_host);
/* rhs = right-hand side of q (device arrays [5][K][Np], caller-owned, not overlapping); the gas
 * must be a perfect gas (else DG_ERR_UNSUPPORTED); with mu > 0 (Navier-Stokes) the first such
 * call allocates 9 doubles per node for the viscous flux; walls are adiabatic and a slip wall
 * shear-free, as on tetrahedra.  Asynchronous on stream. */
int dg_hex_rhs(dg_hex_mesh mesh, dg_gas gas, const double* q_dev, double* rhs_dev, void* stream);
/* LSRK4 stage (as dg_rk_stage): k <- a_s k + dt rhs(q_in); q_out <- q_in + b_s k. */
int dg_hex_rk_stage(dg_hex_mesh mesh, dg_gas gas, int32_t stage, double dt, const double* q_in_dev,
                    double* q_out_dev, double* k_dev, void* stream);
/* Scalar advection du/dt + a . grad u = 0 with a constant velocity (the paper's GPU comparison
 * workload, Sec. 5.2, run there on p = 1 tensor-product elements): flux F_d = a_d u, local
 * Lax-Friedrichs flux with lambda = |a . n| (the upwind flux), the same strong form and lifting.
 * velocity: host [3]; u, rhs: device [K][Np], caller-owned, not overlapping.  Errors:
 * DG_ERR_INVALID_ARG (NULL, overlap, non-finite velocity or dt, stage outside 0..4), DG_ERR_CUDA.
 * Asynchronous on stream. */
int dg_hex_advection_rhs(dg_hex_mesh mesh, const double* velocity, const double* u_dev, double* rhs_dev,
                         void* stream);
/* LSRK4 stage of the advection: k <- a_s k + dt rhs(u_in); u_out <- u_in + b_s k. */
int dg_hex_advection_rk_stage(dg_hex_mesh mesh, const double* velocity, int32_t stage, double dt,
                              const double* u_in_dev, double* u_out_dev, double* k_dev, void* stream);
/* Conserved state q_in[5] (host) imposed on DG_BC_INFLOW box faces; required before a
 * right-hand side on a box with such faces.  Errors: DG_ERR_INVALID_ARG (NULL, nvar != 5,
 * non-finite, rho <= 0).  The advection entry points take periodic boxes only
 * (DG_ERR_UNSUPPORTED otherwise). */
int dg_hex_set_inflow(dg_hex_mesh mesh, const double* q_in, int32_t nvar);
/* Artificial viscosity on hexahedra (the reading of dg_mesh_set_av on tensor-product elements):
 * the indicator is the GLL-weighted energy of the density's Legendre modes with an index equal to
 * N over its total energy; the term div(eps grad q) is added with BR1 central fluxes.  params NULL
 * or eps0 = 0 turns it off; the first call that turns it on allocates 15 doubles per node and one
 * per element.  Errors as dg_mesh_set_av. */
int dg_hex_set_av(dg_hex_mesh mesh, const dg_av_params* params);
/* eps_dev [K] <- the element viscosities of q_dev [5][K][Np] under the mesh's parameters. */
int dg_hex_av_viscosity(dg_hex_mesh mesh, const double* q_dev, double* eps_dev, void* stream);
/* Over-integration (Sec. 5.3 names it among the stabilisations of its shock cases; reading): with
 * enable != 0 the Euler right-hand side uses the weak form with its volume integral evaluated on
 * Q = ceil(3 (N+1) / 2) Gauss-Legendre points per axis (the state interpolated there, the fluxes
 * evaluated there, contracted back with W^-1 (I D)^T W_Q and W^-1 I^T W_Q); the face terms are
 * the collocated weak-form ones.  Navier-Stokes: the whole flux G = F - Fv is integrated on the
 * points, the nodal BR1 viscous flux interpolated to them, and the face terms take the central
 * viscous flux with the walls' exterior viscous fluxes of the collocated form.  Artificial
 * viscosity: its flux sigma = eps grad_h q joins the fluxes on the points and its central flux the
 * face terms. */
int dg_hex_set_overintegration(dg_hex_mesh mesh, int32_t enable);
/* DG_STATUS_* bits of the mesh (rho <= 0 or p <= 0 met); synchronises the device. */
int dg_hex_status(dg_hex_mesh mesh, uint32_t* bits, int reset);

/* ---- precision conversions ------------------------------------------------------------------
 * The FP64 -> FP32 and FP32 -> FP64 conversions that the mixed-precision kernels use, done with
 * integer operations on the IEEE-754 bit patterns (the FP64 pipe, which runs the hardware
 * conversions, is the scarce unit on this GPU).  The paper has no counterpart; exposed so that
 * the conversions can be checked against the hardware's.
 *   dg_round_to_float: y[i] = x[i] rounded to nearest, ties to even (as the hardware for all
 *     inputs; normal and zero results on the integer path, the rest by the hardware).
 *   dg_widen_to_double: y[i] = x[i] exactly for finite, infinite and NaN inputs; float
 *     subnormals become signed zero.
 * x, y: device arrays of n elements (n >= 0), asynchronous on stream. */
int dg_round_to_float(const double* x_dev, float* y_dev, int64_t n, void* stream);
int dg_widen_to_double(const float* x_dev, double* y_dev, int64_t n, void* stream);
/* hi[i] = x[i] rounded to FP32 as dg_round_to_float, lo[i] = (x[i] - hi[i]) rounded to FP32 (the
 * float pair, ~48 significant bits, in which the mixed form keeps density, pressure and
 * temperature); hi, lo: device arrays of n floats. */
int dg_split_to_float_pair(const double* x_dev, float* hi_dev, float* lo_dev, int64_t n, void* stream);

/* ---- device characterisation ----------------------------------------------------------------
 * *tflops_host <- the FP64 FMA throughput of the current device in TFLOP/s (an FMA counted as two
 * flops), measured with a kernel of independent FMA chains on every SM (best of three timed
 * launches after a warm-up; CUDA events).  The measured denominator beside the nominal FP64 peak
 * for kernels that the FP64 pipe bounds.  The paper has no counterpart.  Synchronous; allocates
 * 8 bytes of device memory.  Errors: DG_ERR_INVALID_ARG (NULL), DG_ERR_CUDA. */
int dg_fp64_fma_rate(double* tflops_host);

/* Message of the last failed call on this thread ("" if none). */
const char* dg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DG_H_ */
