"""Python binding of libdg: same names as the C ABI, argument marshalling only.

Device arrays are torch CUDA tensors (float64 / int32, contiguous); torch is
used for device memory and streams, every computation runs in libdg's CUDA
kernels.  Host arrays are numpy arrays.
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import capi
from .capi import check, load


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t, dtype=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _opts(precision=capi.DG_PREC_FP64, t_seed=capi.DG_TSEED_INPUT, t_const=0.0, wait_polls=0, elems=None,
          viscous_given=False, prims_given=False):
    """dg_opts; elems = (begin, end): the element range of a FP64 perfect-gas right-hand side."""
    o = capi.dg_opts()
    o.precision = precision
    o.t_seed = t_seed
    o.t_const = t_const
    o.wait_polls = wait_polls
    o.viscous_given = int(bool(viscous_given))
    o.prims_given = int(bool(prims_given))
    if elems is not None:
        o.elem_range, o.elem_begin, o.elem_end = 1, int(elems[0]), int(elems[1])
    return o


# ---- mesh -------------------------------------------------------------------------------

class Mesh:
    """An uploaded mesh (dg_mesh handle)."""

    # caller tables of dg_mesh_desc: name -> (dtype, shape as a function of K, Np, Nfp)
    _TABLES = {"EToV": (np.int32, lambda K, Np, Nfp: (K, 4)), "EToE": (np.int32, lambda K, Np, Nfp: (K, 4)),
               "EToF": (np.int32, lambda K, Np, Nfp: (K, 4)), "vmapP": (np.int32, lambda K, Np, Nfp: (K, 4 * Nfp)),
               "Dr": (np.float64, lambda K, Np, Nfp: (Np, Np)), "Ds": (np.float64, lambda K, Np, Nfp: (Np, Np)),
               "Dt": (np.float64, lambda K, Np, Nfp: (Np, Np)), "LIFT": (np.float64, lambda K, Np, Nfp: (Np, 4 * Nfp)),
               "Fmask": (np.int32, lambda K, Np, Nfp: (4, Nfp)),
               "geo": (np.float64, lambda K, Np, Nfp: (K, capi.DG_GEO_STRIDE))}

    def __init__(self, vertices, period, N, ref_nodes, host_only=False, face_bc=None, tables=None):
        """face_bc: optional [K][4] DG_BC_* codes of the faces without a partner (0 elsewhere).
        tables: optional dict of caller tables (EToV, EToE, EToF, vmapP, Dr, Ds, Dt, LIFT, Fmask, geo),
        which the library checks and uses instead of building them."""
        lib = load()
        self._v = np.ascontiguousarray(vertices, dtype=np.float64)
        self._r = np.ascontiguousarray(ref_nodes, dtype=np.float64)
        if self._v.ndim != 3 or self._v.shape[1:] != (4, 3):
            raise ValueError("vertices must be [K][4][3]")
        self._bc = None
        if face_bc is not None:
            self._bc = np.ascontiguousarray(face_bc, dtype=np.int32)
            if self._bc.shape != (self._v.shape[0], 4):
                raise ValueError("face_bc must be [K][4]")
        d = capi.dg_mesh_desc()
        d.K = self._v.shape[0]
        d.N = int(N)
        d.ref_nodes = _hptr(self._r)
        d.vertices = _hptr(self._v)
        for i in range(3):
            d.period[i] = float(period[i])
        d.flags = capi.DG_MESH_HOST_ONLY if host_only else 0
        d.face_bc = None if self._bc is None else _hptr(self._bc)
        self._tables = {}
        Np_, Nfp_ = (N + 1) * (N + 2) * (N + 3) // 6, (N + 1) * (N + 2) // 2
        for name, arr in (tables or {}).items():
            if name not in self._TABLES:
                raise ValueError(f"unknown mesh table {name!r}")
            dtype, shape = self._TABLES[name]
            a = np.ascontiguousarray(arr, dtype=dtype)
            if a.shape != shape(d.K, Np_, Nfp_):
                raise ValueError(f"{name} must have the shape {shape(d.K, Np_, Nfp_)}")
            self._tables[name] = a
            setattr(d, name, _hptr(a))
        h = ctypes.c_void_p()
        check(lib.dg_mesh_upload(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        K, N_, Np, Nfp = (ctypes.c_int32() for _ in range(4))
        check(lib.dg_mesh_info(h, ctypes.byref(K), ctypes.byref(N_), ctypes.byref(Np), ctypes.byref(Nfp)))
        self.K, self.N, self.Np, self.Nfp = K.value, N_.value, Np.value, Nfp.value

    def operators(self):
        Np, NF = self.Np, 4 * self.Nfp
        Dr, Ds, Dt = (np.zeros((Np, Np)) for _ in range(3))
        LIFT = np.zeros((Np, NF))
        Fm = np.zeros((4, self.Nfp), dtype=np.int32)
        check(load().dg_mesh_operators(self.handle, _hptr(Dr), _hptr(Ds), _hptr(Dt), _hptr(LIFT), _hptr(Fm)))
        return dict(Dr=Dr, Ds=Ds, Dt=Dt, LIFT=LIFT, Fmask=Fm)

    def connectivity(self):
        vmapP = np.zeros((self.K, 4 * self.Nfp), dtype=np.int32)
        geo = np.zeros((self.K, capi.DG_GEO_STRIDE))
        check(load().dg_mesh_connectivity(self.handle, _hptr(vmapP), _hptr(geo)))
        return vmapP, geo

    def face_pairs(self):
        """(EToE, EToF) [K][4]: the element and face paired with each face (-1 at boundary faces)."""
        EToE = np.zeros((self.K, 4), dtype=np.int32)
        EToF = np.zeros((self.K, 4), dtype=np.int32)
        check(load().dg_mesh_face_pairs(self.handle, _hptr(EToE), _hptr(EToF)))
        return EToE, EToF

    def set_inflow(self, q_in):
        """Conserved state imposed on DG_BC_INFLOW faces (5 values for a perfect gas)."""
        v = np.ascontiguousarray(q_in, dtype=np.float64).reshape(-1)
        check(load().dg_mesh_set_inflow(self.handle, _hptr(v), int(v.size)))

    def set_av(self, eps0, s0=None, kappa=0.5):
        """Artificial viscosity for later right-hand sides (eps0 = 0 turns it off); s0 defaults to
        -4 log10 N."""
        p = capi.dg_av_params()
        p.eps0 = float(eps0)
        p.s0 = float(-4.0 * np.log10(self.N) if s0 is None else s0)
        p.kappa = float(kappa)
        check(load().dg_mesh_set_av(self.handle, ctypes.byref(p)))

    def av_viscosity(self, q, eps, stream=None):
        """eps [K] (CUDA float64) <- the element viscosities of q under the mesh's parameters."""
        import torch
        if eps.numel() != self.K:
            raise ValueError(f"eps must hold {self.K} values")
        check(load().dg_av_viscosity(self.handle, _dptr(q, torch.float64, "q"), _dptr(eps, torch.float64, "eps"),
                                     _stream_ptr(stream)))

    def set_overint(self, q=capi.DG_OVERINT_DEFAULT):
        """Over-integrated volume term for later right-hand sides: q Gauss-Jacobi points per
        collapsed direction (the library's default for DG_OVERINT_DEFAULT, 0 turns it off)."""
        check(load().dg_mesh_set_overint(self.handle, int(q)))

    def set_timing(self, enable=True):
        check(load().dg_mesh_set_timing(self.handle, int(enable)))

    def kernel_times(self, reset=True):
        """{kernel name: (total ms, launches)} of the event-timed launches since the last reset."""
        ms = np.zeros(capi.DG_NUM_KERNELS)
        n = np.zeros(capi.DG_NUM_KERNELS, dtype=np.int64)
        check(load().dg_mesh_kernel_times(self.handle, _hptr(ms), _hptr(n), int(reset)))
        return {name: (float(ms[i]), int(n[i])) for i, name in enumerate(capi.KERNEL_NAMES)}

    def status(self, reset=True):
        bits = ctypes.c_uint32()
        check(load().dg_mesh_status(self.handle, ctypes.byref(bits), int(reset)))
        return bits.value

    def close(self):
        if getattr(self, "handle", None):
            load().dg_mesh_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dg_mesh_upload(vertices, period, N, ref_nodes, host_only=False) -> Mesh:
    return Mesh(vertices, period, N, ref_nodes, host_only=host_only)


def dg_mesh_free(mesh: Mesh) -> None:
    mesh.close()


# ---- gas ----------------------------------------------------------------------------------

class Gas:
    """A gas model (dg_gas handle): perfect gas or NASA-7 mixture."""

    def __init__(self, *, model="perfect", gamma=1.4, R=1.0, mu=0.0, Pr=0.71, W=None, nasa7=None,
                 R_universal=8314.462618, newton_tol=1e-10, newton_max_it=50, Sc=0.0):
        """Sc: Schmidt number of the species diffusion of a viscous NASA-7 mixture."""
        lib = load()
        self.mu = float(mu)
        d = capi.dg_gas_desc()
        d.mu = mu
        d.Pr = Pr
        d.Sc = Sc
        if model == "perfect":
            d.model = capi.DG_GAS_PERFECT
            d.gamma = gamma
            d.R = R
            self.nspecies = 0
        elif model == "nasa7":
            d.model = capi.DG_GAS_NASA7
            self._W = np.ascontiguousarray(W, dtype=np.float64)
            self._a = np.ascontiguousarray(nasa7, dtype=np.float64)
            d.nspecies = self._W.shape[0]
            d.W = _hptr(self._W)
            d.nasa7 = _hptr(self._a)
            d.R_universal = R_universal
            d.newton_tol = newton_tol
            d.newton_max_it = newton_max_it
            self.nspecies = int(self._W.shape[0])
        else:
            raise ValueError(model)
        h = ctypes.c_void_p()
        check(lib.dg_gas_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        self.nvar = 5 + self.nspecies
        self.model = model

    def status(self, reset=True):
        bits = ctypes.c_uint32()
        check(load().dg_gas_status(self.handle, ctypes.byref(bits), int(reset)))
        return bits.value

    def close(self):
        if getattr(self, "handle", None):
            load().dg_gas_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dg_gas_create(**kw) -> Gas:
    return Gas(**kw)


# ---- hot path -------------------------------------------------------------------------------

def dg_rhs(mesh: Mesh, gas: Gas, q, rhs, T_io=None, opts=None, stream=None):
    """rhs <- dq/dt for q [V][K][Np] (CUDA float64)."""
    import torch
    o = opts if opts is not None else _opts()
    check(load().dg_rhs(mesh.handle, gas.handle, _dptr(q, torch.float64, "q"), _dptr(rhs, torch.float64, "rhs"),
                        _dptr(T_io, torch.float64, "T_io"), ctypes.byref(o), _stream_ptr(stream)))


def dg_rk_stage(mesh: Mesh, gas: Gas, stage, dt, q_in, q_out, k, T_io=None, opts=None, stream=None):
    """LSRK4 stage: k <- a_s k + dt rhs(q_in); q_out <- q_in + b_s k."""
    import torch
    o = opts if opts is not None else _opts()
    check(load().dg_rk_stage(mesh.handle, gas.handle, int(stage), float(dt), _dptr(q_in, torch.float64, "q_in"),
                             _dptr(q_out, torch.float64, "q_out"), _dptr(k, torch.float64, "k"),
                             _dptr(T_io, torch.float64, "T_io"), ctypes.byref(o), _stream_ptr(stream)))


def dg_tet_quadrature(q):
    """(points [q^3][3], weights [q^3]) of the library's Stroud rule on the reference tetrahedron
    (host only, no GPU)."""
    pts = np.zeros((q ** 3, 3))
    w = np.zeros(q ** 3)
    check(load().dg_tet_quadrature(int(q), _hptr(pts), _hptr(w)))
    return pts, w


def dg_lsrk4_coefficients():
    a = np.zeros(5)
    b = np.zeros(5)
    check(load().dg_lsrk4_coefficients(_hptr(a), _hptr(b)))
    return a, b


def dg_temperature(gas: Gas, q, T_io, iters=None, opts=None, stream=None):
    """Newton temperature of a NASA-7 mixture, q [V][n] (or [V][K][Np]), T_io [n]."""
    import torch
    n = T_io.numel()
    o = opts if opts is not None else _opts()
    check(load().dg_temperature(gas.handle, n, _dptr(q, torch.float64, "q"), _dptr(T_io, torch.float64, "T_io"),
                                _dptr(iters, torch.int32, "iters"), ctypes.byref(o), _stream_ptr(stream)))


def dg_mixture_energy(gas: Gas, T, Y, e, stream=None):
    """e(T, Y) per node; T [n], Y [nspecies][n], e [n]."""
    import torch
    check(load().dg_mixture_energy(gas.handle, T.numel(), _dptr(T, torch.float64, "T"), _dptr(Y, torch.float64, "Y"),
                                   _dptr(e, torch.float64, "e"), _stream_ptr(stream)))


def lsrk4_step(mesh, gas, q, dt, steps=1, T_io=None, opts=None, stream=None, work=None):  # noqa: D401
    """Advance q in place by ``steps`` LSRK4 steps (5 stages each) with ping-pong buffers."""
    import torch
    if work is None:
        work = (torch.empty_like(q), torch.zeros_like(q))
    qb, k = work
    cur, nxt = q, qb
    for _ in range(steps):
        for s in range(5):
            dg_rk_stage(mesh, gas, s, dt, cur, nxt, k, T_io=T_io, opts=opts, stream=stream)
            cur, nxt = nxt, cur
    if cur is not q:
        q.copy_(cur)
    return q


def dg_round_to_float(x, y, stream=None):
    """y = x rounded to FP32 by the library's integer-pipe conversion (float64 -> float32 CUDA tensors)."""
    import torch
    check(load().dg_round_to_float(_dptr(x, torch.float64, "x"), _dptr(y, torch.float32, "y"), x.numel(),
                                   _stream_ptr(stream)))


def dg_widen_to_double(x, y, stream=None):
    """y = x widened to FP64 by the library's integer-pipe conversion (float32 -> float64 CUDA tensors)."""
    import torch
    check(load().dg_widen_to_double(_dptr(x, torch.float32, "x"), _dptr(y, torch.float64, "y"), x.numel(),
                                    _stream_ptr(stream)))


def dg_split_to_float_pair(x, hi, lo, stream=None):
    """hi, lo = the library's float-pair representation of x (float64 -> two float32 CUDA tensors)."""
    import torch
    check(load().dg_split_to_float_pair(_dptr(x, torch.float64, "x"), _dptr(hi, torch.float32, "hi"),
                                        _dptr(lo, torch.float32, "lo"), x.numel(), _stream_ptr(stream)))


def dg_integrals(mesh: Mesh, q, nvar=None, K_count=None, out=None, stream=None):
    """[nvar] CUDA float64: the integrals of q's variables over the first K_count elements."""
    import torch
    nvar = q.shape[0] if nvar is None else int(nvar)
    K_count = mesh.K if K_count is None else int(K_count)
    if q.dim() != 3 or tuple(q.shape[1:]) != (mesh.K, mesh.Np) or q.shape[0] < nvar:
        raise ValueError("q must be [>= nvar][K][Np]")
    if out is None:
        out = torch.empty(nvar, dtype=torch.float64, device=q.device)
    check(load().dg_integrals(mesh.handle, _dptr(q, torch.float64, "q"), nvar, K_count,
                              _dptr(out, torch.float64, "out"), _stream_ptr(stream)))
    return out


def dg_max_rate(mesh: Mesh, gas: Gas, q, K_count=None, out=None, stream=None):
    """[1] CUDA float64: the largest stability rate over the first K_count elements."""
    import torch
    K_count = mesh.K if K_count is None else int(K_count)
    if q.dim() != 3 or tuple(q.shape[1:]) != (mesh.K, mesh.Np) or q.shape[0] < 5:
        raise ValueError("q must be [5][K][Np]")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=q.device)
    check(load().dg_max_rate(mesh.handle, gas.handle, _dptr(q, torch.float64, "q"), K_count,
                             _dptr(out, torch.float64, "out"), _stream_ptr(stream)))
    return out


def stable_dt(mesh: Mesh, gas: Gas, q, cfl, stream=None) -> float:
    """CFL / (largest stability rate); reads the rate back to the host.  A node with rho <= 0 or
    p <= 0 makes the rate infinite (and sets DG_STATUS_NONPHYSICAL in the mesh status), so the
    step returned is 0."""
    return float(cfl) / float(dg_max_rate(mesh, gas, q, stream=stream).item())


def dg_rk_stage_noalloc(tables, gas_desc, stage, dt, q_in, q_out, k, status, stream=None):
    """Allocation-free viscous stage on caller-owned tables.

    tables: dict(K, N, ops, fmask, geo, vmapP) of CUDA tensors (float64 ops/geo, int32 fmask/vmapP);
    gas_desc: dict(gamma, R, mu, Pr); status: CUDA int32 tensor of one element.
    """
    import torch
    t = capi.dg_mesh_tables()
    t.K, t.N = int(tables["K"]), int(tables["N"])
    t.ops_dev = _dptr(tables["ops"], torch.float64, "ops")
    t.fmask_dev = _dptr(tables["fmask"], torch.int32, "fmask")
    t.geo_dev = _dptr(tables["geo"], torch.float64, "geo")
    t.vmapP_dev = _dptr(tables["vmapP"], torch.int32, "vmapP")
    g = capi.dg_gas_desc()
    g.model = capi.DG_GAS_PERFECT
    g.gamma, g.R, g.mu, g.Pr = (float(gas_desc[x]) for x in ("gamma", "R", "mu", "Pr"))
    check(load().dg_rk_stage_noalloc(ctypes.byref(t), ctypes.byref(g), int(stage), float(dt),
                                     _dptr(q_in, torch.float64, "q_in"), _dptr(q_out, torch.float64, "q_out"),
                                     _dptr(k, torch.float64, "k"), _dptr(status, torch.int32, "status"),
                                     _stream_ptr(stream)))


# ---- tensor-product hexahedra -------------------------------------------------------------------

class HexMesh:
    """A periodic box of axis-aligned hexahedra with tensor-product nodes (dg_hex_mesh handle)."""

    def __init__(self, n, L, N, nodes1d, bc=None):
        """bc: optional ((x-, x+), (y-, y+), (z-, z+)) DG_BC_* codes of the box faces (0: periodic)."""
        n3 = (n, n, n) if np.isscalar(n) else tuple(int(v) for v in n)
        L3 = (L, L, L) if np.isscalar(L) else tuple(float(v) for v in L)
        self.N = int(N)
        self._nodes = np.ascontiguousarray(nodes1d, dtype=np.float64)
        d = capi.dg_hex_desc()
        d.n = (ctypes.c_int32 * 3)(*n3)
        d.L = (ctypes.c_double * 3)(*L3)
        d.N = self.N
        d.nodes1d = self._nodes.ctypes.data_as(ctypes.c_void_p)
        if bc is not None:
            d.bc = (ctypes.c_int32 * 6)(*[int(c) for pair in bc for c in pair])
        h = ctypes.c_void_p()
        check(load().dg_hex_mesh_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        self.K = n3[0] * n3[1] * n3[2]
        self.Np = (self.N + 1) ** 3

    def operators(self):
        M = self.N + 1
        D, w = np.zeros((M, M)), np.zeros(M)
        check(load().dg_hex_operators(self.handle, _hptr(D), _hptr(w)))
        return D, w

    def set_av(self, eps0, s0=None, kappa=0.5):
        """Artificial viscosity for later right-hand sides (eps0 = 0 turns it off); s0 defaults to
        -4 log10 N."""
        p = capi.dg_av_params()
        p.eps0 = float(eps0)
        p.s0 = float(-4.0 * np.log10(self.N) if s0 is None else s0)
        p.kappa = float(kappa)
        check(load().dg_hex_set_av(self.handle, ctypes.byref(p)))

    def av_viscosity(self, q, eps, stream=None):
        """eps [K] (CUDA float64) <- the element viscosities of q under the mesh's parameters."""
        import torch
        if eps.numel() != self.K:
            raise ValueError(f"eps must hold {self.K} values")
        _hex_sized(self, 5, q=q)
        check(load().dg_hex_av_viscosity(self.handle, _dptr(q, torch.float64, "q"), _dptr(eps, torch.float64, "eps"),
                                         _stream_ptr(stream)))

    def set_overintegration(self, enable=True):
        """Weak-form Euler right-hand side with ceil(3 (N+1) / 2) Gauss points per axis."""
        check(load().dg_hex_set_overintegration(self.handle, int(bool(enable))))

    def set_inflow(self, q_in):
        """Conserved state (5 values) imposed on DG_BC_INFLOW box faces."""
        v = np.ascontiguousarray(q_in, dtype=np.float64).reshape(-1)
        check(load().dg_hex_set_inflow(self.handle, _hptr(v), int(v.size)))

    def status(self, reset=True):
        bits = ctypes.c_uint32()
        check(load().dg_hex_status(self.handle, ctypes.byref(bits), int(reset)))
        return bits.value

    def close(self):
        if getattr(self, "handle", None):
            load().dg_hex_mesh_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _hex_sized(mesh: HexMesh, nvar, **tensors):
    for name, t in tensors.items():
        if t is not None and t.numel() != nvar * mesh.K * mesh.Np:
            raise ValueError(f"{name} must hold {nvar} x {mesh.K} x {mesh.Np} values, got {t.numel()}")


def dg_hex_rhs(mesh: HexMesh, gas: Gas, q, rhs, stream=None):
    import torch
    _hex_sized(mesh, 5, q=q, rhs=rhs)
    check(load().dg_hex_rhs(mesh.handle, gas.handle, _dptr(q, torch.float64, "q"), _dptr(rhs, torch.float64, "rhs"),
                            _stream_ptr(stream)))


def dg_hex_rk_stage(mesh: HexMesh, gas: Gas, stage, dt, q_in, q_out, k, stream=None):
    import torch
    _hex_sized(mesh, 5, q_in=q_in, q_out=q_out, k=k)
    check(load().dg_hex_rk_stage(mesh.handle, gas.handle, int(stage), float(dt), _dptr(q_in, torch.float64, "q_in"),
                                 _dptr(q_out, torch.float64, "q_out"), _dptr(k, torch.float64, "k"),
                                 _stream_ptr(stream)))


def hex_lsrk4_step(mesh: HexMesh, gas: Gas, q, dt, steps=1, stream=None, work=None):
    """Advance q in place by ``steps`` LSRK4 steps on the hexahedral mesh (ping-pong buffers)."""
    import torch
    if work is None:
        work = (torch.empty_like(q), torch.zeros_like(q))
    qb, k = work
    cur, nxt = q, qb
    for _ in range(steps):
        for s in range(5):
            dg_hex_rk_stage(mesh, gas, s, dt, cur, nxt, k, stream=stream)
            cur, nxt = nxt, cur
    if cur is not q:
        q.copy_(cur)
    return q


def _velocity(a):
    v = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if v.size != 3:
        raise ValueError("the advection velocity has 3 components")
    return v


def dg_hex_advection_rhs(mesh: HexMesh, velocity, u, rhs, stream=None):
    """rhs = right-hand side of scalar advection of u[K][Np] with the constant velocity[3]."""
    import torch
    _hex_sized(mesh, 1, u=u, rhs=rhs)
    v = _velocity(velocity)
    check(load().dg_hex_advection_rhs(mesh.handle, _hptr(v), _dptr(u, torch.float64, "u"),
                                      _dptr(rhs, torch.float64, "rhs"), _stream_ptr(stream)))


def dg_hex_advection_rk_stage(mesh: HexMesh, velocity, stage, dt, u_in, u_out, k, stream=None):
    import torch
    _hex_sized(mesh, 1, u_in=u_in, u_out=u_out, k=k)
    v = _velocity(velocity)
    check(load().dg_hex_advection_rk_stage(mesh.handle, _hptr(v), int(stage), float(dt),
                                           _dptr(u_in, torch.float64, "u_in"), _dptr(u_out, torch.float64, "u_out"),
                                           _dptr(k, torch.float64, "k"), _stream_ptr(stream)))


def hex_advection_lsrk4_step(mesh: HexMesh, velocity, u, dt, steps=1, stream=None, work=None):
    """Advance u in place by ``steps`` LSRK4 steps of scalar advection (ping-pong buffers)."""
    import torch
    if work is None:
        work = (torch.empty_like(u), torch.zeros_like(u))
    ub, k = work
    cur, nxt = u, ub
    for _ in range(steps):
        for s in range(5):
            dg_hex_advection_rk_stage(mesh, velocity, s, dt, cur, nxt, k, stream=stream)
            cur, nxt = nxt, cur
    if cur is not u:
        u.copy_(cur)
    return u


# ---- learned temperature guess -------------------------------------------------------------

def dg_mlp_set(gas: Gas, params, norm: dict):
    params = np.ascontiguousarray(params, dtype=np.float32)
    n = capi.dg_mlp_norm(**{k: float(v) for k, v in norm.items()})
    check(load().dg_mlp_set(gas.handle, _hptr(params), ctypes.byref(n)))


def dg_mlp_get(gas: Gas):
    params = np.zeros(capi.DG_MLP_PARAMS, dtype=np.float32)
    n = capi.dg_mlp_norm()
    check(load().dg_mlp_get(gas.handle, _hptr(params), ctypes.byref(n)))
    return params, {k: getattr(n, k) for k, _ in capi.dg_mlp_norm._fields_}


def dg_mlp_loss_grad(params, x, t, grad, loss, stream=None):
    import torch
    check(load().dg_mlp_loss_grad(t.numel(), _dptr(params, torch.float32, "params"), _dptr(x, torch.float32, "x"),
                                  _dptr(t, torch.float32, "t"), _dptr(grad, torch.float32, "grad"),
                                  _dptr(loss, torch.float32, "loss"), _stream_ptr(stream)))


def dg_fp64_fma_rate() -> float:
    """Measured FP64 FMA throughput of the current device, TFLOP/s (synchronous)."""
    r = ctypes.c_double()
    check(load().dg_fp64_fma_rate(ctypes.byref(r)))
    return r.value


def dg_mlp_adam_step(t, lr, params, grad, m, v, stream=None):
    """One Adam update in place on float32 CUDA tensors of DG_MLP_PARAMS values (zeroes grad)."""
    import torch
    check(load().dg_mlp_adam_step(int(t), float(lr), _dptr(params, torch.float32, "params"),
                                  _dptr(grad, torch.float32, "grad"), _dptr(m, torch.float32, "m"),
                                  _dptr(v, torch.float32, "v"), _stream_ptr(stream)))


def dg_mlp_train(gas: Gas, e, Y, T, init_params, epochs=20, batch=4096, lr=3e-3, lr_decay=0.9):
    """Train the gas's MLP on device samples (float64 tensors); returns the per-epoch loss history."""
    import torch
    o = capi.dg_mlp_train_opts(epochs=int(epochs), batch=int(batch), lr=float(lr), lr_decay=float(lr_decay))
    init = np.ascontiguousarray(init_params, dtype=np.float32)
    hist = np.zeros(int(epochs), dtype=np.float32)
    check(load().dg_mlp_train(gas.handle, e.numel(), _dptr(e, torch.float64, "e"), _dptr(Y, torch.float64, "Y"),
                              _dptr(T, torch.float64, "T"), _hptr(init), ctypes.byref(o), _hptr(hist)))
    return hist


def dg_mlp_guess(gas: Gas, q, T, stream=None):
    import torch
    check(load().dg_mlp_guess(gas.handle, T.numel(), _dptr(q, torch.float64, "q"), _dptr(T, torch.float64, "T"),
                              _stream_ptr(stream)))


# ---- batched form ----------------------------------------------------------------------------

class Batch:
    """Cases (mesh, gas, dt, CUDA state tensor) advanced together, one graph launch per RK4 step."""

    def __init__(self, cases, autotune=True):
        lib = load()
        arr = (capi.dg_batch_case * len(cases))()
        self._keep = []
        for i, (mesh, gas, dt, q) in enumerate(cases):
            arr[i].mesh = mesh.handle
            arr[i].gas = gas.handle
            arr[i].dt = float(dt)
            arr[i].q_dev = _dptr(q, None, "q")
            self._keep.append((mesh, gas, q))
        h = ctypes.c_void_p()
        check(lib.dg_batch_create(arr, len(cases), capi.DG_BATCH_AUTOTUNE if autotune else 0, ctypes.byref(h)))
        self.handle = h

    def step(self, steps=1, stream=None):
        check(load().dg_batch_step(self.handle, int(steps), _stream_ptr(stream)))

    def tiles(self):
        r = np.zeros((4, 2), dtype=np.int32)
        v = np.zeros(4, dtype=np.int32)
        t = np.zeros((4, 2, 4))
        check(load().dg_batch_tiles(self.handle, _hptr(r), _hptr(v), _hptr(t)))
        return r, v, t

    def status(self, reset=True):
        bits = ctypes.c_uint32()
        check(load().dg_batch_status(self.handle, ctypes.byref(bits), int(reset)))
        return bits.value

    def close(self):
        if getattr(self, "handle", None):
            load().dg_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dg_batch_create(cases, autotune=True) -> Batch:
    return Batch(cases, autotune)
