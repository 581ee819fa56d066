"""Oracle of nodal DG on tensor-product hexahedra (the paper's element type in its timed runs,
§5.2-§5.4: "tensor product elements"), Euler equations of a perfect gas.  Test infrastructure
only: imported by tests/, __graft_entry__.smoke() and bench.py's CPU legs, never by the library.

The paper prints none of the discretisation; this follows the collocated nodal spectral-element
DG on Gauss-Lobatto-Legendre points, written from its definitions:

* 1-D nodal basis l_i through the given node set x_0 < ... < x_N on [-1, 1];
  quadrature weights w_i = integral of l_i over [-1, 1] (exact polynomial integration);
  differentiation matrix D[i][j] = l_j'(x_i).  Evaluated in 40-digit arithmetic (mpmath) and
  rounded once.
* element [x0, x0 + h_x] x ... mapped from [-1, 1]^3: d/dx = (2 / h_x) d/dr; mass matrix
  collocated (diagonal J w_i w_j w_k); face integrals collocated at the face nodes.
* strong form, per conserved variable:
    dq/dt = - sum_d (2/h_d) D_d F_d(q) + sum over the faces f the node lies on of
            (2/h_d(f)) / w_end (n_f . F(q-) - F*_f),
  with the local Lax-Friedrichs flux n.F* = (n.F(q-) + n.F(q+))/2 + lambda (q- - q+)/2,
  lambda = max(|u-.n| + c-, |u+.n| + c+) at the face node; q+ is the neighbour's node at the
  same position on the shared face (periodic box).
* Navier-Stokes: BR1 with central fluxes in both passes, as on tetrahedra
  (oracle/ns.py): grad_d w = (2/h_d) D_d w plus, at the face nodes of the two d-faces,
  (2/h_d)/w_end n_d (w+ - w-)/2, for w = (rho, rho u, rho v, rho w, T); the viscous flux
  (tau, u.tau + kappa grad T) enters G = F - Fv, and the face term gains -n.(Fv- - Fv+)/2;
* artificial viscosity (the reading of oracle/av.py on tensor-product elements): the indicator
  of the density is the energy outside Q_{N-1} (the tensor-product Legendre modes with an index
  equal to N) over the total energy, both in the GLL-weighted inner product, under which the
  Legendre polynomials up to degree N are orthogonal; d q/dt += div(eps grad q) for every
  conserved variable with BR1 central fluxes (exterior q+ of the ghost state at boundary faces,
  exterior flux = interior flux there);
* over-integration (weak form; the paper names it among its shock stabilisations, §5.3): the
  volume integral of grad(phi_i) . F(q_h) with Q Gauss-Legendre points per axis instead of the
  collocated nodes, rhs_vol = sum_d (2/h_d) (A_d (x) B (x) B) F_d(I q), with the interpolation
  I [Q][N+1] from the nodes to the Gauss points, A = W^-1 (I D)^T W_Q along d and
  B = W^-1 I^T W_Q along the other axes (W: nodal weights, W_Q: Gauss weights); the face terms
  are the collocated ones of the weak form;
* boundary conditions on box faces (box["bc"][axis][end], the codes of oracle/boundary.py): q+
  at a boundary face node is the ghost state of the condition, with n = -e_axis or +e_axis;
* weak form (cross-check): dq/dt = sum_d (2/h_d) W^-1 D^T W F_d - sum_f (2/h_d)/w_end n.F*_f;
  with the summation-by-parts identity W D + D^T W = diag(-1, 0, ..., 0, 1) it equals the
  strong form up to rounding.
* scalar advection du/dt + a . grad u = 0, a constant (the paper's GPU comparison workload,
  section 5.2, on p = 1 tensor-product elements): the same strong and weak forms with the flux
  F_d = a_d u and the Lax-Friedrichs flux with lambda = |a . n|, which is the upwind flux
  n.F* = (a.n) u_upwind.

Arrays: q[V][K][Np], node index n = i + (N+1)(j + (N+1)k); element index ex + nx(ey + ny ez).
"""

from __future__ import annotations

from dataclasses import dataclass

import mpmath
import numpy as np

from .euler import euler_flux


@dataclass
class HexRef:
    N: int
    nodes: np.ndarray  # [N+1]
    w: np.ndarray      # [N+1] quadrature weights
    D: np.ndarray      # [N+1][N+1], D[i][j] = l_j'(x_i)


def hex_reference(x1d) -> HexRef:
    x1d = np.asarray(x1d, dtype=np.float64)
    m = x1d.size
    with mpmath.workdps(40):
        xs = [mpmath.mpf(float(v)) for v in x1d]
        w = []
        D = [[mpmath.mpf(0)] * m for _ in range(m)]
        for j in range(m):
            # l_j as a polynomial: coefficients (ascending) of prod_{k != j} (x - x_k) / (x_j - x_k)
            coeff = [mpmath.mpf(1)]
            den = mpmath.mpf(1)
            for k in range(m):
                if k == j:
                    continue
                coeff = [mpmath.mpf(0)] + coeff  # multiply by x
                for a in range(len(coeff) - 1):
                    coeff[a] -= xs[k] * coeff[a + 1]
                den *= xs[j] - xs[k]
            coeff = [c / den for c in coeff]
            # integral over [-1, 1]: sum c_a (1 - (-1)^(a+1)) / (a+1)
            w.append(sum(c * (1 - (-1) ** (a + 1)) / (a + 1) for a, c in enumerate(coeff)))
            dcoeff = [a * coeff[a] for a in range(1, len(coeff))]
            for i in range(m):
                D[i][j] = sum(c * xs[i] ** a for a, c in enumerate(dcoeff))
        w = np.array([float(v) for v in w])
        D = np.array([[float(D[i][j]) for j in range(m)] for i in range(m)])
    return HexRef(N=m - 1, nodes=x1d, w=w, D=D)


def _along(M, a, axis):
    """Apply the 1-D matrix M along tensor axis `axis` (0 = i/x, 1 = j/y, 2 = k/z) of a[..., k, j, i]."""
    ax = {0: -1, 1: -2, 2: -3}[axis]
    a = np.moveaxis(a, ax, -1)
    out = a @ M.T
    return np.moveaxis(out, -1, ax)


def _shape(q, N):
    V, K = q.shape[:2]
    return q.reshape(V, K, N + 1, N + 1, N + 1)  # [V][K][k][j][i]


def _neighbour(box, axis, step):
    """Element index of the periodic neighbour of every element along axis (step = +-1)."""
    nx, ny, nz = box["n"]
    e = np.arange(nx * ny * nz)
    ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
    c = [ex, ey, ez]
    c[axis] = (c[axis] + step) % box["n"][axis]
    return c[0] + nx * (c[1] + ny * c[2])


def _face_slices(N, axis, end):
    """Index tuple selecting the face (axis, end) of a [..., k, j, i] array; end 0 = minus face."""
    idx = [slice(None)] * 3
    idx[2 - axis] = 0 if end == 0 else N
    return (Ellipsis,) + tuple(idx)


def _boundary_elements(box, axis, end):
    """Elements whose face (axis, end) lies on the box boundary."""
    nx, ny, nz = box["n"]
    e = np.arange(nx * ny * nz)
    c = [e % nx, (e // nx) % ny, e // (nx * ny)]
    return c[axis] == (0 if end == 0 else box["n"][axis] - 1)


def _exterior(box, axis, end, qm, qp, q_in):
    """q+ of face (axis, end): the neighbour's trace, or on the box boundary the ghost state of
    the face's condition box["bc"][axis][end] (oracle/boundary.py; n = -e_axis or +e_axis)."""
    code = box.get("bc", ((0, 0), (0, 0), (0, 0)))[axis][end]
    if not code:
        return qp
    from .boundary import exterior_state
    shape = qm.shape[1:]  # [K][face nodes...]
    n = np.zeros((3,) + shape)
    n[axis] = -1.0 if end == 0 else 1.0
    on = _boundary_elements(box, axis, end).reshape((-1,) + (1,) * (len(shape) - 1))
    bc = np.broadcast_to(np.where(on, code, 0), shape)
    return exterior_state(qm, qp, bc, n, q_in)


def _surface_terms(ref, box, q5, gas, q_in=None):
    """Per face (axis, end): (selector, lifting factor, n.F(q-), n.F*) at the face nodes."""
    N = ref.N
    out = []
    for axis in range(3):
        for end in (0, 1):
            sign = -1.0 if end == 0 else 1.0
            nb = _neighbour(box, axis, -1 if end == 0 else 1)
            qm = q5[_face_slices(N, axis, end)]             # [V][K][face]
            qp = q5[:, nb][_face_slices(N, axis, 1 - end)]  # the neighbour's opposite face
            qp = _exterior(box, axis, end, qm, qp, q_in)
            pm, cm = gas.pressure_sound_speed(qm)
            pp, cp = gas.pressure_sound_speed(qp)
            fm = sign * euler_flux(qm, pm)[axis]
            fp = sign * euler_flux(qp, pp)[axis]
            lam = np.maximum(np.abs(sign * qm[1 + axis] / qm[0]) + cm, np.abs(sign * qp[1 + axis] / qp[0]) + cp)
            fstar = 0.5 * (fm + fp) + 0.5 * lam[None] * (qm - qp)
            lift = (2.0 / box["h"][axis]) / ref.w[0 if end == 0 else N]
            out.append((_face_slices(N, axis, end), lift, fm, fstar))
    return out


def _volume_fluxes(q5, gas):
    return list(euler_flux(q5, gas.pressure(q5)))


def hex_rhs_strong(ref, box, q, gas, q_in=None):
    """Strong-form right-hand side, q[5][K][Np] -> rhs[5][K][Np]; box["bc"][axis][end] (optional)
    puts a boundary condition on the box face instead of periodicity."""
    N = ref.N
    q5 = _shape(np.asarray(q, dtype=np.float64), N)
    F = _volume_fluxes(q5, gas)
    rhs = np.zeros_like(q5)
    for d in range(3):
        rhs -= (2.0 / box["h"][d]) * _along(ref.D, F[d], d)
    for sel, lift, fm, fstar in _surface_terms(ref, box, q5, gas, q_in):
        rhs[sel] += lift * (fm - fstar)
    return rhs.reshape(q.shape)


def hex_rhs_weak(ref, box, q, gas, q_in=None):
    """Weak-form right-hand side (the cross-check of the strong form)."""
    N = ref.N
    q5 = _shape(np.asarray(q, dtype=np.float64), N)
    F = _volume_fluxes(q5, gas)
    Wi = np.diag(1.0 / ref.w)
    Mt = Wi @ ref.D.T @ np.diag(ref.w)
    rhs = np.zeros_like(q5)
    for d in range(3):
        rhs += (2.0 / box["h"][d]) * _along(Mt, F[d], d)
    for sel, lift, fm, fstar in _surface_terms(ref, box, q5, gas, q_in):
        rhs[sel] -= lift * fstar
    return rhs.reshape(q.shape)


def _advection_lambda(an):
    """Lax-Friedrichs dissipation coefficient of the flux a u across a face with a.n = an."""
    return abs(an)


def _advection_surface_terms(ref, box, u5, a):
    """Per face (axis, end): (selector, lifting factor, n.F(u-), n.F*) for F = a u."""
    N = ref.N
    out = []
    for axis in range(3):
        for end in (0, 1):
            an = (-1.0 if end == 0 else 1.0) * a[axis]
            nb = _neighbour(box, axis, -1 if end == 0 else 1)
            um = u5[_face_slices(N, axis, end)]
            up = u5[nb][_face_slices(N, axis, 1 - end)]
            fm, fp = an * um, an * up
            fstar = 0.5 * (fm + fp) + 0.5 * _advection_lambda(an) * (um - up)
            lift = (2.0 / box["h"][axis]) / ref.w[0 if end == 0 else N]
            out.append((_face_slices(N, axis, end), lift, fm, fstar))
    return out


def _scalar_shape(u, N):
    u = np.asarray(u, dtype=np.float64)
    return u.reshape(u.shape[-2], N + 1, N + 1, N + 1)  # [K][k][j][i]


def hex_advection_rhs_strong(ref, box, u, a):
    """Strong-form right-hand side of scalar advection with constant velocity a[3]:
    u[K][Np] (or [1][K][Np]) -> rhs of the same shape."""
    u5 = _scalar_shape(u, ref.N)
    rhs = np.zeros_like(u5)
    for d in range(3):
        rhs -= (2.0 / box["h"][d]) * _along(ref.D, a[d] * u5, d)
    for sel, lift, fm, fstar in _advection_surface_terms(ref, box, u5, a):
        rhs[sel] += lift * (fm - fstar)
    return rhs.reshape(np.shape(u))


def hex_advection_rhs_weak(ref, box, u, a):
    """Weak-form right-hand side of scalar advection (the cross-check of the strong form)."""
    u5 = _scalar_shape(u, ref.N)
    Mt = np.diag(1.0 / ref.w) @ ref.D.T @ np.diag(ref.w)
    rhs = np.zeros_like(u5)
    for d in range(3):
        rhs += (2.0 / box["h"][d]) * _along(Mt, a[d] * u5, d)
    for sel, lift, fm, fstar in _advection_surface_terms(ref, box, u5, a):
        rhs[sel] -= lift * fstar
    return rhs.reshape(np.shape(u))


def _w_of(q, gas):
    return np.stack([q[0], q[1], q[2], q[3], gas.temperature(q)])


def hex_gradient(ref, box, w, q=None, gas=None, q_in=None):
    """BR1 gradient grad[3][F][K][Np] of w[F][K][Np] (central flux).  On a box with boundary faces
    (box["bc"]) the exterior values at a boundary face are w(q+) of the ghost state, which needs
    the state q and the gas."""
    N = ref.N
    F = w.shape[0]
    w5 = w.reshape(F, w.shape[1], N + 1, N + 1, N + 1)
    q5 = None if q is None else _shape(np.asarray(q, dtype=np.float64), N)
    out = np.zeros((3,) + w5.shape)
    for d in range(3):
        out[d] = (2.0 / box["h"][d]) * _along(ref.D, w5, d)
        for end in (0, 1):
            nd = -1.0 if end == 0 else 1.0
            nb = _neighbour(box, d, -1 if end == 0 else 1)
            sel = _face_slices(N, d, end)
            wm = w5[sel]
            wp = w5[:, nb][_face_slices(N, d, 1 - end)]
            if box.get("bc", ((0, 0), (0, 0), (0, 0)))[d][end]:
                qm = q5[sel]
                qp = _exterior(box, d, end, qm, q5[:, nb][_face_slices(N, d, 1 - end)], q_in)
                wp = np.where(_boundary_elements(box, d, end).reshape((1, -1, 1, 1)), _w_of(qp, gas), wp)
            lift = (2.0 / box["h"][d]) / ref.w[0 if end == 0 else N]
            out[d][sel] += lift * nd * 0.5 * (wp - wm)
    return out.reshape((3,) + w.shape)


def hex_rhs_ns(ref, box, q, gas, mu, Pr, q_in=None):
    """Navier-Stokes right-hand side [5][K][Np] of a perfect gas.  At boundary faces the exterior
    viscous flux follows the tetrahedral reading (oracle/boundary.py): walls adiabatic
    (E_d+ = -E_d-), a slip wall shear-free (tau_id+ = -tau_id- for i != d, tau_dd+ = tau_dd-),
    inflow and outflow the interior flux."""
    from .ns import viscous_flux
    N = ref.N
    q = np.asarray(q, dtype=np.float64)
    T = gas.temperature(q)
    w = np.stack([q[0], q[1], q[2], q[3], T])
    grad = hex_gradient(ref, box, w, q, gas, q_in)
    Fv = viscous_flux(q, T, grad, mu, mu * gas.cp / Pr)  # [3][5][K][Np]
    q5 = _shape(q, N)
    Fv5 = Fv.reshape((3, 5) + q5.shape[1:])
    Fe = _volume_fluxes(q5, gas)
    rhs = np.zeros_like(q5)
    for d in range(3):
        rhs -= (2.0 / box["h"][d]) * _along(ref.D, Fe[d] - Fv5[d], d)
    for sel, lift, fm, fstar in _surface_terms(ref, box, q5, gas, q_in):
        rhs[sel] += lift * (fm - fstar)
    # central viscous flux: the face term gains -n.(Fv- - Fv+)/2
    for d, end, sel, lift, nd, fvm, fvp in _viscous_face_traces(ref, box, Fv5):
        rhs[sel] -= lift * nd * 0.5 * (fvm - fvp)
    return rhs.reshape(q.shape)


def _viscous_face_traces(ref, box, Fv5):
    """Per axis d and end: the face's node slice, lift factor (2/h_d)/w_end, normal sign, and the
    interior and exterior viscous fluxes along d [5][...]; at a box boundary the exterior flux is
    the interior one, except that walls are adiabatic (E_d+ = -E_d-) and a slip wall is shear-free
    (tau_id+ = -tau_id- for i != d)."""
    from .boundary import NOSLIP_WALL, SLIP_WALL
    N = ref.N
    for d in range(3):
        for end in (0, 1):
            nd = -1.0 if end == 0 else 1.0
            nb = _neighbour(box, d, -1 if end == 0 else 1)
            sel = _face_slices(N, d, end)
            fvm = Fv5[d][sel]
            fvp = Fv5[d][:, nb][_face_slices(N, d, 1 - end)]
            code = box.get("bc", ((0, 0), (0, 0), (0, 0)))[d][end]
            if code:
                ghost = fvm.copy()
                if code in (SLIP_WALL, NOSLIP_WALL):
                    ghost[4] = -fvm[4]
                if code == SLIP_WALL:
                    for i in range(3):
                        if i != d:
                            ghost[1 + i] = -fvm[1 + i]
                on = _boundary_elements(box, d, end).reshape((1, -1, 1, 1))
                fvp = np.where(on, ghost, fvp)
            lift = (2.0 / box["h"][d]) / ref.w[0 if end == 0 else N]
            yield d, end, sel, lift, nd, fvm, fvp


def _gauss_operators(ref, Q):
    """(I, A, B) of the over-integration with Q Gauss-Legendre points (see the module notes)."""
    xg, wg = np.polynomial.legendre.leggauss(Q)
    x = ref.nodes
    M = x.size
    I = np.ones((Q, M))
    for j in range(M):
        for k in range(M):
            if k != j:
                I[:, j] *= (xg - x[k]) / (x[j] - x[k])
    A = (np.diag(1.0 / ref.w) @ (I @ ref.D).T) * wg[None, :]
    B = (np.diag(1.0 / ref.w) @ I.T) * wg[None, :]
    return I, A, B


def _along_rect(Mx, a, axis):
    """Apply the rectangular matrix Mx [out][in] along tensor axis `axis` of a[..., k, j, i]."""
    ax = {0: -1, 1: -2, 2: -3}[axis]
    a = np.moveaxis(a, ax, -1)
    return np.moveaxis(a @ Mx.T, -1, ax)


def hex_overint_volume(ref, box, q5, gas, Q, Fv5=None):
    """Over-integrated volume term [5][K][M][M][M] of the weak form; with a nodal viscous flux
    Fv5 [3][5][K][M][M][M], of G = F(I q) - I Fv."""
    I, A, B = _gauss_operators(ref, Q)
    qg = q5
    for d in range(3):
        qg = _along_rect(I, qg, d)  # nodes -> Gauss points along every axis
    Fg = _volume_fluxes(qg, gas)
    out = np.zeros_like(q5)
    for d in range(3):
        t = Fg[d]
        if Fv5 is not None:
            fvg = Fv5[d]
            for e in range(3):
                fvg = _along_rect(I, fvg, e)
            t = t - fvg
        for e in range(3):
            t = _along_rect(A if e == d else B, t, e)
        out += (2.0 / box["h"][d]) * t
    return out


def hex_rhs_overint(ref, box, q, gas, Q, q_in=None):
    """Weak-form Euler right-hand side with over-integrated volume fluxes (Q Gauss points per axis)."""
    N = ref.N
    q5 = _shape(np.asarray(q, dtype=np.float64), N)
    rhs = hex_overint_volume(ref, box, q5, gas, Q)
    for sel, lift, fm, fstar in _surface_terms(ref, box, q5, gas, q_in):
        rhs[sel] -= lift * fstar
    return rhs.reshape(np.shape(q))


def hex_indicator(ref, u):
    """Smoothness indicator S_e of nodal values u[K][Np]: GLL-weighted energy of the Legendre modes
    outside Q_{N-1} over the total."""
    N = ref.N
    L = np.stack([np.polynomial.legendre.Legendre.basis(a)(ref.nodes) for a in range(N + 1)])  # [a][i]
    norm = (L ** 2) @ ref.w  # discrete norms
    T = (L * ref.w[None, :]) / norm[:, None]  # nodal values -> Legendre coefficients
    u5 = np.asarray(u, dtype=np.float64).reshape(-1, N + 1, N + 1, N + 1)  # [K][k][j][i]
    c = np.einsum("ai,bj,ck,ekji->ecba", T, T, T, u5)  # [K][c][b][a]
    e = c ** 2 * (norm[:, None, None] * norm[None, :, None] * norm[None, None, :])[None]  # [K][c][b][a]
    a, b, cc = np.meshgrid(np.arange(N + 1), np.arange(N + 1), np.arange(N + 1), indexing="ij")  # [c][b][a]
    top = np.maximum(np.maximum(a, b), cc) == N
    return e[:, top].sum(axis=1) / e.reshape(e.shape[0], -1).sum(axis=1)


def hex_gradient_state(ref, box, q, q_in=None):
    """BR1 gradient [3][5][K][Np] of the conserved variables themselves (exterior values: the
    ghost state q+ at boundary faces)."""
    N = ref.N
    q5 = _shape(np.asarray(q, dtype=np.float64), N)
    out = np.zeros((3,) + q5.shape)
    for d in range(3):
        out[d] = (2.0 / box["h"][d]) * _along(ref.D, q5, d)
        for end in (0, 1):
            nd = -1.0 if end == 0 else 1.0
            nb = _neighbour(box, d, -1 if end == 0 else 1)
            sel = _face_slices(N, d, end)
            qm = q5[sel]
            qp = _exterior(box, d, end, qm, q5[:, nb][_face_slices(N, d, 1 - end)], q_in)
            lift = (2.0 / box["h"][d]) / ref.w[0 if end == 0 else N]
            out[d][sel] += lift * nd * 0.5 * (qp - qm)
    return out.reshape((3,) + np.shape(q))


def hex_rhs_av(ref, box, q, eps, q_in=None):
    """div_h(eps grad_h q) [5][K][Np] for the per-element viscosity eps[K] (central fluxes)."""
    N = ref.N
    grad = hex_gradient_state(ref, box, q, q_in)
    sig = (eps[None, None, :, None] * grad).reshape((3, 5, -1, N + 1, N + 1, N + 1))
    out = np.zeros(sig.shape[1:])
    for d in range(3):
        out += (2.0 / box["h"][d]) * _along(ref.D, sig[d], d)
        for end in (0, 1):
            nd = -1.0 if end == 0 else 1.0
            nb = _neighbour(box, d, -1 if end == 0 else 1)
            sel = _face_slices(N, d, end)
            sm = sig[d][sel]
            sp = sig[d][:, nb][_face_slices(N, d, 1 - end)]
            if box.get("bc", ((0, 0), (0, 0), (0, 0)))[d][end]:
                sp = np.where(_boundary_elements(box, d, end).reshape((1, -1, 1, 1)), sm, sp)
            lift = (2.0 / box["h"][d]) / ref.w[0 if end == 0 else N]
            out[sel] += lift * nd * 0.5 * (sp - sm)
    return out.reshape(np.shape(q))


def hex_integrate(ref, box, u):
    """sum over elements of J sum_nodes w_i w_j w_k u, for u[..., K, Np]."""
    N = ref.N
    w3 = (ref.w[None, None, :] * ref.w[None, :, None] * ref.w[:, None, None]).ravel()  # [Np] with k, j, i
    J = np.prod(box["h"]) / 8.0
    return J * np.tensordot(u, w3, axes=([-1], [0])).sum(axis=-1)


def hex_rhs_overint_ns(ref, box, q, gas, mu, Pr, Q, q_in=None):
    """Weak-form Navier-Stokes right-hand side with over-integrated volume fluxes (Q Gauss points per
    axis): the whole flux G = F - Fv on the points, with the nodal BR1 viscous flux Fv interpolated
    to them (a degree-N field per axis, so its part is exact), and the weak-form face term with the
    central viscous flux and the walls' exterior viscous fluxes of hex_rhs_ns."""
    from .ns import viscous_flux
    N = ref.N
    q = np.asarray(q, dtype=np.float64)
    T = gas.temperature(q)
    w = np.stack([q[0], q[1], q[2], q[3], T])
    grad = hex_gradient(ref, box, w, q, gas, q_in)
    Fv = viscous_flux(q, T, grad, mu, mu * gas.cp / Pr)  # [3][5][K][Np]
    q5 = _shape(q, N)
    Fv5 = Fv.reshape((3, 5) + q5.shape[1:])
    rhs = hex_overint_volume(ref, box, q5, gas, Q, Fv5)
    for sel, lift, fm, fstar in _surface_terms(ref, box, q5, gas, q_in):
        rhs[sel] -= lift * fstar
    for d, end, sel, lift, nd, fvm, fvp in _viscous_face_traces(ref, box, Fv5):
        rhs[sel] += lift * nd * 0.5 * (fvm + fvp)
    return rhs.reshape(q.shape)


def hex_rhs_overint_av(ref, box, q, gas, eps, Q, mu=0.0, Pr=0.71, q_in=None):
    """The over-integrated Euler (mu = 0) or Navier-Stokes right-hand side with the artificial-
    viscosity term of hex_rhs_av: its flux sigma = eps grad_h q (a degree-N field per axis in each
    element) is interpolated to the Gauss points and integrated with the other fluxes, and the
    face terms gain its central flux n.(sigma- + sigma+)/2, sigma+ = sigma- at box boundaries."""
    from .ns import viscous_flux
    N = ref.N
    q = np.asarray(q, dtype=np.float64)
    q5 = _shape(q, N)
    sig5 = (eps[None, None, :, None] * hex_gradient_state(ref, box, q, q_in)).reshape((3, 5) + q5.shape[1:])
    Fv5 = None
    if mu > 0:
        T = gas.temperature(q)
        grad = hex_gradient(ref, box, np.stack([q[0], q[1], q[2], q[3], T]), q, gas, q_in)
        Fv5 = viscous_flux(q, T, grad, mu, mu * gas.cp / Pr).reshape((3, 5) + q5.shape[1:])
    rhs = hex_overint_volume(ref, box, q5, gas, Q, sig5 if Fv5 is None else Fv5 + sig5)
    for sel, lift, fm, fstar in _surface_terms(ref, box, q5, gas, q_in):
        rhs[sel] -= lift * fstar
    if Fv5 is not None:
        for d, end, sel, lift, nd, fvm, fvp in _viscous_face_traces(ref, box, Fv5):
            rhs[sel] += lift * nd * 0.5 * (fvm + fvp)
    for d in range(3):
        for end in (0, 1):
            nd = -1.0 if end == 0 else 1.0
            nb = _neighbour(box, d, -1 if end == 0 else 1)
            sel = _face_slices(N, d, end)
            sm = sig5[d][sel]
            sp = sig5[d][:, nb][_face_slices(N, d, 1 - end)]
            if box.get("bc", ((0, 0), (0, 0), (0, 0)))[d][end]:
                sp = np.where(_boundary_elements(box, d, end).reshape((1, -1, 1, 1)), sm, sp)
            lift = (2.0 / box["h"][d]) / ref.w[0 if end == 0 else N]
            rhs[sel] += lift * nd * 0.5 * (sm + sp)
    return rhs.reshape(q.shape)
