"""Oracle of over-integration on tetrahedra.  Test infrastructure only: imported by tests/,
__graft_entry__.smoke() and bench.py's CPU legs, never by the library.

§5.3 names over-integration among the stabilisations of its shock runs and does not write it out.
The reading here (the same as on hexahedra): the Euler right-hand side in weak form, with the
volume integral of every test function's gradient against the flux evaluated by a quadrature rule
with more points than nodes, so the flux of the interpolated state is integrated, not its nodal
interpolant:

    rhs_vol = sum_a M^-1 (I D_a)^T W F_a(I q),   F_a = sum_d (dr_a/dx_d) F_d,

* I [Ng][Np]: the nodal basis at the quadrature points (interpolation to the points);
* I D_a: the r_a-derivative of the nodal basis at the points (D_a is exact on degree-N fields);
* W = diag(w_g): the rule's weights on the reference tetrahedron.

The faces keep the collocated weak-form term -LIFT(Fscale f*) with the pointwise Lax-Friedrichs
flux f* of the face-node traces, and boundary faces take the ghost states of oracle/boundary.py.

Navier-Stokes: the whole flux G = F - Fv is integrated on the rule, with the nodal BR1 viscous flux
Fv (oracle/boundary.py viscous_flux_bc) interpolated to the points.  Fv is a degree-N field, so its
part of the integral is exact and equals the collocated weak-form term; the convective part is the
over-integrated one.  The faces take the weak-form normal flux n.G* of the collocated
Navier-Stokes right-hand side (Lax-Friedrichs minus the central viscous flux, with the walls'
exterior viscous fluxes).

Rule: the Stroud conical product on the collapsed cube (a, b, c) in [-1, 1]^3,
    r = (1+a)(1-b)(1-c)/4 - 1,  s = (1+b)(1-c)/2 - 1,  t = c,   dr ds dt = (1-b)(1-c)^2/8 da db dc,
with q Gauss-Jacobi points per direction for the weights 1, (1-b) and (1-c)^2 (scipy's roots),
so q^3 points with positive weights, exact for total degree 2q - 1.  The default
q = ceil(3N/2) integrates degree 3N - 1: a degree-(N-1) test-function gradient times a quadratic
flux of degree-N fields, the tetrahedral counterpart of the 3/2 rule.
"""

from __future__ import annotations

import functools

import mpmath
import numpy as np
from scipy.special import roots_jacobi

from .boundary import _traces, ns_face_flux, viscous_flux_bc
from .euler import euler_flux, lax_friedrichs, lift
from .refelem import _DPS, _monomials3, _to_np


def default_points(N):
    """Gauss-Jacobi points per collapsed direction: ceil(3N/2)."""
    return (3 * N + 1) // 2


@functools.lru_cache(maxsize=None)
def tet_rule(q):
    """(points [q^3][3], weights [q^3]) of the Stroud conical product rule on the reference
    tetrahedron; the point of (a_i, b_j, c_k) is row (k q + j) q + i."""
    a, wa = roots_jacobi(q, 0.0, 0.0)
    b, wb = roots_jacobi(q, 1.0, 0.0)
    c, wc = roots_jacobi(q, 2.0, 0.0)
    C, B, A = np.meshgrid(c, b, a, indexing="ij")
    WC, WB, WA = np.meshgrid(wc, wb, wa, indexing="ij")
    r = 0.25 * (1 + A) * (1 - B) * (1 - C) - 1
    s = 0.5 * (1 + B) * (1 - C) - 1
    t = C
    pts = np.stack([r.ravel(), s.ravel(), t.ravel()], axis=1)
    return pts, (WA * WB * WC / 8.0).ravel()


@functools.lru_cache(maxsize=None)
def _interp_cached(nodes_key, N, q):
    nodes = np.array(nodes_key).reshape(-1, 3)
    pts, _ = tet_rule(q)
    with mpmath.workdps(_DPS):
        return _to_np(_monomials3(pts, N) * mpmath.inverse(_monomials3(nodes, N)))


def interpolation(ref, q):
    """I [q^3][Np]: the nodal basis of ref at the rule's points (monomial Vandermonde solve in
    extended precision, rounded once)."""
    return _interp_cached(tuple(np.asarray(ref.nodes, dtype=np.float64).ravel()), ref.N, q)


def overint_volume(ref, geo, q, gas, Q, Fv=None):
    """sum_a M^-1 (I D_a)^T W G_a [V][K][Np] with Q points per collapsed direction, G = F(I q), or
    F(I q) - I Fv with a nodal viscous flux Fv [3][5][K][Np]."""
    Iq = interpolation(ref, Q)
    _, w = tet_rule(Q)
    qg = np.einsum("gj,vkj->vkg", Iq, q)  # the state at the points
    p, _ = gas.pressure_sound_speed(qg)
    F = euler_flux(qg, p)  # [3][V][K][Ng]
    if Fv is not None:
        F = F - np.einsum("gj,dvkj->dvkg", Iq, Fv)
    drdx = geo.drdx()  # [a][d][K]
    Minv = ref.Minv
    out = np.zeros(q.shape)
    for a, D in enumerate((ref.Dr, ref.Ds, ref.Dt)):
        Fa = sum(drdx[a, d][None, :, None] * F[d] for d in range(3))
        P = Minv @ (Iq @ D).T  # [Np][Ng]
        out += np.einsum("ig,vkg->vki", P, w[None, None, :] * Fa)
    return out


def rhs_overint(ref, geo, conn, q, gas, Q=None, q_in=None):
    """Weak-form Euler right-hand side [5][K][Np] of a perfect gas with over-integrated volume
    fluxes (Q points per collapsed direction; default ceil(3N/2)); periodic or boundary faces."""
    Q = default_points(ref.N) if Q is None else Q
    n, qM, qP = _traces(conn, geo, ref, q, q_in)
    pM, cM = gas.pressure_sound_speed(qM)
    pP, cP = gas.pressure_sound_speed(qP)
    fstar = lax_friedrichs(qM, qP, pM, pP, cM, cP, n)
    return overint_volume(ref, geo, q, gas, Q) - lift(ref, geo, fstar)


def rhs_overint_ns(ref, geo, conn, q, gas, mu, Pr, Q=None, q_in=None, Fv=None):
    """Weak-form Navier-Stokes right-hand side [5][K][Np] of a perfect gas (BR1, central viscous
    fluxes) with the volume integral of G = F - Fv on the rule (default ceil(3N/2) points per
    collapsed direction); periodic or boundary faces.  Fv: the nodal viscous flux of the first BR1
    pass, computed here when not given."""
    Q = default_points(ref.N) if Q is None else Q
    if Fv is None:
        Fv = viscous_flux_bc(ref, geo, conn, q, gas, mu, Pr, q_in)
    fstar = ns_face_flux(ref, geo, conn, q, gas, Fv, q_in)[0]
    return overint_volume(ref, geo, q, gas, Q, Fv) - lift(ref, geo, fstar)


def rhs_overint_av(ref, geo, conn, q, gas, eps, mu=0.0, Pr=0.71, Q=None, q_in=None):
    """The over-integrated Euler (mu = 0) or Navier-Stokes right-hand side plus the artificial-
    viscosity term div(eps grad_h q) of oracle/av.py for the element viscosities eps [K].  The AV
    flux sigma = eps grad_h q is a degree-N field in each element (eps is constant there), so its
    weak form on the rule is exact and equals that collocated strong term."""
    from .av import rhs_av
    base = (rhs_overint_ns(ref, geo, conn, q, gas, mu, Pr, Q=Q, q_in=q_in) if mu > 0
            else rhs_overint(ref, geo, conn, q, gas, Q=Q, q_in=q_in))
    return base + rhs_av(ref, geo, conn, q, eps, q_in)
