"""Oracle of shock capturing by artificial viscosity on the tetrahedral path.  Test infrastructure
only: imported by tests/, __graft_entry__.smoke() and bench.py's CPU legs, never by the library.

The paper stabilises its shock cases with artificial viscosity, over-integration and limiting
(§5.3) without writing any of them out.  The reading here is the sub-cell shock capturing of
Persson and Peraire (2006), restated from its definitions:

* smoothness indicator per element, on the density: S_e = ||u - P u||^2 / ||u||^2 with P the
  L2 projection onto polynomials of degree <= N-1 on the element (for an orthonormal modal
  basis: the energy of the degree-N modes over the total), s_e = log10 S_e;
* viscosity per element: eps_e = 0 for s_e < s0 - kappa, eps0 for s_e > s0 + kappa, and
  eps0/2 (1 + sin(pi (s_e - s0) / (2 kappa))) in between;
* artificial-viscosity term added to every conserved variable: d q/dt += div(eps grad q),
  with BR1 central fluxes in both passes: sigma = eps_e grad_h q, where grad_h q has the lifted
  jump (q+ - q-)/2, and div_h sigma has the lifted jump n.(sigma+ - sigma-)/2.  At a boundary
  face q+ is the face's ghost state (oracle/boundary.py) and sigma+ = sigma- (no artificial
  flux through boundaries beyond the interior one).
"""

from __future__ import annotations

import mpmath
import numpy as np

from .boundary import exterior_state
from .euler import divergence, face_normals, gather, lift, normal_flux, ref_derivatives
from .refelem import _monomials3, _to_np, exponents3, tet_monomial_integral


_RESIDUAL_CACHE = {}


def _residual_operator(ref):
    """Nodal matrices (I - P, M) of the element: P the L2 projection onto the polynomials of
    degree <= N-1, M the mass matrix, both from the monomial basis with exact integrals, in
    40-digit arithmetic (mpmath), rounded to float64 once."""
    key = (ref.N, ref.nodes.tobytes())
    if key not in _RESIDUAL_CACHE:
        N, Np = ref.N, ref.Np
        ex = exponents3(N)
        with mpmath.workdps(40):
            V = _monomials3(ref.nodes, N)  # [Np][Np]: node i, monomial m
            G = mpmath.matrix([[mpmath.mpf(tet_monomial_integral(a1 + a2, b1 + b2, c1 + c2).numerator) /
                                tet_monomial_integral(a1 + a2, b1 + b2, c1 + c2).denominator
                                for (a2, b2, c2) in ex] for (a1, b1, c1) in ex])
            Vi = V ** -1
            M = Vi.T * G * Vi  # nodal mass matrix of the reference element
            low = [i for i, e in enumerate(ex) if sum(e) <= N - 1]
            Q = mpmath.matrix(Np, len(low))
            for i in range(Np):
                for j, m in enumerate(low):
                    Q[i, j] = V[i, m]
            P = Q * (Q.T * M * Q) ** -1 * Q.T * M
            R = mpmath.eye(Np) - P
            _RESIDUAL_CACHE[key] = (_to_np(R), _to_np(M))
    return _RESIDUAL_CACHE[key]


def smoothness_indicator(ref, u):
    """S_e of u[K][Np] (nodal values), per element [K]: the L2 energy of u - P_{N-1} u over the
    energy of u, P_{N-1} the L2 projection onto degree <= N-1 (the element's affine map has a
    constant Jacobian, which cancels)."""
    R, M = _residual_operator(ref)
    u = np.asarray(u, dtype=np.float64)
    res = u @ R.T
    return np.einsum("ki,ij,kj->k", res, M, res) / np.einsum("ki,ij,kj->k", u, M, u)


def viscosity(S, eps0, s0, kappa):
    """eps_e from the indicator S_e (s_e = log10 S_e; S_e = 0 gives 0)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.log10(S)
        ramp = 0.5 * eps0 * (1.0 + np.sin(np.pi * (s - s0) / (2.0 * kappa)))
    return np.where(s < s0 - kappa, 0.0, np.where(s > s0 + kappa, eps0, ramp))


def element_viscosity(ref, q, eps0, s0, kappa):
    """eps_e [K] from the density q[0]."""
    return viscosity(smoothness_indicator(ref, q[0]), eps0, s0, kappa)


def br1_gradient(ref, geo, conn, q, q_in=None):
    """grad_h q [3][V][K][Np] with the central flux; exterior values from the ghost states."""
    n = face_normals(geo, ref.Nfp)
    qM = gather(q, conn.vmapM)
    bc = conn.bc if conn.bc is not None else np.zeros(conn.vmapM.shape, dtype=np.int64)
    qP = exterior_state(qM, gather(q, conn.vmapP), bc, n, q_in)
    drdx = geo.drdx()
    dref = ref_derivatives(ref, q)
    out = np.zeros((3,) + q.shape)
    for d in range(3):
        for a in range(3):
            out[d] += drdx[a, d][None, :, None] * dref[a]
        out[d] += lift(ref, geo, n[d][None] * 0.5 * (qP - qM))
    return out


def rhs_av(ref, geo, conn, q, eps, q_in=None):
    """div_h(eps grad_h q) [V][K][Np] for the per-element viscosity eps [K]."""
    grad = br1_gradient(ref, geo, conn, q, q_in)
    sigma = eps[None, None, :, None] * grad  # [3][V][K][Np]
    n = face_normals(geo, ref.Nfp)
    sM = np.stack([gather(sigma[d], conn.vmapM) for d in range(3)])
    sP = np.stack([gather(sigma[d], conn.vmapP) for d in range(3)])
    if conn.bc is not None:
        sP = np.where((conn.bc != 0)[None, None], sM, sP)
    return divergence(ref, geo, sigma) + lift(ref, geo, 0.5 * (normal_flux(sP, n) - normal_flux(sM, n)))
