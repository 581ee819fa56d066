"""Oracle of the boundary conditions of the tetrahedral Euler and Navier-Stokes right-hand sides.
Test infrastructure only: imported by tests/, __graft_entry__.smoke() and bench.py's CPU legs,
never by the library.

The paper's wall-bounded and inflow/outflow runs (§5.3: the shock/boundary-layer case, the
forward-facing step; §5.4) do not write out how boundaries enter the discretisation.  The
reading here is the ghost-state (weak) treatment: at a node of a boundary face the exterior
trace q+ is built from the interior trace q- and the outward unit normal n, and the interior
numerical fluxes are used unchanged with that q+ (§8(f)2 of the scope):

* slip wall (adiabatic, inviscid wall): q+ = (rho, m - 2 (m.n) n, rho E, rho Y), the mirror
  state, so the Lax-Friedrichs mass and energy fluxes through the face vanish;
* no-slip adiabatic wall: q+ = (rho, -m, rho E, rho Y), so the central trace of the velocity is
  zero and T+ = T-;
* supersonic inflow: q+ = q_in, a prescribed constant state;
* supersonic outflow: q+ = q-.
Navier-Stokes (BR1, central fluxes): the exterior values of the gradient pass are w+ = w(q+);
the exterior normal viscous fluxes, with traction t = tau n and energy flux e = n.Q
(Q = u.tau + kappa grad T), are
* no-slip adiabatic wall: t+ = t-, e+ = -e-: the wall takes the interior traction and no heat
  or work crosses it;
* slip wall (shear-free, adiabatic): t+ = 2 (n.t-) n - t-, e+ = -e-: the central traction is
  the normal part of the interior one;
* inflow and outflow: t+ = t-, e+ = e- (the central viscous flux is the interior one).

Mixtures (the multi-species Euler right-hand side, §5.4's reacting runs in walled geometry
without the reactions): the same ghost states, species densities carried like the density.  A
wall or outflow ghost keeps the node's rho, |m|, rho E and rho Y, hence its internal energy, so
its temperature is the node's own (T+ = T-); an inflow ghost has the temperature of q_in, the
root of e(T) = e_in that a Newton solve gives (rhs_mixture_bc takes it as T_in).

Codes (the library's DG_BC_* values): 1 slip wall, 2 no-slip wall, 3 inflow, 4 outflow.
"""

from __future__ import annotations

import numpy as np

from .euler import divergence, euler_flux, face_normals, gather, lax_friedrichs, lift, normal_flux
from .euler import ref_derivatives
from .ns import viscous_flux

SLIP_WALL, NOSLIP_WALL, INFLOW, OUTFLOW = 1, 2, 3, 4


def exterior_state(qM, qP_interior, bc, n, q_in=None):
    """q+ at every face node: the neighbour's trace on interior faces, the ghost state of the
    face's boundary condition elsewhere.  qM, qP_interior [V][K][4 Nfp]; bc [K][4 Nfp]; n [3][K][4 Nfp]."""
    qP = np.array(qP_interior, copy=True)
    mn = qM[1] * n[0] + qM[2] * n[1] + qM[3] * n[2]
    slip = bc == SLIP_WALL
    for d in range(3):
        qP[1 + d] = np.where(slip, qM[1 + d] - 2.0 * mn * n[d], qP[1 + d])
    noslip = bc == NOSLIP_WALL
    for d in range(3):
        qP[1 + d] = np.where(noslip, -qM[1 + d], qP[1 + d])
    for v in (0, 4) + tuple(range(5, qM.shape[0])):
        qP[v] = np.where(slip | noslip, qM[v], qP[v])
    inflow = bc == INFLOW
    if np.any(inflow):
        if q_in is None:
            raise ValueError("inflow faces need the inflow state q_in")
        for v in range(qM.shape[0]):
            qP[v] = np.where(inflow, q_in[v], qP[v])
    outflow = bc == OUTFLOW
    for v in range(qM.shape[0]):
        qP[v] = np.where(outflow, qM[v], qP[v])
    return qP


def _traces(conn, geo, ref, q, q_in):
    n = face_normals(geo, ref.Nfp)
    qM = gather(q, conn.vmapM)
    qP = exterior_state(qM, gather(q, conn.vmapP), conn.bc, n, q_in)
    return n, qM, qP


def rhs_euler_bc(ref, geo, conn, q, gas, q_in=None, form="strong"):
    """Euler right-hand side [5][K][Np] of a perfect gas with boundary faces (strong or weak form)."""
    p, c = gas.pressure_sound_speed(q)
    F = euler_flux(q, p)
    n, qM, qP = _traces(conn, geo, ref, q, q_in)
    pM, cM = gas.pressure_sound_speed(qM)
    pP, cP = gas.pressure_sound_speed(qP)
    fstar = lax_friedrichs(qM, qP, pM, pP, cM, cP, n)
    if form == "strong":
        return -divergence(ref, geo, F) + lift(ref, geo, normal_flux(euler_flux(qM, pM), n) - fstar)
    return _weak_volume(ref, geo, F) - lift(ref, geo, fstar)


def rhs_mixture_bc(ref, geo, conn, q, gas, T, q_in=None, T_in=None, form="strong"):
    """Euler right-hand side [5 + ns][K][Np] of a NASA-7 mixture with boundary faces (strong or weak
    form).  T [K][Np]: the node temperatures of q (the temperature solve's); T_in: the temperature
    of the inflow state q_in.  The exterior temperature is the neighbour's on interior faces, the
    node's own at wall and outflow ghosts (their internal energy is the node's) and T_in at inflow
    ghosts; p and c of both traces follow from (q, T) as at the nodes."""
    p, c = gas.pressure_sound_speed(q, T)
    F = euler_flux(q, p)
    n, qM, qP = _traces(conn, geo, ref, q, q_in)
    TM = gather(T[None], conn.vmapM)[0]
    TP = gather(T[None], conn.vmapP)[0]  # a boundary face node points at itself
    inflow = conn.bc == INFLOW
    if np.any(inflow):
        if T_in is None:
            raise ValueError("inflow faces need the inflow temperature T_in")
        TP = np.where(inflow, T_in, TP)
    pM, cM = gas.pressure_sound_speed(qM, TM)
    pP, cP = gas.pressure_sound_speed(qP, TP)
    fstar = lax_friedrichs(qM, qP, pM, pP, cM, cP, n)
    if form == "strong":
        return -divergence(ref, geo, F) + lift(ref, geo, normal_flux(euler_flux(qM, pM), n) - fstar)
    return _weak_volume(ref, geo, F) - lift(ref, geo, fstar)


def _weak_volume(ref, geo, F):
    drdx = geo.drdx()
    Minv = ref.Minv
    out = np.zeros(F.shape[1:])
    for a, D in enumerate((ref.Dr, ref.Ds, ref.Dt)):
        W = Minv @ D.T @ ref.M
        Fa = sum(drdx[a, d][None, :, None] * F[d] for d in range(3))
        out += np.einsum("ij,vkj->vki", W, Fa)
    return out


def _w_of(q, gas):
    p, _ = gas.pressure_sound_speed(q)
    return np.stack([q[0], q[1], q[2], q[3], p / (q[0] * gas.R)])


def viscous_flux_bc(ref, geo, conn, q, gas, mu, Pr, q_in=None):
    """The first BR1 pass: the viscous flux Fv[3][5][K][Np] of q from the BR1 gradients of
    w = (rho, rho u, rho v, rho w, T) with central fluxes, exterior values w(q+) at boundary faces."""
    kappa = mu * gas.cp / Pr
    n, qM, qP = _traces(conn, geo, ref, q, q_in)
    w = _w_of(q, gas)
    wM, wP = gather(w, conn.vmapM), _w_of(qP, gas)
    drdx = geo.drdx()
    dref = ref_derivatives(ref, w)
    grad = np.zeros((3,) + w.shape)
    for d in range(3):
        for a in range(3):
            grad[d] += drdx[a, d][None, :, None] * dref[a]
        grad[d] += lift(ref, geo, n[d][None] * 0.5 * (wP - wM))
    return viscous_flux(q, w[4], grad, mu, kappa)


def ns_face_flux(ref, geo, conn, q, gas, Fv, q_in=None):
    """Normal numerical flux n.G* [5][K][4 Nfp] of G = F - Fv at the face nodes: Lax-Friedrichs for
    the Euler part and the central viscous flux, with the exterior viscous fluxes of the boundary
    conditions; also n, q-, p- and the interior viscous flux FvM [3][5][K][4 Nfp]."""
    n, qM, qP = _traces(conn, geo, ref, q, q_in)
    FvM = np.stack([gather(Fv[d], conn.vmapM) for d in range(3)])
    nvM = normal_flux(FvM, n)  # [5][K][4 Nfp]: 0, traction t, energy flux e
    nvP = normal_flux(np.stack([gather(Fv[d], conn.vmapP) for d in range(3)]), n)
    nvP = np.where((conn.bc != 0)[None], nvM, nvP)
    wall = (conn.bc == NOSLIP_WALL) | (conn.bc == SLIP_WALL)
    nvP[4] = np.where(wall, -nvM[4], nvP[4])
    tn = nvM[1] * n[0] + nvM[2] * n[1] + nvM[3] * n[2]
    for i in range(3):
        nvP[1 + i] = np.where(conn.bc == SLIP_WALL, 2.0 * tn * n[i] - nvM[1 + i], nvP[1 + i])
    pM, cM = gas.pressure_sound_speed(qM)
    pP, cP = gas.pressure_sound_speed(qP)
    fstar = lax_friedrichs(qM, qP, pM, pP, cM, cP, n) - 0.5 * (nvM + nvP)
    return fstar, n, qM, pM, FvM


def rhs_ns_bc(ref, geo, conn, q, gas, mu, Pr, q_in=None, form="strong", Fv=None):
    """Navier-Stokes right-hand side [5][K][Np] (BR1, central fluxes) with boundary faces.  Fv: the
    viscous flux of the first BR1 pass (viscous_flux_bc), computed here when not given (a
    partitioned run passes it with its halo filled from the owners)."""
    p, c = gas.pressure_sound_speed(q)
    if Fv is None:
        Fv = viscous_flux_bc(ref, geo, conn, q, gas, mu, Pr, q_in)
    fstar, n, qM, pM, FvM = ns_face_flux(ref, geo, conn, q, gas, Fv, q_in)
    G = euler_flux(q, p) - Fv
    if form == "strong":
        GM = euler_flux(qM, pM) - FvM
        return -divergence(ref, geo, G) + lift(ref, geo, normal_flux(GM, n) - fstar)
    return _weak_volume(ref, geo, G) - lift(ref, geo, fstar)
