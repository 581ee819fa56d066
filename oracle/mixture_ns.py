"""Oracle of the Navier-Stokes right-hand side of a NASA-7 mixture with species diffusion, on
periodic tetrahedral meshes.  Test infrastructure only: imported by tests/,
__graft_entry__.smoke() and bench.py's CPU legs, never by the library.

The paper's solver targets viscous multi-species flows (§4, §5: "reactive mixture viscous
flows") and names none of the transport model.  The reading here is the simplest closed one:
* viscosity mu constant, Stokes hypothesis (no bulk viscosity), as for the single gas;
* heat conduction kappa = mu cp_mix(T, Y) / Pr, per node;
* Fickian species diffusion at a constant Schmidt number Sc, with the correction that makes
  the diffusive fluxes sum to zero:  J_k = -(mu / Sc) (grad Y_k - Y_k sum_j grad Y_j);
* the energy flux carries the enthalpy diffusion: q = -kappa grad T + sum_k h_k(T) J_k.
Viscous flux (subtracted from the Euler flux): momentum tau, energy u.tau - q, species -J_k.
BR1 with central fluxes in both passes, on w = (rho, rho u, rho v, rho w, T, Y_1 .. Y_ns);
the velocity gradient by the product rule, as for the single gas (oracle/ns.py).

Boundary faces (rhs_ns_mixture_bc; §5.4 runs its multi-species flows in walled geometry): the
ghost states of oracle/boundary.py, with the temperature of rhs_mixture_bc (the node's own at walls
and outflow, T_in at inflow).  The gradient pass takes w+ = w(q+, T+).  The exterior normal viscous
fluxes are those of the single gas for the traction and the energy (a no-slip wall takes the
interior traction, a slip wall only its normal part; both are adiabatic, e+ = -e-, and e holds the
enthalpy diffusion too), and walls are impermeable to diffusion: the species rows' normal flux
s_k = n.(-J_k) has s_k+ = -s_k-.  Inflow and outflow take the interior viscous flux.
"""

from __future__ import annotations

import numpy as np

from .euler import divergence, euler_flux, face_normals, gather, lax_friedrichs, lift, normal_flux
from .ns import dg_gradient


def viscous_flux_mixture(q, T, grad, gas, mu, Pr, Sc):
    """Fv[3][V][...] from the BR1 gradients grad[3][W][...] of w = (rho, rho u, T, Y_k)."""
    rho, vel, Y, _ = gas.split_state(q)
    ns = Y.shape[0]
    du = np.empty((3, 3) + rho.shape)  # du[i][d] = d u_i / d x_d
    for i in range(3):
        for d in range(3):
            du[i, d] = (grad[d, 1 + i] - vel[i] * grad[d, 0]) / rho
    divu = du[0, 0] + du[1, 1] + du[2, 2]
    tau = np.empty_like(du)
    for i in range(3):
        for j in range(3):
            tau[i, j] = mu * (du[i, j] + du[j, i])
        tau[i, i] -= 2.0 / 3.0 * mu * divu
    kappa = mu * gas.mixture_cp(T, Y) / Pr
    gY = grad[:, 5:5 + ns]  # [3][ns][...]
    sum_gY = gY.sum(axis=1)  # [3][...]
    J = -(mu / Sc) * (gY - Y[None] * sum_gY[:, None])  # [3][ns][...]
    h = gas.h_species(T)  # [ns][...]
    Fv = np.zeros((3, 5 + ns) + rho.shape)
    for d in range(3):
        for i in range(3):
            Fv[d, 1 + i] = tau[i, d]
        heat = -kappa * grad[d, 4] + np.sum(h * J[d], axis=0)
        Fv[d, 4] = vel[0] * tau[0, d] + vel[1] * tau[1, d] + vel[2] * tau[2, d] - heat
        Fv[d, 5:] = -J[d]
    return Fv


def rhs_ns_mixture(ref, geo, conn, q, gas, T, mu, Pr, Sc):
    """Navier-Stokes right-hand side [5 + ns][K][Np] of the mixture, temperatures T[K][Np]."""
    rho, vel, Y, _ = gas.split_state(q)
    w = np.concatenate([q[0:4], T[None], Y])
    grad = dg_gradient(ref, geo, conn, w)
    Fv = viscous_flux_mixture(q, T, grad, gas, mu, Pr, Sc)
    p, c = gas.pressure_sound_speed(q, T)
    G = euler_flux(q, p) - Fv
    n = face_normals(geo, ref.Nfp)
    qM, qP = gather(q, conn.vmapM), gather(q, conn.vmapP)
    TM, TP = gather(T[None], conn.vmapM)[0], gather(T[None], conn.vmapP)[0]
    pM, cM = gas.pressure_sound_speed(qM, TM)
    pP, cP = gas.pressure_sound_speed(qP, TP)
    FvM = np.stack([gather(Fv[d], conn.vmapM) for d in range(3)])
    FvP = np.stack([gather(Fv[d], conn.vmapP) for d in range(3)])
    fstar = lax_friedrichs(qM, qP, pM, pP, cM, cP, n) - 0.5 * normal_flux(FvM + FvP, n)
    GM = euler_flux(qM, pM) - FvM
    return -divergence(ref, geo, G) + lift(ref, geo, normal_flux(GM, n) - fstar)


def exterior_viscous(nvM, nvP, bc, n):
    """Exterior normal viscous fluxes [V][K][4 Nfp] of the mixture: the neighbour's on interior faces
    (nvP), at boundary faces the interior one except that walls are adiabatic (energy row
    e+ = -e-) and impermeable (species rows s+ = -s-), and a slip wall is shear-free
    (t+ = 2 (n.t-) n - t-)."""
    from .boundary import NOSLIP_WALL, SLIP_WALL
    out = np.where((bc != 0)[None], nvM, nvP)
    wall = (bc == NOSLIP_WALL) | (bc == SLIP_WALL)
    for v in [4] + list(range(5, nvM.shape[0])):
        out[v] = np.where(wall, -nvM[v], out[v])
    tn = nvM[1] * n[0] + nvM[2] * n[1] + nvM[3] * n[2]
    for i in range(3):
        out[1 + i] = np.where(bc == SLIP_WALL, 2.0 * tn * n[i] - nvM[1 + i], out[1 + i])
    return out


def rhs_ns_mixture_bc(ref, geo, conn, q, gas, T, mu, Pr, Sc, q_in=None, T_in=None):
    """Navier-Stokes right-hand side [5 + ns][K][Np] of the mixture on a mesh with boundary faces
    (conn.bc codes), temperatures T[K][Np]; q_in and T_in: the inflow state and its temperature."""
    from .boundary import INFLOW, exterior_state
    n = face_normals(geo, ref.Nfp)
    qM = gather(q, conn.vmapM)
    qP = exterior_state(qM, gather(q, conn.vmapP), conn.bc, n, q_in)
    TM, TP = gather(T[None], conn.vmapM)[0], gather(T[None], conn.vmapP)[0]
    inflow = conn.bc == INFLOW
    if np.any(inflow):
        if T_in is None:
            raise ValueError("inflow faces need the inflow temperature T_in")
        TP = np.where(inflow, T_in, TP)
    # BR1 gradients with the exterior values w(q+, T+)
    rho, vel, Y, _ = gas.split_state(q)
    w = np.concatenate([q[0:4], T[None], Y])
    wM = gather(w, conn.vmapM)
    wP = np.concatenate([qP[0:4], TP[None], qP[5:] / qP[0]])
    drdx = geo.drdx()
    dref = [ref.Dr, ref.Ds, ref.Dt]
    grad = np.zeros((3,) + w.shape)
    for d in range(3):
        for a in range(3):
            grad[d] += drdx[a, d][None, :, None] * np.einsum("ij,vkj->vki", dref[a], w)
        grad[d] += lift(ref, geo, n[d][None] * 0.5 * (wP - wM))
    Fv = viscous_flux_mixture(q, T, grad, gas, mu, Pr, Sc)
    # exterior normal viscous fluxes
    FvM = np.stack([gather(Fv[d], conn.vmapM) for d in range(3)])
    nvM = normal_flux(FvM, n)  # [V][K][4 Nfp]: 0, traction, energy, species
    nvP = exterior_viscous(nvM, normal_flux(np.stack([gather(Fv[d], conn.vmapP) for d in range(3)]), n),
                           conn.bc, n)
    p, c = gas.pressure_sound_speed(q, T)
    pM, cM = gas.pressure_sound_speed(qM, TM)
    pP, cP = gas.pressure_sound_speed(qP, TP)
    fstar = lax_friedrichs(qM, qP, pM, pP, cM, cP, n) - 0.5 * (nvM + nvP)
    G = euler_flux(q, p) - Fv
    GM = euler_flux(qM, pM) - FvM
    return -divergence(ref, geo, G) + lift(ref, geo, normal_flux(GM, n) - fstar)
