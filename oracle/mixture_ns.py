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
