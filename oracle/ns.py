"""Compressible Navier-Stokes in nodal DG with BR1 (Bassi-Rebay) gradients.

MIRGE-Com solves "the full compressible Navier-Stokes equations" (§5.3) for
"reactive mixture viscous flows" (§5); the paper does not give the viscous
discretisation.  The standard BR1 scheme is used, in two passes, for a perfect
gas with constant viscosity mu, Stokes' hypothesis (no bulk viscosity) and
heat conductivity kappa = mu cp / Pr:

1. DG gradients with the central flux {{w}} = (w- + w+)/2 of the fields
   w = (rho, rho u, rho v, rho w, T):
       dw/dx_d = sum_a (dr_a/dx_d) D_a w + LIFT( Fscale n_d (w+ - w-)/2 ).
   Velocity gradients by the product rule du_i/dx_d = (d(rho u_i)/dx_d - u_i drho/dx_d) / rho.
2. Viscous stress tau_ij = mu (du_i/dx_j + du_j/dx_i) - 2/3 mu (div u) delta_ij,
   heat flux q_d = -kappa dT/dx_d, viscous flux
       Fv_d = (0, tau_0d, tau_1d, tau_2d, sum_i u_i tau_id - q_d),
   and with the total flux G_d = F_d (Euler) - Fv_d:
       dq/dt = -sum_d dG_d/dx_d
               + LIFT( Fscale * ( n.G(q-) - [ f*_LF - n.{{Fv}} ] ) ),
   {{Fv}} = (Fv- + Fv+)/2 built from each side's own nodal gradients.
"""

from __future__ import annotations

import numpy as np

from .euler import (divergence, euler_flux, face_normals, gather, lax_friedrichs, lift, normal_flux,
                    ref_derivatives)


def dg_gradient(ref, geo, conn, w):
    """BR1 gradient of w[F][K][Np] -> [3][F][K][Np]."""
    drdx = geo.drdx()
    dref = ref_derivatives(ref, w)
    wM, wP = gather(w, conn.vmapM), gather(w, conn.vmapP)
    jump = 0.5 * (wP - wM)
    n = face_normals(geo, ref.Nfp)
    out = np.zeros((3,) + w.shape)
    for d in range(3):
        for a in range(3):
            out[d] += drdx[a, d][None, :, None] * dref[a]
        out[d] += lift(ref, geo, n[d][None] * jump)
    return out


def viscous_flux(q, T, grad, mu, kappa):
    """Viscous flux Fv[3][5][...] from the BR1 gradients grad[3][5][...] of (rho, rho u, rho v, rho w, T)."""
    rho = q[0]
    vel = q[1:4] / rho
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
    Fv = np.zeros((3, 5) + rho.shape)
    for d in range(3):
        for i in range(3):
            Fv[d, 1 + i] = tau[i, d]
        Fv[d, 4] = vel[0] * tau[0, d] + vel[1] * tau[1, d] + vel[2] * tau[2, d] + kappa * grad[d, 4]
    return Fv


def rhs_ns(ref, geo, conn, q, gas, mu, Pr):
    """Navier-Stokes right-hand side [5][K][Np] for a perfect gas ``gas`` (gamma, R)."""
    kappa = mu * gas.cp / Pr
    p, c = gas.pressure_sound_speed(q)
    T = p / (q[0] * gas.R)
    w = np.stack([q[0], q[1], q[2], q[3], T])
    grad = dg_gradient(ref, geo, conn, w)
    Fv = viscous_flux(q, T, grad, mu, kappa)
    G = euler_flux(q, p) - Fv
    div = divergence(ref, geo, G)
    n = face_normals(geo, ref.Nfp)
    qM, qP = gather(q, conn.vmapM), gather(q, conn.vmapP)
    pM, pP = gather(p[None], conn.vmapM)[0], gather(p[None], conn.vmapP)[0]
    cM, cP = gather(c[None], conn.vmapM)[0], gather(c[None], conn.vmapP)[0]
    FvM = np.stack([gather(Fv[d], conn.vmapM) for d in range(3)])
    FvP = np.stack([gather(Fv[d], conn.vmapP) for d in range(3)])
    fstar = lax_friedrichs(qM, qP, pM, pP, cM, cP, n) - 0.5 * normal_flux(FvM + FvP, n)
    GM = euler_flux(qM, pM) - FvM
    return -div + lift(ref, geo, normal_flux(GM, n) - fstar)
