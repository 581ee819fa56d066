"""Euler equations in nodal DG: fluxes, Lax-Friedrichs flux, strong and weak form.

The paper's inviscid benchmark solves the Euler equations with a DG
discretisation advanced by explicit RK4 (§5.2); the equations and the
numerical flux are not written out there.  Standard forms used here, for
q = (rho, rho u, rho v, rho w, rho E, rho Y_1..):

    F_d(q) = (rho u_d, rho u u_d + p e_d, rho u_d E + p u_d ... , rho Y_k u_d)
    i.e. F_d[0] = rho u_d,  F_d[1+i] = rho u_i u_d + p delta_id,
         F_d[4] = u_d (rho E + p),  F_d[5+k] = rho Y_k u_d.

Lax-Friedrichs flux at a face node with outward unit normal n (minus = own
element, plus = neighbour), evaluated pointwise:
    f* = 1/2 n.(F(q-) + F(q+)) + lambda/2 (q- - q+),
    lambda = max(|u-.n| + c-, |u+.n| + c+).

Strong form (integrate by parts twice):
    dq/dt = -sum_d dF_d/dx_d + LIFT( Fscale * (n.F(q-) - f*) ),
    dF/dx_d = sum_a (dr_a/dx_d) D_a F   (D_a = Dr, Ds, Dt; r_a = r, s, t).
Weak form (once):
    dq/dt = M^-1 sum_a D_a^T M (sum_d dr_a/dx_d F_d) - LIFT( Fscale * f* ).
For polynomial interpolants on affine elements the two agree up to rounding.
"""

from __future__ import annotations

import numpy as np


def euler_flux(q, p):
    """F[3][V][...] for state q[V][...] and pressure p[...]."""
    rho = q[0]
    vel = q[1:4] / rho
    V = q.shape[0]
    F = np.empty((3,) + q.shape)
    for d in range(3):
        F[d, 0] = q[1 + d]
        for i in range(3):
            F[d, 1 + i] = q[1 + i] * vel[d]
        F[d, 1 + d] += p
        F[d, 4] = vel[d] * (q[4] + p)
        for k in range(5, V):
            F[d, k] = q[k] * vel[d]
    return F


def normal_flux(F, n):
    """n.F for F[3][V][...] and n[3][...] (broadcast over V)."""
    return n[0][None] * F[0] + n[1][None] * F[1] + n[2][None] * F[2]


def lax_friedrichs(qM, qP, pM, pP, cM, cP, n):
    """Pointwise Lax-Friedrichs flux f*[V][...] at face nodes."""
    unM = np.abs(np.sum(qM[1:4] / qM[0] * n, axis=0))
    unP = np.abs(np.sum(qP[1:4] / qP[0] * n, axis=0))
    lam = np.maximum(unM + cM, unP + cP)
    avg = 0.5 * (normal_flux(euler_flux(qM, pM), n) + normal_flux(euler_flux(qP, pP), n))
    return avg + 0.5 * lam[None] * (qM - qP)


def face_normals(geo, Nfp):
    """Per face node normals n[3][K][4 Nfp] (constant on each face of an affine element)."""
    return np.stack([np.repeat(geo.nx, Nfp, axis=1), np.repeat(geo.ny, Nfp, axis=1), np.repeat(geo.nz, Nfp, axis=1)])


def face_fscale(geo, Nfp):
    return np.repeat(geo.Fscale, Nfp, axis=1)  # [K][4 Nfp]


def gather(u, idx):
    """u[V][K][Np] sampled at flat node indices idx[K][4 Nfp] -> [V][K][4 Nfp]."""
    V = u.shape[0]
    return u.reshape(V, -1)[:, idx]


def ref_derivatives(ref, u):
    """(Dr u, Ds u, Dt u) along the node axis of u[V][K][Np]."""
    return [np.einsum("ij,vkj->vki", D, u) for D in (ref.Dr, ref.Ds, ref.Dt)]


def divergence(ref, geo, F):
    """sum_d dF_d/dx_d for F[3][V][K][Np], element-wise constant metric terms."""
    drdx = geo.drdx()  # [a][d][K]
    out = np.zeros(F.shape[1:])
    for d in range(3):
        dF = ref_derivatives(ref, F[d])
        for a in range(3):
            out += drdx[a, d][None, :, None] * dF[a]
    return out


def lift(ref, geo, g):
    """LIFT (Fscale * g) for g[V][K][4 Nfp]."""
    return np.einsum("ij,vkj->vki", ref.LIFT, face_fscale(geo, ref.Nfp)[None] * g)


def rhs_strong(ref, geo, conn, q, gas, T=None):
    """Strong-form Euler right-hand side [V][K][Np].

    ``gas`` supplies pressure_sound_speed(q, T); T (temperature at every node)
    is needed for a mixture and ignored by a perfect gas.
    """
    p, c = gas.pressure_sound_speed(q, T)
    F = euler_flux(q, p)
    div = divergence(ref, geo, F)
    qM, qP = gather(q, conn.vmapM), gather(q, conn.vmapP)
    pM, pP = gather(p[None], conn.vmapM)[0], gather(p[None], conn.vmapP)[0]
    cM, cP = gather(c[None], conn.vmapM)[0], gather(c[None], conn.vmapP)[0]
    n = face_normals(geo, ref.Nfp)
    fstar = lax_friedrichs(qM, qP, pM, pP, cM, cP, n)
    return -div + lift(ref, geo, normal_flux(euler_flux(qM, pM), n) - fstar)


def rhs_weak(ref, geo, conn, q, gas, T=None):
    """Weak-form Euler right-hand side [V][K][Np] (cross-check of rhs_strong)."""
    p, c = gas.pressure_sound_speed(q, T)
    F = euler_flux(q, p)
    drdx = geo.drdx()
    Minv = ref.Minv
    out = np.zeros(q.shape)
    for a, D in enumerate((ref.Dr, ref.Ds, ref.Dt)):
        W = Minv @ D.T @ ref.M
        Fa = sum(drdx[a, d][None, :, None] * F[d] for d in range(3))
        out += np.einsum("ij,vkj->vki", W, Fa)
    qM, qP = gather(q, conn.vmapM), gather(q, conn.vmapP)
    pM, pP = gather(p[None], conn.vmapM)[0], gather(p[None], conn.vmapP)[0]
    cM, cP = gather(c[None], conn.vmapM)[0], gather(c[None], conn.vmapP)[0]
    n = face_normals(geo, ref.Nfp)
    fstar = lax_friedrichs(qM, qP, pM, pP, cM, cP, n)
    return out - lift(ref, geo, fstar)
