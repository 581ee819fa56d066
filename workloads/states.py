"""Closed-form initial states sampled at the nodes, plus seeded noise.

Conserved-variable layout (the paper's element-local nodal layout, §1 Fig. 1):
float64 q[V][K][Np] with V = 5 for a single species:
    q[0] = rho, q[1:4] = rho*u, q[4] = rho*E  (total energy per volume).

For a perfect gas rho*E = p/(gamma-1) + rho*|u|^2/2; that relation only
defines the initial state here.  Mixture states are returned as primitive
fields (see workloads.gas) and converted by each consumer with its own
equation of state.
"""

from __future__ import annotations

import numpy as np


def _conserved_perfect_gas(rho, u, v, w, p, gamma):
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    q = np.stack([rho, rho * u, rho * v, rho * w, E])
    # complex inputs (complex-step derivatives in tests) keep their dtype
    return q if np.iscomplexobj(q) else q.astype(np.float64)


def _min_image(d, L):
    if L <= 0:
        return d
    return d - L * np.round(np.real(d) / L)


def isentropic_vortex(xyz, t=0.0, *, gamma=1.4, beta=5.0, center=(0.5, 0.5), radius=0.1,
                      u_inf=(1.0, 0.0), period=None, rho_inf=1.0, p_inf=1.0):
    """Translating 2-D isentropic vortex (Shu's form), extruded along z.

    The paper's inviscid case (§5.2) is this vortex.  With the length scale R
    (``radius``), at time t and minimum-image offsets
    (dx, dy) = (x - xc - u_inf t, y - yc - v_inf t), rho2 = (dx^2+dy^2)/R^2:
        T   = 1 - (gamma-1) beta^2 exp(1 - rho2) / (8 gamma pi^2)
        rho = rho_inf T^(1/(gamma-1)),   p = p_inf T^(gamma/(gamma-1))
        u   = u_inf - beta/(2 pi) exp((1 - rho2)/2) dy/R
        v   = v_inf + beta/(2 pi) exp((1 - rho2)/2) dx/R,   w = 0.
    With rho_inf = p_inf = 1 this is an exact solution of the Euler equations
    in free space; in a periodic box it is exact up to the tail of the Gaussian
    at the seam (keep L/R large).  xyz: [..., 3].  Returns q[5][...].
    """
    x, y = xyz[..., 0], xyz[..., 1]
    Lx = Ly = 0.0
    if period is not None:
        Lx, Ly = float(period[0]), float(period[1])
    dx = _min_image(x - center[0] - u_inf[0] * t, Lx)
    dy = _min_image(y - center[1] - u_inf[1] * t, Ly)
    r2 = (dx * dx + dy * dy) / (radius * radius)
    ef = np.exp(0.5 * (1.0 - r2))
    T = 1.0 - (gamma - 1.0) * beta * beta * ef * ef / (8.0 * gamma * np.pi * np.pi)
    rho = rho_inf * T ** (1.0 / (gamma - 1.0))
    p = p_inf * T ** (gamma / (gamma - 1.0))
    u = u_inf[0] - beta / (2.0 * np.pi) * ef * dy / radius
    v = u_inf[1] + beta / (2.0 * np.pi) * ef * dx / radius
    w = np.zeros_like(u)
    return _conserved_perfect_gas(rho, u, v, w, p, gamma)


def taylor_green(xyz, *, gamma=1.4, mach=0.1, rho0=1.0, c0=1.0, L=1.0, noise=0.0, seed=0):
    """Taylor-Green vortex in a periodic box of side L (wavenumber k = 2 pi / L).

    u = V0 sin(kx) cos(ky) cos(kz), v = -V0 cos(kx) sin(ky) cos(kz), w = 0,
    p = p0 + rho0 V0^2/16 (cos 2kx + cos 2ky)(cos 2kz + 2), rho = rho0,
    with V0 = mach*c0 and p0 = rho0 c0^2 / gamma.  ``noise`` multiplies each
    velocity component by (1 + noise*U(-1,1)), drawn per node from
    numpy's PCG64 with ``seed``.  Returns q[5][...].
    """
    k = 2.0 * np.pi / L
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    V0 = mach * c0
    p0 = rho0 * c0 * c0 / gamma
    u = V0 * np.sin(k * x) * np.cos(k * y) * np.cos(k * z)
    v = -V0 * np.cos(k * x) * np.sin(k * y) * np.cos(k * z)
    w = np.zeros_like(u)
    if noise:
        rng = np.random.Generator(np.random.PCG64(seed))
        u = u * (1.0 + noise * rng.uniform(-1.0, 1.0, size=u.shape))
        v = v * (1.0 + noise * rng.uniform(-1.0, 1.0, size=v.shape))
        w = w * (1.0 + noise * rng.uniform(-1.0, 1.0, size=w.shape))
    p = p0 + rho0 * V0 * V0 / 16.0 * (np.cos(2 * k * x) + np.cos(2 * k * y)) * (np.cos(2 * k * z) + 2.0)
    rho = np.full_like(u, rho0)
    return _conserved_perfect_gas(rho, u, v, w, p, gamma)


def freestream(shape, *, gamma=1.4, rho=1.0, vel=(0.3, -0.2, 0.1), p=1.0):
    """Uniform state of the given node-array shape.  Returns q[5][*shape]."""
    ones = np.ones(shape)
    return _conserved_perfect_gas(rho * ones, vel[0] * ones, vel[1] * ones, vel[2] * ones, p * ones, gamma)


def sin_shear(xyz, *, gamma=1.4, amp=0.1, L=1.0, rho=1.0, p=1.0):
    """Shear layer u = amp sin(2 pi y / L), v = w = 0, uniform rho and p.  Returns q[5][...]."""
    y = xyz[..., 1]
    u = amp * np.sin(2.0 * np.pi * y / L)
    z = np.zeros_like(u)
    return _conserved_perfect_gas(rho + z, u, z, z, p + z, gamma)


def channel_flow(xyz, *, gamma=1.4, mach=0.3, noise=0.01, seed=0, height=1.0):
    """Parabolic channel profile between walls at y = 0 and y = height: rho = 1, p = 1/gamma
    (c = 1), u = 4 M y (h - y) / h^2, times (1 + noise U(-1, 1)) per node; v = w = noise M U(-1, 1)
    / 10 (PCG64, ``seed``).  Conserved variables [5][...]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    y = xyz[..., 1]
    shape = y.shape
    u = 4.0 * mach * y * (height - y) / height ** 2 * (1.0 + noise * rng.uniform(-1, 1, shape))
    v = 0.1 * noise * mach * rng.uniform(-1, 1, shape)
    w = 0.1 * noise * mach * rng.uniform(-1, 1, shape)
    return _conserved_perfect_gas(np.ones(shape), u, v, w, np.full(shape, 1.0 / gamma), gamma)


def sod_fronts(xyz, *, gamma=1.4, width=0.01, L=1.0):
    """Two smoothed Sod shock-tube states on a periodic box: (rho, p) = (1, 1) for x in
    [L/4, 3L/4] and (0.125, 0.1) outside, joined by tanh profiles of the given width; at rest."""
    x = xyz[..., 0]
    S = 0.5 * (np.tanh((x - 0.25 * L) / width) - np.tanh((x - 0.75 * L) / width))
    rho = 0.125 + 0.875 * S
    p = 0.1 + 0.9 * S
    zero = np.zeros_like(x)
    return _conserved_perfect_gas(rho, zero, zero, zero, p, gamma)


def advected_wave(xyz, t=0.0, *, velocity=(1.0, 0.5, 0.25), L=1.0):
    """Smooth periodic scalar on the box [0, L]^3 translated by velocity t: the exact solution of
    du/dt + a . grad u = 0 for u(x, 0) = sin(2 pi x/L) cos(2 pi y/L) + 0.3 sin(2 pi z/L)."""
    k = 2.0 * np.pi / L
    x, y, z = (xyz[..., d] - velocity[d] * t for d in range(3))
    return np.sin(k * x) * np.cos(k * y) + 0.3 * np.sin(k * z)


def uniform_perturbation(q, amplitude, seed=0):
    """q + U(-amplitude, amplitude), drawn per conserved variable per node (PCG64, ``seed``)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return q + rng.uniform(-amplitude, amplitude, size=q.shape)
