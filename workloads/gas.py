"""Gas-model parameters: a perfect gas, and a seeded NASA-7 mixture.

The paper's flows are a perfect gas with gamma = 1.4 (§5.3) and reacting
multi-species mixtures (§4, §5).  The paper prints no species data, so the
mixture here is synthetic: per species a molar mass and NASA 7-coefficient
polynomials, drawn from a seed so that cp_k(T)/R_k is smooth, increasing and
well above 1 on [300, 3000] K (then e(T) is strictly increasing and the
temperature inversion has a unique root).

NASA-7 convention (coefficients a1..a7 per species, R_k = R_u / W_k):
    cp_k/R_k = a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4
    h_k/(R_k T) = a1 + a2 T/2 + a3 T^2/3 + a4 T^3/4 + a5 T^4/5 + a6/T
This module only draws the coefficients; it evaluates none of these.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

R_UNIVERSAL = 8314.462618  # J / (kmol K)


@dataclass(frozen=True)
class IdealGas:
    """Single-species perfect gas (nondimensional by default: R = 1)."""

    gamma: float = 1.4
    R: float = 1.0
    mu: float = 0.0  # dynamic viscosity; 0 = inviscid (Euler)
    Pr: float = 0.71


@dataclass(frozen=True)
class Nasa7Mixture:
    """ns species with molar masses W [kg/kmol] and NASA-7 coefficients [ns][7]."""

    W: np.ndarray
    coeffs: np.ndarray
    T_min: float = 300.0
    T_max: float = 3000.0
    R_universal: float = R_UNIVERSAL
    mu: float = 0.0
    Pr: float = 0.71
    extra: dict = field(default_factory=dict)

    @property
    def nspecies(self) -> int:
        return int(self.W.shape[0])


def seeded_nasa7_mixture(nspecies=7, seed=0, T_min=300.0, T_max=3000.0) -> Nasa7Mixture:
    """Draw a synthetic mixture.

    Per species: W ~ U(2, 44) kg/kmol; cp/R follows a saturating rise from
    c_lo ~ U(2.5, 4) at T_min to c_lo + U(0.5, 3) at T_max with a random time
    constant, and a1..a5 interpolate it at 5 Chebyshev points of [T_min,
    T_max]; the draw is repeated until cp/R > 2 on a fine grid.  a6 puts
    h(298.15 K)/R_k at U(-3e4, 3e4) K; a7 ~ U(0, 30) (unused).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    W = rng.uniform(2.0, 44.0, size=nspecies)
    coeffs = np.zeros((nspecies, 7))
    cheb = 0.5 * (T_min + T_max) + 0.5 * (T_max - T_min) * np.cos(np.pi * (2 * np.arange(5) + 1) / 10)
    fine = np.linspace(T_min, T_max, 2001)
    for k in range(nspecies):
        while True:
            c_lo = rng.uniform(2.5, 4.0)
            c_hi = c_lo + rng.uniform(0.5, 3.0)
            tau = rng.uniform(500.0, 1500.0)
            shape = lambda T: (1 - np.exp(-(T - T_min) / tau)) / (1 - np.exp(-(T_max - T_min) / tau))
            target = c_lo + (c_hi - c_lo) * shape(cheb)
            A = np.vander(cheb, 5, increasing=True)
            a = np.linalg.solve(A, target)
            cp_fine = np.vander(fine, 5, increasing=True) @ a
            if np.all(cp_fine > 2.0):
                break
        h298 = rng.uniform(-3.0e4, 3.0e4)
        T0 = 298.15
        poly_int = a[0] * T0 + a[1] * T0 ** 2 / 2 + a[2] * T0 ** 3 / 3 + a[3] * T0 ** 4 / 4 + a[4] * T0 ** 5 / 5
        coeffs[k, :5] = a
        coeffs[k, 5] = h298 - poly_int
        coeffs[k, 6] = rng.uniform(0.0, 30.0)
    return Nasa7Mixture(W=W, coeffs=coeffs, T_min=T_min, T_max=T_max)


def mixture_primitive_state(xyz, nspecies=7, seed=0, p0=1.0e5, T_mean=1650.0, T_amp=1350.0, vel_amp=10.0,
                            L=1.0):
    """Primitive fields of the multi-species workload, sampled at the nodes.

    T = T_mean + T_amp sin(kx) sin(ky) sin(kz) (k = 2 pi / L, so T spans
    [300, 3000] K with the defaults); mass fractions Y ~ Dirichlet(1,...,1)
    per node (PCG64, ``seed``); velocity (vel_amp sin(ky), vel_amp sin(kz),
    vel_amp sin(kx)) m/s; uniform pressure p0.  The density follows from
    p0 and T through the mixture gas constant, which the consumer computes;
    this returns (Y[ns][...], T[...], vel[3][...], p0).
    """
    k = 2.0 * np.pi / L
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    T = T_mean + T_amp * np.sin(k * x) * np.sin(k * y) * np.sin(k * z)
    rng = np.random.Generator(np.random.PCG64(seed))
    Y = rng.dirichlet(np.ones(nspecies), size=T.shape)  # [..., ns]
    Y = np.moveaxis(Y, -1, 0)
    vel = np.stack([vel_amp * np.sin(k * y), vel_amp * np.sin(k * z), vel_amp * np.sin(k * x)])
    return Y, T, vel, p0
