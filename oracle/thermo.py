"""Gas models: perfect gas and NASA-7 mixture; temperature from internal energy.

The paper's flows use a perfect gas with gamma = 1.4 (§5.3) and the solver
targets multi-species reacting mixtures (§4 "compressible multispecies flow",
§5 "reactive mixture viscous flows").  It gives no thermodynamic formulas;
these are the standard definitions:

Perfect gas:  p = (gamma-1)(rho E - rho |u|^2 / 2),  T = p / (rho R),
              c = sqrt(gamma p / rho),  cp = gamma R / (gamma-1).

NASA-7 mixture (species k, R_k = R_u / W_k, mass fractions Y_k):
    cp_k = R_k (a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4)
    h_k  = R_k (a1 T + a2 T^2/2 + a3 T^3/3 + a4 T^4/4 + a5 T^5/5 + a6)
    e_k  = h_k - R_k T,   e(T) = sum_k Y_k e_k(T),   cv = sum_k Y_k (cp_k - R_k)
    p = rho R_mix T with R_mix = sum_k Y_k R_k,  c^2 = (cp_mix / cv_mix) p / rho.
Temperature: the root of e(T) = e with e = rho E / rho - |u|^2 / 2, by Newton
T <- T - (e(T) - e) / cv(T), stopping at the first update with |dT| < tol
(1e-10 K) and failing after max_it updates.  A bisection solve is kept as an
independent check.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class PerfectGas:
    gamma: float = 1.4
    R: float = 1.0

    @property
    def cp(self):
        return self.gamma * self.R / (self.gamma - 1.0)

    def pressure(self, q):
        rho = q[0]
        ke = 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2) / rho
        return (self.gamma - 1.0) * (q[4] - ke)

    def temperature(self, q):
        return self.pressure(q) / (q[0] * self.R)

    def pressure_sound_speed(self, q, T=None):
        p = self.pressure(q)
        return p, np.sqrt(self.gamma * p / q[0])


@dataclass
class Nasa7Gas:
    W: np.ndarray  # [ns] kg/kmol
    coeffs: np.ndarray  # [ns][7]
    R_universal: float = 8314.462618
    newton_tol: float = 1e-10
    newton_max_it: int = 50

    @property
    def Rk(self):
        return self.R_universal / np.asarray(self.W, dtype=np.float64)

    @property
    def nspecies(self):
        return int(np.asarray(self.W).shape[0])

    def _expand(self, T):
        a = self.coeffs
        shape = (self.nspecies,) + (1,) * np.ndim(T)
        return [a[:, i].reshape(shape) for i in range(7)], self.Rk.reshape(shape)

    def cp_species(self, T):
        (a1, a2, a3, a4, a5, a6, a7), Rk = self._expand(T)
        return Rk * (a1 + a2 * T + a3 * T ** 2 + a4 * T ** 3 + a5 * T ** 4)

    def h_species(self, T):
        (a1, a2, a3, a4, a5, a6, a7), Rk = self._expand(T)
        return Rk * (a1 * T + a2 * T ** 2 / 2 + a3 * T ** 3 / 3 + a4 * T ** 4 / 4 + a5 * T ** 5 / 5 + a6)

    def e_species(self, T):
        _, Rk = self._expand(T)
        return self.h_species(T) - Rk * T

    def mixture_e(self, T, Y):
        return np.sum(Y * self.e_species(T), axis=0)

    def mixture_cv(self, T, Y):
        _, Rk = self._expand(T)
        return np.sum(Y * (self.cp_species(T) - Rk), axis=0)

    def mixture_cp(self, T, Y):
        return np.sum(Y * self.cp_species(T), axis=0)

    def R_mix(self, Y):
        shape = (self.nspecies,) + (1,) * (np.ndim(Y) - 1)
        return np.sum(Y * self.Rk.reshape(shape), axis=0)

    # -- state <-> primitives ------------------------------------------------
    def split_state(self, q):
        """(rho, velocity[3], Y[ns], e) from q = [rho, rho u(3), rho E, rho Y_k (ns)]."""
        rho = q[0]
        vel = q[1:4] / rho
        Y = q[5:] / rho
        e = q[4] / rho - 0.5 * np.sum(vel ** 2, axis=0)
        return rho, vel, Y, e

    def conserved(self, rho, vel, Y, T):
        e = self.mixture_e(T, Y)
        E = rho * (e + 0.5 * np.sum(vel ** 2, axis=0))
        return np.concatenate([rho[None], rho[None] * vel, E[None], rho[None] * Y]).astype(np.float64)

    def pressure_sound_speed(self, q, T):
        rho, vel, Y, e = self.split_state(q)
        p = rho * self.R_mix(Y) * T
        gam = self.mixture_cp(T, Y) / self.mixture_cv(T, Y)
        return p, np.sqrt(gam * p / rho)

    # -- temperature inversion -----------------------------------------------
    def newton_temperature(self, e, Y, T0, tol=None, max_it=None):
        """Per-node Newton; returns (T, iterations, converged)."""
        tol = self.newton_tol if tol is None else tol
        max_it = self.newton_max_it if max_it is None else max_it
        shape = np.shape(e)
        e = np.asarray(e, dtype=np.float64).reshape(-1)
        Y = np.asarray(Y, dtype=np.float64).reshape(self.nspecies, -1)
        T = np.array(T0, dtype=np.float64, copy=True).reshape(-1)
        iters = np.zeros(T.shape, dtype=np.int64)
        active = np.ones(T.shape, dtype=bool)
        for _ in range(max_it):
            if not active.any():
                break
            Ta = T[active]
            Ya = Y[:, active]
            dT = (self.mixture_e(Ta, Ya) - e[active]) / self.mixture_cv(Ta, Ya)
            T[active] = Ta - dT
            iters[active] += 1
            done = np.abs(dT) < tol
            idx = np.flatnonzero(active)
            active[idx[done]] = False
        return T.reshape(shape), iters.reshape(shape), ~active.reshape(shape)

    def bisect_temperature(self, e, Y, lo=300.0, hi=3000.0, tol=1e-12):
        """Bisection on [lo, hi] (e(T) is increasing there); independent check of Newton."""
        a = np.full(np.shape(e), lo, dtype=np.float64)
        b = np.full(np.shape(e), hi, dtype=np.float64)
        for _ in range(200):  # halving 2700 K reaches the spacing of doubles long before 200 steps
            if np.max(b - a) <= tol:
                break
            m = 0.5 * (a + b)
            above = self.mixture_e(m, Y) > e
            b = np.where(above, m, b)
            a = np.where(above, a, m)
        return 0.5 * (a + b)
