"""Pins of the oracle's gas models, temperature inversion and LSRK4 scheme."""

from fractions import Fraction

import numpy as np
import pytest

from oracle.lsrk import NSTAGES, RK4A_EXACT, RK4B_EXACT, butcher_tableau, lsrk4_step, rk4_classic_step
from oracle.thermo import Nasa7Gas, PerfectGas
from workloads.gas import seeded_nasa7_mixture


def _gas():
    mix = seeded_nasa7_mixture(7, seed=0)
    return Nasa7Gas(W=mix.W, coeffs=mix.coeffs)


def test_stability_polynomial_is_fourth_order():
    """For y' = z y the step multiplies y by R(z); a 4th-order method has R = 1 + z + z^2/2 + z^3/6 + z^4/24 + O(z^5)."""
    # exact rational arithmetic on the published coefficients, as polynomial coefficient lists
    y = [Fraction(1)]
    k = [Fraction(0)]

    def add(a, b):
        n = max(len(a), len(b))
        return [(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)]

    for s in range(NSTAGES):
        k = add([RK4A_EXACT[s] * c for c in k], [Fraction(0)] + y)  # a k + z y
        y = add(y, [RK4B_EXACT[s] * c for c in k])
    target = [1, 1, Fraction(1, 2), Fraction(1, 6), Fraction(1, 24)]
    for i, t in enumerate(target):
        assert abs(float(y[i] - t)) < 1e-14
    assert len(y) == 6  # five stages: degree-5 polynomial


def test_all_fourth_order_conditions():
    """The eight order conditions of a 4th-order Runge-Kutta method, in Butcher form (c = row sums of A)."""
    A, b = butcher_tableau()
    c = [sum(row) for row in A]
    n = NSTAGES
    Ac = [sum(A[i][j] * c[j] for j in range(n)) for i in range(n)]
    Ac2 = [sum(A[i][j] * c[j] ** 2 for j in range(n)) for i in range(n)]
    AAc = [sum(A[i][j] * Ac[j] for j in range(n)) for i in range(n)]
    conds = [
        (sum(b), 1), (sum(b[i] * c[i] for i in range(n)), Fraction(1, 2)),
        (sum(b[i] * c[i] ** 2 for i in range(n)), Fraction(1, 3)), (sum(b[i] * Ac[i] for i in range(n)), Fraction(1, 6)),
        (sum(b[i] * c[i] ** 3 for i in range(n)), Fraction(1, 4)),
        (sum(b[i] * c[i] * Ac[i] for i in range(n)), Fraction(1, 8)),
        (sum(b[i] * Ac2[i] for i in range(n)), Fraction(1, 12)), (sum(b[i] * AAc[i] for i in range(n)), Fraction(1, 24)),
    ]
    for got, want in conds:
        assert abs(float(got - want)) < 1e-14
    assert c[0] == 0 and all(0 < float(ci) < 1 for ci in c[1:])


@pytest.mark.parametrize("stepper", [lsrk4_step, rk4_classic_step])
def test_ode_order_four(stepper):
    f = lambda y: np.array([y[1], -y[0]])  # harmonic oscillator, exact solution (cos t, -sin t)
    errs = []
    for n in (20, 40, 80):
        y = np.array([1.0, 0.0])
        dt = 2.0 / n
        for _ in range(n):
            y = stepper(y, dt, f)
        errs.append(np.abs(y - [np.cos(2.0), -np.sin(2.0)]).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.8), rates


def test_perfect_gas_closed_forms():
    g = PerfectGas(1.4, 287.0)
    rho, u, p = 1.2, np.array([10.0, -3.0, 2.0]), 1.0e5
    q = np.array([rho, *(rho * u), p / 0.4 + 0.5 * rho * u @ u])
    pp, c = g.pressure_sound_speed(q)
    assert abs(pp - p) < 1e-9 * p
    assert abs(c - np.sqrt(1.4 * p / rho)) < 1e-12 * c
    assert abs(g.temperature(q) - p / (rho * 287.0)) < 1e-9


def test_cp_is_derivative_of_enthalpy():
    g = _gas()
    T = np.linspace(300, 3000, 50)
    h = 1e-3
    dh = (g.h_species(T + h) - g.h_species(T - h)) / (2 * h)
    assert np.abs(dh - g.cp_species(T)).max() < 1e-6 * np.abs(g.cp_species(T)).max()
    # e = h - R T  =>  de/dT = cp - R = cv
    Y = np.full((7, T.size), 1 / 7)
    de = (g.mixture_e(T + h, Y) - g.mixture_e(T - h, Y)) / (2 * h)
    assert np.abs(de - g.mixture_cv(T, Y)).max() < 1e-6 * g.mixture_cv(T, Y).max()


def test_seeded_mixture_is_physical():
    g = _gas()
    T = np.linspace(300, 3000, 2001)
    cpR = g.cp_species(T) / g.Rk[:, None]
    assert cpR.min() > 2.0
    Y = np.random.default_rng(0).dirichlet(np.ones(7), size=T.size).T
    assert np.all(np.diff(g.mixture_e(T, Y[:, :1] * np.ones((1, T.size)))) > 0)


def test_newton_against_bisection_and_generating_temperature():
    g = _gas()
    rng = np.random.default_rng(1)
    n = 10000
    T_true = rng.uniform(300, 3000, n)
    Y = rng.dirichlet(np.ones(7), size=n).T
    e = g.mixture_e(T_true, Y)
    T, it, ok = g.newton_temperature(e, Y, np.full(n, 1500.0))
    assert ok.all()
    assert it.max() <= 50
    Tb = g.bisect_temperature(e, Y)
    assert np.abs(T - Tb).max() < 1e-9
    assert np.abs(T - T_true).max() < 1e-9


def test_constant_cp_reduces_to_closed_form():
    """a2..a5 = 0: e_k is linear in T, so T = (e - sum Y R a6) / cv exactly and Newton needs one update plus a check."""
    W = np.array([28.0, 2.0, 32.0])
    coeffs = np.zeros((3, 7))
    coeffs[:, 0] = [3.5, 3.4, 3.6]
    coeffs[:, 5] = [-1000.0, 200.0, 0.0]
    g = Nasa7Gas(W=W, coeffs=coeffs)
    Y = np.array([[0.7], [0.1], [0.2]])
    Rk = g.Rk[:, None]
    cv = np.sum(Y * Rk * (coeffs[:, :1] - 1))
    for T0 in (300.0, 1234.5, 2999.0):
        e = cv * T0 + np.sum(Y[:, 0] * g.Rk * coeffs[:, 5])
        T, it, ok = g.newton_temperature(np.array([e]), Y, np.array([2000.0]))
        assert ok.all() and it[0] == 2
        assert abs(T[0] - T0) < 1e-10


def test_newton_reports_failure_when_capped():
    g = _gas()
    Y = np.full((7, 4), 1 / 7)
    e = g.mixture_e(np.full(4, 2500.0), Y)
    T, it, ok = g.newton_temperature(e, Y, np.full(4, 300.0), max_it=1)
    assert not ok.any() and np.all(it == 1)
