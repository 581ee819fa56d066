"""Pins of the artificial-viscosity oracle (oracle/av.py): the smoothness indicator against a
closed form and against the textbook orthonormal (Dubiner / Koornwinder) modes, the viscosity
ramp, and the BR1 artificial-viscosity operator against what the mathematics fixes (zero on
constants, conservation, the discrete energy identity of BR1, consistency with eps Laplacian);
planted mistakes must break a pin."""

import numpy as np
import pytest
from scipy.special import eval_jacobi, gamma as Gamma

import oracle.av as av
from oracle.euler import ref_derivatives
from tests._oracle_case import box_disc, reference

S0, KAPPA, EPS0 = -4.0 * np.log10(3.0), 0.5, 1e-2


def _jacobi_normed(x, al, be, n):
    h = 2.0 ** (al + be + 1) / (2 * n + al + be + 1) * Gamma(n + al + 1) * Gamma(n + be + 1) / (
        Gamma(n + al + be + 1) * Gamma(n + 1))
    return eval_jacobi(n, al, be, x) / np.sqrt(h)


def _dubiner(i, j, k, rst):
    """The orthonormal mode psi_ijk of degree i + j + k on the reference tetrahedron."""
    r, s, t = rst[:, 0], rst[:, 1], rst[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.where(np.abs(s + t) > 1e-13, -2 * (1 + r) / (s + t) - 1, -1.0)
        b = np.where(np.abs(1 - t) > 1e-13, 2 * (1 + s) / (1 - t) - 1, -1.0)
    c = t
    return (2 * np.sqrt(2.0) * _jacobi_normed(a, 0, 0, i) * _jacobi_normed(b, 2 * i + 1, 0, j) * (1 - b) ** i
            * _jacobi_normed(c, 2 * i + 2 * j + 2, 0, k) * (1 - c) ** (i + j))


def _modes(N):
    return [(i, j, k) for i in range(N + 1) for j in range(N + 1 - i) for k in range(N + 1 - i - j)]


# --- indicator ------------------------------------------------------------------------------------

def test_indicator_closed_form_n1():
    """N = 1, u = the barycentric coordinate of vertex 0: mean 1/4, ||u||^2 = |T|/10,
    ||u - 1/4||^2 = 3|T|/80, so S = 3/8."""
    ref = reference(1)
    u = np.array([[1.0, 0.0, 0.0, 0.0]])
    assert abs(av.smoothness_indicator(ref, u)[0] - 3.0 / 8.0) <= 1e-14


@pytest.mark.parametrize("N", [2, 3, 4])
def test_indicator_vanishes_below_degree_n(N):
    ref = reference(N)
    rng = np.random.default_rng(N)
    r, s, t = ref.nodes.T
    u = sum(rng.uniform(-1, 1) * r ** a * s ** b * t ** c for (a, b, c) in _modes(N - 1))
    assert av.smoothness_indicator(ref, (u + 2.0)[None])[0] <= 1e-26


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_indicator_is_the_top_mode_energy(N):
    """u = sum of orthonormal modes: S = (sum of the squared degree-N coefficients) / (sum of all)."""
    ref = reference(N)
    modes = _modes(N)
    Psi = np.stack([_dubiner(i, j, k, ref.nodes) for (i, j, k) in modes], axis=1)
    assert np.abs(Psi.T @ ref.M @ Psi - np.eye(len(modes))).max() <= 1e-12  # orthonormal
    rng = np.random.default_rng(10 + N)
    coef = rng.uniform(-1, 1, (3, len(modes)))
    top = np.array([sum(m) == N for m in modes])
    want = (coef[:, top] ** 2).sum(1) / (coef ** 2).sum(1)
    got = av.smoothness_indicator(ref, coef @ Psi.T)
    assert np.abs(got - want).max() <= 1e-12


def test_viscosity_ramp():
    s = np.array([S0 - KAPPA - 1e-9, S0 - KAPPA, S0, S0 + KAPPA, S0 + KAPPA + 1.0])
    e = av.viscosity(10.0 ** s, EPS0, S0, KAPPA)
    assert e[0] == 0.0 and abs(e[1]) <= 1e-15 and abs(e[2] - EPS0 / 2) <= 1e-15
    assert abs(e[3] - EPS0) <= 1e-15 and e[4] == EPS0
    ss = np.linspace(S0 - KAPPA, S0 + KAPPA, 101)
    assert np.all(np.diff(av.viscosity(10.0 ** ss, EPS0, S0, KAPPA)) >= 0)
    assert av.viscosity(np.array([0.0]), EPS0, S0, KAPPA)[0] == 0.0


# --- the artificial-viscosity operator ----------------------------------------------------------

def _state(d, seed=0):
    x, y, z = d.xyz[..., 0], d.xyz[..., 1], d.xyz[..., 2]
    k = 2 * np.pi
    q = np.stack([1 + 0.2 * np.sin(k * x) * np.cos(k * z), 0.3 * np.cos(k * y), 0.1 * np.sin(k * (x + z)),
                  0.05 * np.cos(k * x), 2.5 + 0.3 * np.sin(k * y)])
    return q + 1e-2 * np.random.default_rng(seed).uniform(-1, 1, q.shape)


def _eps(d, seed=1):
    return np.random.default_rng(seed).uniform(0.0, 1e-2, d.K)


def _constant_is_steady(N=2):
    d = box_disc(2, N)
    q = np.ones((5,) + d.xyz.shape[:-1]) * np.array([1.0, 0.2, -0.1, 0.3, 2.0])[:, None, None]
    return np.abs(av.rhs_av(d.ref, d.geo, d.conn, q, _eps(d))).max() <= 1e-13


def _conserves(N=2):
    d = box_disc(2, N)
    r = av.rhs_av(d.ref, d.geo, d.conn, _state(d), _eps(d))
    return all(abs(d.integrate(r[v])) <= 1e-12 * d.abs_integral(r[v]) for v in range(5))


def _energy_identity(N=2):
    """(q, div_h(eps grad_h q))_M = -sum_e eps_e ||grad_h q||^2_{M,e}: the BR1 divergence with
    central fluxes is the negative adjoint of the BR1 gradient on a periodic mesh."""
    d = box_disc(2, N)
    q, eps = _state(d), _eps(d)
    r = av.rhs_av(d.ref, d.geo, d.conn, q, eps)
    g = av.br1_gradient(d.ref, d.geo, d.conn, q)
    lhs = sum(np.einsum("kn,nm,km,k->", q[v], d.ref.M, r[v], d.geo.J) for v in range(5))
    rhs = -sum(np.einsum("kn,nm,km,k->", g[dd, v], d.ref.M, g[dd, v], d.geo.J * eps)
               for dd in range(3) for v in range(5))
    return abs(lhs - rhs) <= 1e-11 * abs(rhs) and rhs < 0


def _consistent(N=3):
    """Constant eps: div_h(eps grad_h q) -> eps Laplacian(q) for q = sin 2 pi x cos 2 pi y.  The
    BR1 Laplacian's pointwise error converges at about order N - 1 (measured 0.56 -> 0.18, rate
    1.67, at N = 3 from 3 to 6 cells per side)."""
    errs = []
    for n in (3, 6):
        d = box_disc(n, N)
        x, y = d.xyz[..., 0], d.xyz[..., 1]
        k = 2 * np.pi
        q = np.stack([np.sin(k * x) * np.cos(k * y)] * 5)
        r = av.rhs_av(d.ref, d.geo, d.conn, q, np.full(d.K, 0.1))
        exact = -0.1 * 2 * k * k * q
        errs.append(d.l2(r[0] - exact[0]) / d.l2(exact[0]))
    return np.log2(errs[0] / errs[1]) >= 1.5 and errs[1] < 0.2


def _av_pins_hold():
    return _constant_is_steady() and _conserves() and _energy_identity() and _consistent()


def test_av_operator_pins():
    assert _constant_is_steady()
    assert _conserves()
    assert _energy_identity()
    assert _consistent()


@pytest.mark.parametrize("N", [1, 3, 4])
def test_av_energy_identity_other_orders(N):
    assert _energy_identity(N)


def test_zero_viscosity_adds_nothing():
    d = box_disc(2, 2)
    assert np.abs(av.rhs_av(d.ref, d.geo, d.conn, _state(d), np.zeros(d.K))).max() == 0.0


# --- planted mistakes ----------------------------------------------------------------------------

def test_planted_full_jump_in_the_gradient_fails(monkeypatch):
    orig = av.br1_gradient

    def bad(ref, geo, conn, q, q_in=None):  # jump (q+ - q-) instead of (q+ - q-)/2
        g = orig(ref, geo, conn, q, q_in)
        return 2 * g - np.stack([sum(geo.drdx()[a, dd][None, :, None] * ref_derivatives(ref, q)[a]
                                     for a in range(3)) for dd in range(3)])
    monkeypatch.setattr(av, "br1_gradient", bad)
    assert not _av_pins_hold()


def test_planted_sign_fails(monkeypatch):
    orig = av.rhs_av
    monkeypatch.setattr(av, "rhs_av", lambda *a, **k: -orig(*a, **k))
    assert not _av_pins_hold()


def test_planted_projection_to_degree_n_fails(monkeypatch):
    """Projecting onto degree <= N instead of N - 1 leaves nothing: S = 0 everywhere."""
    orig = av.smoothness_indicator

    def bad(ref, u):
        class R:
            pass
        r2 = R()
        r2.N, r2.nodes = ref.N + 1, ref.nodes
        try:
            return orig(r2, u)
        except Exception:
            return np.zeros(np.asarray(u).shape[0])
    monkeypatch.setattr(av, "smoothness_indicator", bad)
    ref = reference(1)
    assert abs(av.smoothness_indicator(ref, np.array([[1.0, 0.0, 0.0, 0.0]]))[0] - 3.0 / 8.0) > 1e-3
