"""Pins of the over-integrated hexahedral right-hand side (oracle/hex.py: hex_rhs_overint):
freestream preservation, conservation, exact integration of polynomial fluxes (Q >= 2N Gauss points
reproduce a 24-point rule for fluxes of degree 3N, while N + 1 points alias them), convergence to
the translating vortex; and of its Navier-Stokes form (hex_rhs_overint_ns): for a gas at rest with a
temperature of x alone its viscous part is the collocated one (adiabatic walls included),
conservation in periodic and no-slip boxes, a steady rest state between walls; with artificial
viscosity (hex_rhs_overint_av), for a state of x alone its AV part is the collocated AV term, and
periodic boxes conserve; planted mistakes must break a pin."""

import numpy as np
import pytest

import oracle.hex as hx
from oracle.lsrk import lsrk4_step
from oracle.thermo import PerfectGas
from workloads import isentropic_vortex
from workloads.hexmesh import gll_nodes, hex_box, hex_nodes

GAS = PerfectGas(1.4, 1.0)


def _q32(N):
    return int(np.ceil(3 * (N + 1) / 2))


def _freestream(N=3):
    box = hex_box((3, 2, 2), 1.0)
    ref = hx.hex_reference(gll_nodes(N))
    xyz = hex_nodes(box, ref.nodes)
    one = np.ones(xyz.shape[:-1])
    q = np.stack([1.2 * one, 0.3 * one, -0.2 * one, 0.1 * one, 2.5 * one])
    return np.abs(hx.hex_rhs_overint(ref, box, q, GAS, _q32(N))).max() <= 1e-11


def _conserves(N=3):
    box = hex_box((3, 2, 2), 1.0)
    ref = hx.hex_reference(gll_nodes(N))
    xyz = hex_nodes(box, ref.nodes)
    q = isentropic_vortex(xyz, 0.0, center=(0.45, 0.55), radius=0.15, period=box["L"])
    r = hx.hex_rhs_overint(ref, box, q, GAS, _q32(N))
    return bool(np.all(np.abs(hx.hex_integrate(ref, box, r)) <= 1e-12 * hx.hex_integrate(ref, box, np.abs(r))))


def _exact_for_polynomial_fluxes(N=3):
    """rho = 1, p = 1, v = w = 0, u a degree-N polynomial in x: the x-fluxes have degree <= 3N, so
    Q = 2N Gauss points integrate grad(phi) . F exactly (degree 4N - 1) and agree with 24 points."""
    box = hex_box((2, 1, 1), 1.0)
    ref = hx.hex_reference(gll_nodes(N))
    xyz = hex_nodes(box, ref.nodes)
    x = xyz[..., 0]
    u = 0.3 + 0.2 * x ** N - 0.1 * x
    one = np.ones_like(x)
    q = np.stack([one, u, 0 * one, 0 * one, 1.0 / 0.4 + 0.5 * u * u])
    q5 = q.reshape(5, -1, N + 1, N + 1, N + 1)
    exact = hx.hex_overint_volume(ref, box, q5, GAS, 24)
    ok = np.abs(hx.hex_overint_volume(ref, box, q5, GAS, 2 * N) - exact).max() <= 1e-12 * np.abs(exact).max()
    aliased = np.abs(hx.hex_overint_volume(ref, box, q5, GAS, N + 1) - exact).max() > 1e-8 * np.abs(exact).max()
    return ok and (aliased or N == 1)


def _vortex_error(n, N, T=0.2):
    L = 10.0
    box = hex_box((n, n, 1), (L, L, L / n))
    ref = hx.hex_reference(gll_nodes(N))
    xyz = hex_nodes(box, ref.nodes)
    kw = dict(center=(5.0, 5.0), radius=1.0, u_inf=(1.0, 0.0), period=box["L"])
    q = isentropic_vortex(xyz, 0.0, **kw)
    f = lambda u: hx.hex_rhs_overint(ref, box, u, GAS, _q32(N))
    dt0 = 0.3 * (L / n) / ((N + 1) ** 2 * 2.5)
    steps = int(np.ceil(T / dt0))
    for _ in range(steps):
        q = lsrk4_step(q, T / steps, f)
    err = q - isentropic_vortex(xyz, T, **kw)
    return np.sqrt(np.abs(hx.hex_integrate(ref, box, err ** 2)).sum())


def _all_pins_hold():
    return _freestream() and _conserves() and _exact_for_polynomial_fluxes()


def test_freestream_and_conservation():
    assert _freestream()
    assert _conserves()


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_exact_integration_of_polynomial_fluxes(N):
    assert _exact_for_polynomial_fluxes(N)


@pytest.mark.parametrize("N", [2, 3])
def test_vortex_convergence(N):
    """Rates 2.19 and 3.52 for N = 2, 3 from 8 to 16 cells; the test asks for N."""
    rate = np.log2(_vortex_error(8, N) / _vortex_error(16, N))
    assert rate >= N, rate


def test_planted_gll_weights_fail(monkeypatch):
    orig = hx._gauss_operators

    def bad(ref, Q):  # Gauss points with uniform weights
        I, A, B = orig(ref, Q)
        xg, wg = np.polynomial.legendre.leggauss(Q)
        return I, A / wg[None, :] * (2.0 / Q), B / wg[None, :] * (2.0 / Q)
    monkeypatch.setattr(hx, "_gauss_operators", bad)
    assert not _all_pins_hold()


def test_planted_swapped_operators_fail(monkeypatch):
    orig = hx._gauss_operators
    monkeypatch.setattr(hx, "_gauss_operators", lambda ref, Q: (lambda I, A, B: (I, B, A))(*orig(ref, Q)))
    assert not _all_pins_hold()


# --- Navier-Stokes ---------------------------------------------------------------------------------

import oracle.boundary as bd  # noqa: E402

MU, PR = 2e-2, 0.71


def _ns_case(N, bc, n=(2, 2, 2)):
    box = hex_box(n, 1.0)
    box["bc"] = bc
    ref = hx.hex_reference(gll_nodes(N))
    return box, ref, hex_nodes(box, ref.nodes)


def _ns_state(rho, u, v, w, p):
    E = p / 0.4 + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E])


def _ns_viscous_part_is_collocated(N=3):
    """A gas at rest with a temperature of x alone between a no-slip wall at x = 0 and a slip wall
    at x = 1: the viscous flux is the heat flux kappa T'(x) along x only, a field of x alone, on
    which the rule and the collocation agree; so the viscous part (Navier-Stokes minus Euler) of
    the over-integrated right-hand side is that of the collocated one.  (The whole right-hand sides
    differ: the pressure enters the transverse momentum fluxes, across which the collocation lumps
    the mass and the rule does not.)"""
    box, ref, xyz = _ns_case(N, ((bd.NOSLIP_WALL, bd.SLIP_WALL), (0, 0), (0, 0)))
    x = xyz[..., 0]
    one = np.ones_like(x)
    p = 1.0 + 0.1 * (x - 0.5) ** N + 0.05 * np.sin(3 * x)
    q = _ns_state(one, 0 * one, 0 * one, 0 * one, p)
    Q = _q32(N)
    vo = hx.hex_rhs_overint_ns(ref, box, q, GAS, MU, PR, Q) - hx.hex_rhs_overint(ref, box, q, GAS, Q)
    vc = hx.hex_rhs_ns(ref, box, q, GAS, MU, PR) - hx.hex_rhs_ns(ref, box, q, GAS, 0.0, PR)
    return np.abs(vo - vc).max() <= 1e-11 * np.abs(vc).max() and np.abs(vc).max() > 1e-3


def _ns_conserves(N=3):
    box, ref, xyz = _ns_case(N, ((0, 0), (0, 0), (0, 0)), n=(3, 2, 2))
    q = isentropic_vortex(xyz, 0.0, center=(0.45, 0.55), radius=0.15, period=box["L"])
    r = hx.hex_rhs_overint_ns(ref, box, q, GAS, MU, PR, _q32(N))
    periodic = bool(np.all(np.abs(hx.hex_integrate(ref, box, r)) <= 1e-12 * hx.hex_integrate(ref, box, np.abs(r))))
    box, ref, xyz = _ns_case(N, ((bd.NOSLIP_WALL,) * 2, (bd.NOSLIP_WALL,) * 2, (bd.NOSLIP_WALL,) * 2))
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    qb = _ns_state(1.0 + 0.1 * np.sin(2 * x), 0.1 * np.sin(3 * y), 0.05 * np.cos(2 * x), 0 * x, 0.8 + 0.05 * z)
    rb = hx.hex_rhs_overint_ns(ref, box, qb, GAS, MU, PR, _q32(N))
    ib, ab = hx.hex_integrate(ref, box, rb), hx.hex_integrate(ref, box, np.abs(rb))
    closed = abs(ib[0]) <= 1e-12 * ab[0] and abs(ib[4]) <= 1e-12 * ab[4]
    return periodic and closed


def _ns_rest(N=3):
    box, ref, xyz = _ns_case(N, ((bd.NOSLIP_WALL,) * 2, (bd.NOSLIP_WALL,) * 2, (bd.SLIP_WALL,) * 2))
    one = np.ones(xyz.shape[:-1])
    q = _ns_state(one, 0 * one, 0 * one, 0 * one, 0.8 * one)
    return np.abs(hx.hex_rhs_overint_ns(ref, box, q, GAS, MU, PR, _q32(N))).max() <= 1e-11


def test_ns_viscous_part_is_the_collocated_one():
    assert _ns_viscous_part_is_collocated(2)
    assert _ns_viscous_part_is_collocated(3)


def test_ns_conservation_and_rest_state():
    assert _ns_conserves(2)
    assert _ns_rest(2)
    assert _ns_rest(3)


def _av_part_is_collocated(N=3, mu=0.0):
    """A state of x alone with the element viscosities varying along x, between walls at x = 0 and
    x = 1: the AV flux is along x only and a field of x alone, so the AV part of the
    over-integrated right-hand side (with minus without AV) equals the collocated AV term."""
    box, ref, xyz = _ns_case(N, ((bd.SLIP_WALL, bd.NOSLIP_WALL), (0, 0), (0, 0)), n=(3, 1, 1))
    x = xyz[..., 0]
    rho = 1.0 + 0.2 * np.sin(3 * x)
    q = _ns_state(rho, 0.3 + 0.1 * np.cos(2 * x), 0 * x, 0 * x, 1.0 + 0.1 * x ** 2)
    eps = np.array([0.0, 0.02, 0.05])
    Q = _q32(N)
    with_av = hx.hex_rhs_overint_av(ref, box, q, GAS, eps, Q, mu=mu, Pr=PR)
    without = hx.hex_rhs_overint_av(ref, box, q, GAS, 0 * eps, Q, mu=mu, Pr=PR)
    want = hx.hex_rhs_av(ref, box, q, eps)
    return np.abs((with_av - without) - want).max() <= 1e-11 * np.abs(want).max() and np.abs(want).max() > 1e-3


def _av_conserves(N=2):
    box, ref, xyz = _ns_case(N, ((0, 0), (0, 0), (0, 0)), n=(3, 2, 2))
    q = isentropic_vortex(xyz, 0.0, center=(0.45, 0.55), radius=0.15, period=box["L"])
    eps = np.linspace(0.0, 0.03, q.shape[1])
    r = hx.hex_rhs_overint_av(ref, box, q, GAS, eps, _q32(N), mu=MU, Pr=PR)
    return bool(np.all(np.abs(hx.hex_integrate(ref, box, r)) <= 1e-12 * hx.hex_integrate(ref, box, np.abs(r))))


def test_av_part_is_the_collocated_one():
    assert _av_part_is_collocated(2)
    assert _av_part_is_collocated(3)
    assert _av_part_is_collocated(3, mu=MU)
    assert _av_conserves(2)


def _ns_pins_hold():
    return (_ns_viscous_part_is_collocated(2) and _ns_conserves(2) and _ns_rest(2)
            and _av_part_is_collocated(2))


_VOL = hx.hex_overint_volume


@pytest.mark.parametrize("plant", ["no_viscous_volume", "viscous_faces_dropped"])
def test_planted_ns_mistake_fails(plant, monkeypatch):
    assert _ns_pins_hold()
    if plant == "no_viscous_volume":
        monkeypatch.setattr(hx, "hex_overint_volume", lambda ref, box, q5, gas, Q, Fv5=None: _VOL(ref, box, q5, gas, Q))
    else:
        monkeypatch.setattr(hx, "_viscous_face_traces", lambda ref, box, Fv5: iter(()))
    assert not _ns_pins_hold()
