"""Pins of the reductions oracle (oracle/diagnostics.py): the integrals against exact volumes and
monomial integrals of the box, and against conservation (a periodic right-hand side integrates to
zero); the stability rate against its closed form on the Kuhn box, whose tetrahedra all have
max Fscale = 2 sqrt(2) / h (largest face area sqrt(2) h^2 / 2 over twice the reference face area,
divided by J = (h^3 / 6) / (4 / 3)), and against its scaling laws."""

import numpy as np
import pytest

import oracle.diagnostics as dgn
from oracle.euler import rhs_strong
from oracle.ns import rhs_ns
from oracle.thermo import PerfectGas
from tests._oracle_case import Disc
from workloads import box_mesh, isentropic_vortex, uniform_perturbation

GAS = PerfectGas(1.4, 1.0)


def _disc(n, N, L):
    v, per = box_mesh(n, L)
    return Disc(v, per, N)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_integral_of_one_is_the_box_volume(N):
    L = (1.3, 0.7, 2.1)
    d = _disc((2, 3, 2), N, L)
    got = dgn.integrals(d.ref, d.geo, np.ones((1, d.K, d.ref.Np)))[0]
    assert abs(got - np.prod(L)) <= 1e-13 * np.prod(L)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_monomials_up_to_degree_N_integrate_exactly(N):
    L = (1.3, 0.7, 2.1)
    d = _disc((2, 2, 3), N, L)
    x, y, z = (d.xyz[..., a] for a in range(3))
    for a in range(N + 1):
        for b in range(N + 1 - a):
            c = N - a - b
            want = L[0] ** (a + 1) / (a + 1) * L[1] ** (b + 1) / (b + 1) * L[2] ** (c + 1) / (c + 1)
            got = dgn.integrals(d.ref, d.geo, (x ** a * y ** b * z ** c)[None])[0]
            assert abs(got - want) <= 1e-13 * want, (a, b, c)


@pytest.mark.parametrize("viscous", [False, True])
def test_periodic_right_hand_side_conserves(viscous):
    d = _disc((3, 2, 2), 3, 1.0)
    q = uniform_perturbation(isentropic_vortex(d.xyz, 0.0, period=d.period), 1e-2, seed=2)
    r = rhs_ns(d.ref, d.geo, d.conn, q, GAS, 0.05, 0.71) if viscous else rhs_strong(d.ref, d.geo, d.conn, q, GAS)
    tot = dgn.integrals(d.ref, d.geo, r)
    scale = dgn.integrals(d.ref, d.geo, np.abs(r))
    assert np.all(np.abs(tot) <= 1e-12 * scale), tot / scale
    # and a non-conserving change (a dropped surface term) is seen
    from oracle.euler import divergence, euler_flux
    vol_only = -divergence(d.ref, d.geo, euler_flux(q, GAS.pressure(q)))
    assert np.abs(dgn.integrals(d.ref, d.geo, vol_only)).max() > 1e-6 * scale.max()


@pytest.mark.parametrize("N", [1, 3])
@pytest.mark.parametrize("mu", [0.0, 0.03])
def test_rate_closed_form_on_a_uniform_state(N, mu):
    h = 0.25
    d = _disc(4, N, 1.0)
    rho, u, p = 1.3, np.array([0.4, -0.2, 0.1]), 0.9
    q = np.empty((5, d.K, d.ref.Np))
    q[0] = rho
    q[1:4] = (rho * u)[:, None, None]
    q[4] = p / 0.4 + 0.5 * rho * (u @ u)
    speed = np.linalg.norm(u) + np.sqrt(1.4 * p / rho)
    nu = mu / rho * max(4.0 / 3.0, 1.4 / 0.71)
    want = (N + 1) ** 2 * np.sqrt(2.0) * speed / h + (N + 1) ** 4 * 2.0 * nu / h ** 2
    got = dgn.max_rate(d.ref, d.geo, q, GAS, mu, 0.71)
    assert abs(got - want) <= 1e-13 * want
    assert np.allclose(d.geo.Fscale.max(axis=1), 2.0 * np.sqrt(2.0) / h, rtol=1e-13, atol=0)


def test_rate_scales_with_the_mesh_and_takes_the_largest_node():
    N = 2
    d1, d2 = _disc(3, N, 1.0), _disc(3, N, 2.0)  # same tetrahedra, twice the size
    q = uniform_perturbation(isentropic_vortex(d1.xyz, 0.0, period=d1.period), 1e-2, seed=4)
    a1 = dgn.max_rate(d1.ref, d1.geo, q, GAS)
    a2 = dgn.max_rate(d2.ref, d2.geo, q, GAS)
    assert abs(a1 / a2 - 2.0) <= 1e-13
    # with viscosity each node's rate is 2x (advective part) plus 4x (diffusive part) that of the
    # larger mesh, so the ratio of the maxima lies in [2, 4], above 2 once viscosity counts
    v1 = dgn.max_rate(d1.ref, d1.geo, q, GAS, 0.1, 0.71)
    v2 = dgn.max_rate(d2.ref, d2.geo, q, GAS, 0.1, 0.71)
    assert v1 > a1 and 2.0 + 1e-3 <= v1 / v2 <= 4.0 + 1e-12
    # raising one node's speed raises the rate to exactly that node's value
    q2 = q.copy()
    k, i = 7, 3
    q2[1, k, i] *= 30.0
    q2[4, k, i] += 0.5 * (q2[1, k, i] ** 2 - q[1, k, i] ** 2) / q[0, k, i]
    rates = dgn.element_rates(d1.ref, d1.geo, q2, GAS)
    assert int(np.argmax(rates)) == k
    uk = q2[1:4, k, i] / q2[0, k, i]
    pk = 0.4 * (q2[4, k, i] - 0.5 * q2[0, k, i] * (uk @ uk))
    node = (N + 1) ** 2 / 2 * d1.geo.Fscale[k].max() * (np.linalg.norm(uk) + np.sqrt(1.4 * pk / q2[0, k, i]))
    assert abs(rates[k] - node) <= 1e-13 * node
