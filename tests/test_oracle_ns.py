"""Pins of the oracle's BR1 Navier-Stokes right-hand side.

Each viscous term is checked on a smooth periodic state whose viscous
contribution has a closed form derived by hand (shear stress, compression with
the -2/3 div u term, heat conduction, and the product rule for velocity
gradients under variable density), together with conservation, the rest
state, gradient exactness and mirror symmetry.
"""

import numpy as np
import pytest

from oracle.euler import rhs_strong
from oracle.ns import dg_gradient, rhs_ns
from oracle.thermo import PerfectGas
from tests._oracle_case import Disc, box_disc
from workloads import box_mesh, freestream, taylor_green, uniform_perturbation

GAS = PerfectGas(1.4, 1.0)
MU, PR = 2e-2, 0.71
KAPPA = MU * GAS.cp / PR
K2PI = 2 * np.pi


def _state(rho, u, v, w, p):
    E = p / (GAS.gamma - 1) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E])


def _case(name, xyz):
    """(q, exact viscous contribution [5][...]) for the closed-form cases."""
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    one, zero = np.ones_like(x), np.zeros_like(x)
    A, B, k = 0.2, 0.1, K2PI
    if name == "shear_y":  # u = A sin(ky): tau_xy = mu u'
        u, du, d2u = A * np.sin(k * y), A * k * np.cos(k * y), -A * k * k * np.sin(k * y)
        q = _state(one, u, zero, zero, one)
        visc = np.stack([zero, MU * d2u, zero, zero, MU * (du * du + u * d2u)])
    elif name == "compress_x":  # u = A sin(kx): tau_xx = 4/3 mu u'
        u, du, d2u = A * np.sin(k * x), A * k * np.cos(k * x), -A * k * k * np.sin(k * x)
        q = _state(one, u, zero, zero, one)
        visc = np.stack([zero, 4 / 3 * MU * d2u, zero, zero, 4 / 3 * MU * (du * du + u * d2u)])
    elif name == "heat_z":  # at rest, T = p / rho = 1 + B sin(kz)
        p = 1 + B * np.sin(k * z)
        q = _state(one, zero, zero, zero, p)
        visc = np.stack([zero, zero, zero, zero, -KAPPA * B * k * k * np.sin(k * z)])
    elif name == "variable_density":  # rho = 1 + B sin(kx), v = A sin(kx), p = 1: T = 1 / rho
        rho = 1 + B * np.sin(k * x)
        drho, d2rho = B * k * np.cos(k * x), -B * k * k * np.sin(k * x)
        v, dv, d2v = A * np.sin(k * x), A * k * np.cos(k * x), -A * k * k * np.sin(k * x)
        d2T = -d2rho / rho ** 2 + 2 * drho ** 2 / rho ** 3
        q = _state(rho, zero, v, zero, one)
        visc = np.stack([zero, zero, MU * d2v, zero, MU * (dv * dv + v * d2v) + KAPPA * d2T])
    else:
        raise ValueError(name)
    return q, visc


def _viscous_part(d, q):
    return rhs_ns(d.ref, d.geo, d.conn, q, GAS, MU, PR) - rhs_strong(d.ref, d.geo, d.conn, q, GAS)


@pytest.mark.parametrize("name", ["shear_y", "compress_x", "heat_z", "variable_density"])
def test_viscous_terms_converge_to_closed_form(name):
    errs = []
    for n in (3, 6):
        d = box_disc(n, 4)
        q, visc = _case(name, d.xyz)
        err = _viscous_part(d, q) - visc
        errs.append(np.linalg.norm(d.l2(err)))
        scale = np.linalg.norm(d.l2(visc))
    # BR1's pointwise second-derivative operator converges at about order N - 1 (= 3 here)
    assert errs[1] < 0.02 * scale, (errs, scale)
    assert np.log2(errs[0] / errs[1]) > 2.0, errs


@pytest.mark.parametrize("N", [1, 2, 3])
def test_rest_and_uniform_states(N):
    d = box_disc(2, N)
    q = freestream((d.K, d.ref.Np))
    assert np.abs(rhs_ns(d.ref, d.geo, d.conn, q, GAS, MU, PR)).max() < 1e-12


@pytest.mark.parametrize("N", [2, 3])
def test_conservation(N):
    d = box_disc(3, N)
    q = uniform_perturbation(taylor_green(d.xyz, mach=0.3), 1e-2, seed=2)
    rhs = rhs_ns(d.ref, d.geo, d.conn, q, GAS, MU, PR)
    assert np.all(np.abs(d.integrate(rhs)) <= 1e-12 * d.abs_integral(rhs))


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_gradient_of_constants_and_polynomial_interior(N):
    d = box_disc(2, N)
    c = np.full((1, d.K, d.ref.Np), 3.7)
    assert np.abs(dg_gradient(d.ref, d.geo, d.conn, c)).max() < 1e-12
    # a global polynomial of degree <= N of the coordinates is continuous inside the box: on
    # every element whose face traces agree with the neighbours' (all but those at the periodic
    # seam) the BR1 surface term vanishes and the volume term differentiates it exactly
    d3 = box_disc(4, N)
    xyz = d3.xyz
    f = (xyz[..., 0] - 0.5) ** N + 0.3 * (xyz[..., 1] - 0.5) * (xyz[..., 2] - 0.5) ** (N - 1)
    g = dg_gradient(d3.ref, d3.geo, d3.conn, f[None])[:, 0]
    exact = np.stack([N * (xyz[..., 0] - 0.5) ** (N - 1), 0.3 * (xyz[..., 2] - 0.5) ** (N - 1),
                      0.3 * (N - 1) * (xyz[..., 1] - 0.5) * (xyz[..., 2] - 0.5) ** max(N - 2, 0)])
    flat = f.ravel()
    jump = np.abs(flat[d3.conn.vmapM] - flat[d3.conn.vmapP]).max(axis=1)
    sel = jump < 1e-14
    assert sel.sum() > d3.K // 4
    assert np.abs(g[:, sel] - exact[:, sel]).max() < 1e-11


def test_mirror_symmetry():
    from tests.test_oracle_euler import _node_match, _transformed_disc
    d = box_disc(2, 2)
    A = np.diag([1.0, -1.0, 1.0])
    shift = np.array([0.0, 1.0, 0.0])
    d2 = _transformed_disc(d, A, shift)
    j = _node_match(d, d2, A, shift)
    q = uniform_perturbation(taylor_green(d.xyz, mach=0.3), 0.0)
    q[0] += 0.05 * np.sin(K2PI * d.xyz[..., 1] + 0.3)
    rhs = rhs_ns(d.ref, d.geo, d.conn, q, GAS, MU, PR)

    def act(u):
        out = u.copy()
        out[1:4] = np.einsum("ab,b...->a...", A, u[1:4])
        return out

    q2 = act(np.take_along_axis(q, j[None], axis=2))
    rhs2 = rhs_ns(d2.ref, d2.geo, d2.conn, q2, GAS, MU, PR)
    assert np.abs(rhs2 - act(np.take_along_axis(rhs, j[None], axis=2))).max() < 1e-11 * np.abs(rhs).max()


def _plant(ns, kind):
    orig = ns.viscous_flux
    if kind == "drop_transpose":
        def bad(q, T, grad, mu, kappa):
            Fv = orig(q, T, grad, mu, kappa)
            half = orig(q, T, grad, mu / 2, kappa)  # mu (du_i/dx_j + du_j/dx_i) -> roughly half of it
            return half
        return bad
    if kind == "heat_sign":
        return lambda q, T, grad, mu, kappa: orig(q, T, grad, mu, -kappa)
    if kind == "product_rule":
        def bad(q, T, grad, mu, kappa):
            g = grad.copy()
            g[:, 0] = 0.0  # forget the u grad(rho) term
            return orig(q, T, g, mu, kappa)
        return bad
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["drop_transpose", "heat_sign", "product_rule"])
def test_planted_viscous_mistake_fails_a_pin(kind, monkeypatch):
    import oracle.ns as ns
    monkeypatch.setattr(ns, "viscous_flux", _plant(ns, kind))
    failed = False
    for name in ["shear_y", "compress_x", "heat_z", "variable_density"]:
        d = box_disc(6, 4)
        q, visc = _case(name, d.xyz)
        err = np.linalg.norm(d.l2(_viscous_part(d, q) - visc))
        failed |= err >= 0.02 * np.linalg.norm(d.l2(visc))
    assert failed
