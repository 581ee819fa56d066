"""Pins of the oracle's Euler right-hand side and LSRK4 against what the method fixes.

freestream preservation, discrete conservation on periodic meshes, strong = weak
form, mirror / axis-swap symmetry, element relabelling, and order N+1 convergence
to the translating isentropic vortex (order N for the right-hand side itself).
"""

import numpy as np
import pytest

from oracle.euler import rhs_strong, rhs_weak
from oracle.lsrk import lsrk4_step
from oracle.thermo import PerfectGas
from tests._oracle_case import Disc, box_disc
from workloads import box_mesh, freestream, isentropic_vortex, uniform_perturbation, taylor_green

GAS = PerfectGas(1.4, 1.0)


def vortex_state(d, noise=0.0):
    q = isentropic_vortex(d.xyz, 0.0, center=(0.45, 0.55), radius=0.15, period=d.period)
    return uniform_perturbation(q, noise, seed=3) if noise else q


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_freestream_preservation(N):
    d = box_disc(3, N)
    q = freestream((d.K, d.ref.Np))
    assert np.abs(rhs_strong(d.ref, d.geo, d.conn, q, GAS)).max() < 1e-12
    # the weak form is a cross-check only; M^-1 D^T M in float64 costs it about a digit at N = 4
    assert np.abs(rhs_weak(d.ref, d.geo, d.conn, q, GAS)).max() < 1e-11


@pytest.mark.parametrize("N", [1, 2, 3])
def test_discrete_conservation(N):
    d = box_disc(3, N)
    q = vortex_state(d, noise=1e-2)
    rhs = rhs_strong(d.ref, d.geo, d.conn, q, GAS)
    total = d.integrate(rhs)
    scale = d.abs_integral(rhs)
    assert np.all(np.abs(total) <= 1e-12 * scale)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_strong_equals_weak(N):
    d = box_disc(3, N)
    q = vortex_state(d, noise=1e-3)
    a = rhs_strong(d.ref, d.geo, d.conn, q, GAS)
    b = rhs_weak(d.ref, d.geo, d.conn, q, GAS)
    for v in range(5):
        assert np.abs(a[v] - b[v]).max() <= 1e-11 * np.abs(a[v]).max()


def _transformed_disc(d, A, shift):
    """Mesh mapped by x -> A x + shift (A orthogonal with det -1), re-oriented by swapping vertices 2, 3."""
    v = d.vertices @ A.T + shift
    v = v[:, [0, 1, 3, 2]]
    return Disc(v, d.period, d.N)


def _node_match(d, d2, A, shift):
    """For each element k and node i of d2, the node j of d with A x_j + shift = x2_i."""
    mapped = d.xyz @ A.T + shift
    dist = np.linalg.norm(d2.xyz[:, :, None, :] - mapped[:, None, :, :], axis=3)
    j = np.argmin(dist, axis=2)
    assert np.take_along_axis(dist, j[:, :, None], 2).max() < 1e-12
    return j


def _smooth_state(xyz):
    q = taylor_green(xyz, mach=0.3)
    # add a smooth density/energy variation so that every flux component is exercised
    bump = 0.05 * np.sin(2 * np.pi * xyz[..., 0] + 1.0) * np.cos(2 * np.pi * xyz[..., 1] - 0.5) * np.sin(
        2 * np.pi * xyz[..., 2] + 0.3)
    q[0] = q[0] + bump
    q[4] = q[4] + 2.0 * bump
    q[3] = q[3] + 0.03 * np.cos(2 * np.pi * xyz[..., 0])
    return q


@pytest.mark.parametrize("N", [1, 3])
@pytest.mark.parametrize("kind", ["mirror_x", "swap_xy", "mirror_z"])
def test_symmetry(N, kind):
    d = box_disc(2, N)
    if kind == "mirror_x":
        A = np.diag([-1.0, 1.0, 1.0])
    elif kind == "mirror_z":
        A = np.diag([1.0, 1.0, -1.0])
    else:
        A = np.array([[0.0, 1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    shift = np.where(np.diag(A) < 0, d.period, 0.0)
    d2 = _transformed_disc(d, A, shift)
    j = _node_match(d, d2, A, shift)
    q = _smooth_state(d.xyz)
    rhs = rhs_strong(d.ref, d.geo, d.conn, q, GAS)

    def act(u):  # u[5][...] -> transformed state: velocity components rotate with A
        out = u.copy()
        out[1:4] = np.einsum("ab,b...->a...", A, u[1:4])
        return out

    q2 = act(np.take_along_axis(q, j[None], axis=2))
    rhs2 = rhs_strong(d2.ref, d2.geo, d2.conn, q2, GAS)
    expect = act(np.take_along_axis(rhs, j[None], axis=2))
    assert np.abs(rhs2 - expect).max() < 1e-11 * np.abs(rhs).max()


def test_element_relabelling():
    d = box_disc(3, 2)
    rng = np.random.default_rng(5)
    perm = rng.permutation(d.K)
    d2 = Disc(d.vertices[perm], d.period, 2)
    q = vortex_state(d, noise=1e-3)
    a = rhs_strong(d.ref, d.geo, d.conn, q, GAS)
    b = rhs_strong(d2.ref, d2.geo, d2.conn, q[:, perm], GAS)
    assert np.abs(b - a[:, perm]).max() < 1e-13 * np.abs(a).max()


def _lf_properties_hold(rng):
    """Consistency, conservation and dissipativity of the numerical flux on random face states."""
    from oracle.euler import euler_flux, lax_friedrichs, normal_flux
    m = 64
    qM = np.stack([rng.uniform(0.5, 2, m), *rng.uniform(-1, 1, (3, m)), rng.uniform(4, 8, m)])
    qP = np.stack([rng.uniform(0.5, 2, m), *rng.uniform(-1, 1, (3, m)), rng.uniform(4, 8, m)])
    n = rng.normal(size=(3, m))
    n /= np.linalg.norm(n, axis=0)
    pM, cM = GAS.pressure_sound_speed(qM)
    pP, cP = GAS.pressure_sound_speed(qP)
    f = lax_friedrichs(qM, qP, pM, pP, cM, cP, n)
    ok = np.allclose(lax_friedrichs(qM, qM, pM, pM, cM, cM, n), normal_flux(euler_flux(qM, pM), n), atol=1e-13)
    ok &= np.allclose(f, -lax_friedrichs(qP, qM, pP, pM, cP, cM, -n), atol=1e-13)
    avg = 0.5 * (normal_flux(euler_flux(qM, pM), n) + normal_flux(euler_flux(qP, pP), n))
    diss = f - avg  # = lambda/2 (qM - qP) with lambda >= the largest wave speed
    lam = 2 * np.sum(diss * (qM - qP), axis=0) / np.sum((qM - qP) ** 2, axis=0)
    un = lambda q, c: np.abs(np.sum(q[1:4] / q[0] * n, axis=0)) + c
    ok &= bool(np.all(lam >= np.maximum(un(qM, cM), un(qP, cP)) - 1e-12))
    return bool(ok)


def _consistency_holds():
    """rhs of the exact vortex within 10% of its exact time derivative (N = 3, 16 x 16 x 1 cells)."""
    v, per = box_mesh((16, 16, 1), (_L, _L, _L / 16))
    d = Disc(v, per, 3)
    kw = dict(center=(5.0, 5.0), radius=_R, u_inf=(1.0, 0.0), period=per)
    q = isentropic_vortex(d.xyz, 0.0, **kw)
    dq = np.imag(isentropic_vortex(d.xyz, 1e-30j, **kw)) / 1e-30
    r = rhs_strong(d.ref, d.geo, d.conn, q, GAS)
    scale = d.l2(dq).max()
    return bool(np.all(d.l2(r - dq) < 0.1 * scale))


def _conservation_holds():
    d = box_disc(2, 2)
    q = vortex_state(d, noise=1e-2)
    rhs = rhs_strong(d.ref, d.geo, d.conn, q, GAS)
    return bool(np.all(np.abs(d.integrate(rhs)) <= 1e-12 * d.abs_integral(rhs)))


def _all_pins_hold():
    return _lf_properties_hold(np.random.default_rng(9)) and _consistency_holds() and _conservation_holds()


def test_flux_and_consistency_pins_hold():
    assert _lf_properties_hold(np.random.default_rng(9))
    assert _consistency_holds()
    assert _conservation_holds()


def _plant_lf_antidissipative(eu):
    orig = eu.lax_friedrichs
    return "lax_friedrichs", lambda qM, qP, pM, pP, cM, cP, n: (
        2 * (0.5 * (eu.normal_flux(eu.euler_flux(qM, pM), n) + eu.normal_flux(eu.euler_flux(qP, pP), n)))
        - orig(qM, qP, pM, pP, cM, cP, n))


def _plant_pressure_sign(eu):
    orig = eu.euler_flux

    def bad(q, p):
        return orig(q, -p)
    return "euler_flux", bad


def _plant_drop_surface(eu):
    return "lift", lambda ref, geo, g: np.zeros(g.shape[:2] + (ref.Np,))


def _plant_swapped_normal(eu):
    orig = eu.face_normals
    return "face_normals", lambda geo, Nfp: orig(geo, Nfp)[[1, 0, 2]]


def _plant_transposed_ds(eu):
    orig = eu.ref_derivatives
    return "ref_derivatives", lambda ref, u: [orig(ref, u)[0], np.einsum("ji,vkj->vki", ref.Ds, u), orig(ref, u)[2]]


@pytest.mark.parametrize("plant", [_plant_lf_antidissipative, _plant_pressure_sign, _plant_drop_surface,
                                   _plant_swapped_normal, _plant_transposed_ds])
def test_planted_mistake_fails_a_pin(plant, monkeypatch):
    import oracle.euler as eu
    name, fn = plant(eu)
    monkeypatch.setattr(eu, name, fn)
    assert not _all_pins_hold()


# --- convergence to the translating isentropic vortex ---------------------------------------

_L, _R = 10.0, 1.0


def _vortex_run(n, N, T):
    v, per = box_mesh((n, n, 1), (_L, _L, _L / n))
    d = Disc(v, per, N)
    kw = dict(center=(5.0, 5.0), radius=_R, u_inf=(1.0, 0.0), period=per)
    q = isentropic_vortex(d.xyz, 0.0, **kw)
    f = lambda u: rhs_strong(d.ref, d.geo, d.conn, u, GAS)
    eps = 1e-30
    dqdt = np.imag(isentropic_vortex(d.xyz, 1j * eps, **kw)) / eps  # complex-step time derivative
    consistency = np.linalg.norm(d.l2(f(q) - dqdt))
    dt0 = 0.3 * (_L / n) / ((N + 1) ** 2 * 2.5)
    steps = int(np.ceil(T / dt0))
    for _ in range(steps):
        q = lsrk4_step(q, T / steps, f)
    err = q - isentropic_vortex(d.xyz, T, **kw)
    return np.linalg.norm(d.l2(err)), consistency


@pytest.mark.slow
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_vortex_convergence(N):
    T = 0.2 if N < 4 else 0.1
    e8, c8 = _vortex_run(8, N, T)
    e16, c16 = _vortex_run(16, N, T)
    rate = np.log2(e8 / e16)
    assert rate >= N + 0.5, (N, rate)
    assert np.log2(c8 / c16) >= N - 0.9, (N, np.log2(c8 / c16))
