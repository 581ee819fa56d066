"""Pins of the tensor-product hexahedron oracle (oracle/hex.py) against what the mathematics fixes:
closed-form Gauss-Lobatto-Legendre nodes and weights, quadrature exactness, exact
differentiation, the summation-by-parts identity, freestream preservation, discrete
conservation, strong = weak form, translation invariance and convergence to the translating
isentropic vortex; for scalar advection also the upwind energy identity, the reduction to the
textbook 1-D upwind scheme written out by loops, and convergence against the exact translated
wave.  Planted mistakes must break at least one pin."""

import numpy as np
import pytest

import oracle.hex as hx
from oracle.lsrk import lsrk4_step
from oracle.thermo import PerfectGas
from workloads import isentropic_vortex, uniform_perturbation
from workloads.hexmesh import gll_nodes, hex_box, hex_nodes

GAS = PerfectGas(1.4, 1.0)
S5, S37 = np.sqrt(1.0 / 5.0), np.sqrt(3.0 / 7.0)
CLOSED = {  # nodes, weights of the (N+1)-point Gauss-Lobatto-Legendre rule
    1: ([-1, 1], [1, 1]),
    2: ([-1, 0, 1], [1 / 3, 4 / 3, 1 / 3]),
    3: ([-1, -S5, S5, 1], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    4: ([-1, -S37, 0, S37, 1], [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
}


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_gll_closed_forms(N):
    x, w = CLOSED[N]
    ref = hx.hex_reference(gll_nodes(N))
    assert np.abs(ref.nodes - np.array(x)).max() <= 1e-15
    assert np.abs(ref.w - np.array(w)).max() <= 1e-15


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_quadrature_exact_to_degree_2n_minus_1(N):
    ref = hx.hex_reference(gll_nodes(N))
    for m in range(2 * N):
        exact = (1 - (-1) ** (m + 1)) / (m + 1)
        assert abs(ref.w @ ref.nodes ** m - exact) <= 1e-14
    m = 2 * N  # the first degree the rule misses
    assert abs(ref.w @ ref.nodes ** m - 2.0 / (m + 1)) > 1e-3


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_exact_differentiation_and_sbp(N):
    ref = hx.hex_reference(gll_nodes(N))
    x = ref.nodes
    for m in range(N + 1):
        want = m * x ** (m - 1) if m else np.zeros_like(x)
        assert np.abs(ref.D @ x ** m - want).max() <= 1e-13
    B = np.zeros((N + 1, N + 1))
    B[0, 0], B[N, N] = -1.0, 1.0
    W = np.diag(ref.w)
    assert np.abs(W @ ref.D + ref.D.T @ W - B).max() <= 1e-14


def _case(n, N, noise=0.0, seed=0):
    box = hex_box(n, 1.0)
    x = gll_nodes(N)
    ref = hx.hex_reference(x)
    q = isentropic_vortex(hex_nodes(box, x), 0.0, center=(0.45, 0.55), radius=0.15, period=box["L"])
    if noise:
        q = uniform_perturbation(q, noise, seed=seed)
    return box, ref, q


def _freestream_holds(N=3):
    box, ref, q = _case((3, 2, 2), N)
    qf = np.ones_like(q)
    qf[1], qf[2], qf[3], qf[4] = 0.3, -0.2, 0.1, 2.5
    return np.abs(hx.hex_rhs_strong(ref, box, qf, GAS)).max() <= 1e-12


def _conservation_holds(N=3):
    box, ref, q = _case((3, 2, 2), N, noise=1e-2)
    rhs = hx.hex_rhs_strong(ref, box, q, GAS)
    tot = hx.hex_integrate(ref, box, rhs)
    scale = hx.hex_integrate(ref, box, np.abs(rhs))
    return bool(np.all(np.abs(tot) <= 1e-12 * scale))


def _strong_equals_weak(N=3):
    box, ref, q = _case((3, 2, 2), N, noise=1e-2)
    rs, rw = hx.hex_rhs_strong(ref, box, q, GAS), hx.hex_rhs_weak(ref, box, q, GAS)
    return np.abs(rs - rw).max() <= 1e-12 * np.abs(rs).max()


def _consistency_holds(N=3):
    # the semi-discrete rate of the translating vortex approaches the exact one with h
    errs = []
    for n in (4, 8):
        box = hex_box((n, n, 1), (10.0, 10.0, 10.0 / n))
        x = gll_nodes(N)
        ref = hx.hex_reference(x)
        xyz = hex_nodes(box, x)
        kw = dict(center=(5.0, 5.0), radius=1.0, u_inf=(1.0, 0.0), period=box["L"])
        dqdt = np.imag(isentropic_vortex(xyz, 1e-30j, **kw)) / 1e-30
        r = hx.hex_rhs_strong(ref, box, isentropic_vortex(xyz, 0.0, **kw), GAS) - dqdt
        errs.append(np.sqrt(hx.hex_integrate(ref, box, r ** 2).sum()))
    return np.log2(errs[0] / errs[1]) >= N - 0.9


def _all_pins_hold():
    return _freestream_holds() and _conservation_holds() and _strong_equals_weak() and _consistency_holds()


def test_rhs_pins_hold():
    assert _freestream_holds()
    assert _conservation_holds()
    assert _strong_equals_weak()
    assert _consistency_holds()


@pytest.mark.parametrize("N", [1, 2, 4])
def test_rhs_pins_other_orders(N):
    assert _freestream_holds(N) and _conservation_holds(N) and _strong_equals_weak(N)


def test_translation_invariance():
    """Shifting the state by one element along x shifts the right-hand side the same way."""
    box, ref, q = _case((3, 2, 2), 2, noise=1e-2)
    nx, ny, nz = box["n"]
    e = np.arange(nx * ny * nz)
    shifted = ((e % nx) + 1) % nx + nx * (e // nx)
    qs = np.empty_like(q)
    qs[:, shifted] = q
    r, rs = hx.hex_rhs_strong(ref, box, q, GAS), hx.hex_rhs_strong(ref, box, qs, GAS)
    assert np.abs(rs[:, shifted] - r).max() <= 1e-13 * np.abs(r).max()


# --- planted mistakes: each must break a pin -----------------------------------------------------

def _plant_wrong_lift(m):
    orig = m._surface_terms
    return "_surface_terms", lambda ref, box, q5, gas, q_in=None: [(s, 0.5 * l, fm, fs) for s, l, fm, fs in
                                                                   orig(ref, box, q5, gas, q_in)]


def _plant_no_dissipation_sign(m):
    orig = m._surface_terms

    def bad(ref, box, q5, gas, q_in=None):
        return [(s, l, fm, 2 * fm - fs) for s, l, fm, fs in orig(ref, box, q5, gas, q_in)]
    return "_surface_terms", bad


def _plant_transposed_d(m):
    orig = m._along
    return "_along", lambda M, a, axis: orig(M.T, a, axis)


def _plant_drop_a_face(m):
    orig = m._surface_terms
    return "_surface_terms", lambda ref, box, q5, gas, q_in=None: orig(ref, box, q5, gas, q_in)[1:]


@pytest.mark.parametrize("plant", [_plant_wrong_lift, _plant_no_dissipation_sign, _plant_transposed_d,
                                   _plant_drop_a_face])
def test_planted_mistake_fails_a_pin(plant, monkeypatch):
    name, fn = plant(hx)
    monkeypatch.setattr(hx, name, fn)
    assert not _all_pins_hold()


# --- convergence to the translating isentropic vortex ------------------------------------------

def _vortex_run(n, N, T):
    L = 10.0
    box = hex_box((n, n, 1), (L, L, L / n))
    x = gll_nodes(N)
    ref = hx.hex_reference(x)
    xyz = hex_nodes(box, x)
    kw = dict(center=(5.0, 5.0), radius=1.0, u_inf=(1.0, 0.0), period=box["L"])
    q = isentropic_vortex(xyz, 0.0, **kw)
    f = lambda u: hx.hex_rhs_strong(ref, box, u, GAS)
    dt0 = 0.3 * (L / n) / ((N + 1) ** 2 * 2.5)
    steps = int(np.ceil(T / dt0))
    for _ in range(steps):
        q = lsrk4_step(q, T / steps, f)
    err = q - isentropic_vortex(xyz, T, **kw)
    return np.sqrt(np.abs(hx.hex_integrate(ref, box, err ** 2)).sum())


@pytest.mark.slow
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_vortex_convergence(N):
    """Collocated GLL integration of the nonlinear flux: rates between N + 1/2 and N + 1 on
    these meshes (1.55, 2.55, 3.72, 4.71 for N = 1..4 at h = 10/8 -> 10/16)."""
    T = 0.2 if N < 4 else 0.1
    rate = np.log2(_vortex_run(8, N, T) / _vortex_run(16, N, T))
    assert rate >= N + 0.3, (N, rate)


# --- scalar advection (the paper's section 5.2 GPU workload) --------------------------------------

ADV_A = (1.0, -0.5, 0.25)


def _adv_case(n, N, noise=0.0, seed=0):
    box = hex_box(n, 1.0)
    x = gll_nodes(N)
    ref = hx.hex_reference(x)
    xyz = hex_nodes(box, x)
    u = np.sin(2 * np.pi * xyz[..., 0]) * np.cos(2 * np.pi * xyz[..., 1]) + 0.3 * np.sin(2 * np.pi * xyz[..., 2])
    if noise:
        u = u + noise * np.random.default_rng(seed).uniform(-1.0, 1.0, u.shape)
    return box, ref, u


def _adv_freestream_holds(N=3):
    box, ref, u = _adv_case((3, 2, 2), N)
    return np.abs(hx.hex_advection_rhs_strong(ref, box, np.full_like(u, 0.7), ADV_A)).max() <= 1e-12


def _adv_conservation_holds(N=3):
    box, ref, u = _adv_case((3, 2, 2), N, noise=1e-2)
    r = hx.hex_advection_rhs_strong(ref, box, u, ADV_A)
    return abs(hx.hex_integrate(ref, box, r[None])[0]) <= 1e-12 * hx.hex_integrate(ref, box, np.abs(r)[None])[0]


def _adv_strong_equals_weak(N=3):
    box, ref, u = _adv_case((3, 2, 2), N, noise=1e-2)
    rs = hx.hex_advection_rhs_strong(ref, box, u, ADV_A)
    rw = hx.hex_advection_rhs_weak(ref, box, u, ADV_A)
    return np.abs(rs - rw).max() <= 1e-12 * np.abs(rs).max()


def _face_jump_energy(ref, box, u, a):
    """1/2 sum over the shared faces (each once) of |a_d| times the collocated face integral of the
    squared jump of u."""
    N, (nx, ny, nz) = ref.N, box["n"]
    u5 = u.reshape(-1, N + 1, N + 1, N + 1)  # [K][k][j][i]
    e = np.arange(nx * ny * nz)
    c = [e % nx, (e // nx) % ny, e // (nx * ny)]
    total = 0.0
    for d in range(3):
        cn = list(c)
        cn[d] = (cn[d] + 1) % box["n"][d]
        nb = cn[0] + nx * (cn[1] + ny * cn[2])
        hi = [slice(None)] * 3
        lo = [slice(None)] * 3
        hi[2 - d], lo[2 - d] = N, 0
        jump = u5[(slice(None),) + tuple(hi)] - u5[nb][(slice(None),) + tuple(lo)]  # [K][face]
        t = [k for k in range(3) if k != d]
        Jf = box["h"][t[0]] * box["h"][t[1]] / 4.0
        wf = np.outer(ref.w, ref.w)  # same tensor weights for either face ordering
        total += 0.5 * abs(a[d]) * Jf * np.sum(wf[None] * jump ** 2)
    return total


def _adv_energy_identity_holds(N=3):
    """d/dt (1/2 ||u||^2) = u^T M rhs = - 1/2 sum_faces |a.n| integral [u]^2: the upwind flux
    dissipates exactly the jump energy (summation by parts, collocated quadrature)."""
    box, ref, u = _adv_case((3, 2, 2), N, noise=5e-2)
    r = hx.hex_advection_rhs_strong(ref, box, u, ADV_A)
    lhs = hx.hex_integrate(ref, box, (u * r)[None])[0]
    rhs = -_face_jump_energy(ref, box, u, ADV_A)
    return abs(lhs - rhs) <= 1e-11 * max(abs(rhs), 1e-300) and rhs < 0


def _adv_matches_1d_upwind(N=3):
    """With a = (a_x, 0, 0) and u varying along x only, every x-line is the textbook 1-D upwind
    nodal DG: rhs = -(2/h) a D u, plus (2/h)/w_0 a (u_left - u_0) at the inflow node (a > 0)."""
    n, ax = 4, 1.3
    box = hex_box((n, 2, 1), 1.0)
    x = gll_nodes(N)
    ref = hx.hex_reference(x)
    xs = hex_nodes(box, x)[..., 0]
    u = np.sin(2 * np.pi * xs) + 0.2 * np.cos(6 * np.pi * xs) + 1e-2 * np.random.default_rng(1).uniform(-1, 1, n)[
        (np.arange(xs.shape[0]) % n)][:, None]
    got = hx.hex_advection_rhs_strong(ref, box, u, (ax, 0.0, 0.0)).reshape(-1, N + 1, N + 1, N + 1)
    u5 = u.reshape(-1, N + 1, N + 1, N + 1)
    h = box["h"][0]
    for e in range(xs.shape[0]):
        left = e - 1 if e % n else e + n - 1
        for k in range(N + 1):
            for j in range(N + 1):
                line = u5[e, k, j, :]
                want = [-(2.0 / h) * ax * sum(ref.D[i][l] * line[l] for l in range(N + 1)) for i in range(N + 1)]
                want[0] += (2.0 / h) / ref.w[0] * ax * (u5[left, k, j, N] - line[0])
                if np.abs(got[e, k, j, :] - np.array(want)).max() > 1e-12 * (1 + np.abs(want).max()):
                    return False
    return True


def _adv_all_pins_hold():
    return (_adv_freestream_holds() and _adv_conservation_holds() and _adv_strong_equals_weak()
            and _adv_energy_identity_holds() and _adv_matches_1d_upwind())


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_advection_pins_hold(N):
    assert _adv_freestream_holds(N)
    assert _adv_conservation_holds(N)
    assert _adv_strong_equals_weak(N)
    assert _adv_energy_identity_holds(N)
    assert _adv_matches_1d_upwind(N)


def test_advection_translation_invariance():
    box, ref, u = _adv_case((3, 2, 2), 2, noise=1e-2)
    nx = box["n"][0]
    e = np.arange(u.shape[0])
    shifted = ((e % nx) + 1) % nx + nx * (e // nx)
    us = np.empty_like(u)
    us[shifted] = u
    r, rs = hx.hex_advection_rhs_strong(ref, box, u, ADV_A), hx.hex_advection_rhs_strong(ref, box, us, ADV_A)
    assert np.abs(rs[shifted] - r).max() <= 1e-13 * np.abs(r).max()


def _plant_adv_downwind(m):
    return "_advection_lambda", lambda an: -abs(an)


def _plant_adv_central(m):
    return "_advection_lambda", lambda an: 0.0


def _plant_adv_wrong_lift(m):
    orig = m._advection_surface_terms
    return "_advection_surface_terms", lambda ref, box, u5, a: [(s, 2.0 * l, fm, fs) for s, l, fm, fs in
                                                                 orig(ref, box, u5, a)]


def _plant_adv_transposed_d(m):
    orig = m._along
    return "_along", lambda M, arr, axis: orig(M.T, arr, axis)


def _plant_adv_drop_a_face(m):
    orig = m._advection_surface_terms
    return "_advection_surface_terms", lambda ref, box, u5, a: orig(ref, box, u5, a)[:-1]


@pytest.mark.parametrize("plant", [_plant_adv_downwind, _plant_adv_central, _plant_adv_wrong_lift,
                                   _plant_adv_transposed_d, _plant_adv_drop_a_face])
def test_advection_planted_mistake_fails_a_pin(plant, monkeypatch):
    name, fn = plant(hx)
    monkeypatch.setattr(hx, name, fn)
    assert not _adv_all_pins_hold()


def _adv_run(n, N, T, a=(1.0, 0.5, 0.0)):
    box = hex_box((n, n, 1), (1.0, 1.0, 1.0 / n))
    x = gll_nodes(N)
    ref = hx.hex_reference(x)
    xyz = hex_nodes(box, x)
    exact = lambda t: np.sin(2 * np.pi * (xyz[..., 0] - a[0] * t)) * np.cos(2 * np.pi * (xyz[..., 1] - a[1] * t))
    u = exact(0.0)
    f = lambda v: hx.hex_advection_rhs_strong(ref, box, v, a)
    dt0 = 0.2 * (1.0 / n) / ((N + 1) ** 2 * (abs(a[0]) + abs(a[1])))
    steps = int(np.ceil(T / dt0))
    for _ in range(steps):
        u = lsrk4_step(u, T / steps, f)
    err = u - exact(T)
    return np.sqrt(hx.hex_integrate(ref, box, (err ** 2)[None])[0])


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_advection_convergence(N):
    """Upwind DG for linear advection converges at order N + 1 or better (measured 1.99, 3.37,
    4.66, 5.65 for N = 1..4 at h = 1/4 -> 1/8); the test asks for N + 1/2."""
    T = 0.25
    rate = np.log2(_adv_run(4, N, T) / _adv_run(8, N, T))
    assert rate >= N + 0.5, (N, rate)
