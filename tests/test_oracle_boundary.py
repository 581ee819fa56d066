"""Pins of the boundary-condition oracle (oracle/boundary.py) against what the mathematics fixes:
it reduces to the periodic right-hand sides when no face is a boundary, preserves uniform states
that satisfy the boundary conditions, conserves mass and energy in boxes closed by walls, matches
the mirror-image periodic problem for a slip wall, passes an entropy wave out through supersonic
inflow/outflow boundaries at the order of the scheme, and strong = weak form; planted mistakes
must break at least one pin."""

import numpy as np
import pytest

import oracle.boundary as bd
from oracle.euler import rhs_strong
from oracle.geometry import affine_nodes
from oracle.lsrk import lsrk4_step
from oracle.ns import rhs_ns
from oracle.thermo import PerfectGas
from tests._oracle_case import Disc, bc_disc, box_disc
from workloads import box_mesh, isentropic_vortex, uniform_perturbation

GAS = PerfectGas(1.4, 1.0)
MU, PR = 2e-2, 0.71
SLIP, NOSLIP, INFLOW, OUTFLOW = bd.SLIP_WALL, bd.NOSLIP_WALL, bd.INFLOW, bd.OUTFLOW


def _state(rho, u, v, w, p):
    E = p / (GAS.gamma - 1) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E])


def _smooth(xyz, amp=0.1, seed=0):
    """A smooth non-symmetric state with flow across the box (not periodic)."""
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    rho = 1.0 + amp * np.sin(2.1 * x + 0.7 * y) * np.cos(1.3 * z)
    u = 0.3 + amp * np.cos(1.7 * y + 0.4 * z)
    v = amp * np.sin(2.3 * x) * np.sin(0.9 * z + 0.2)
    w = 0.1 + amp * np.cos(1.1 * x + 1.9 * y)
    p = 1.0 / 1.4 + amp * np.sin(0.8 * x - 1.4 * z)
    return uniform_perturbation(_state(rho, u, v, w, p), 1e-3, seed=seed)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# --- reduction to the periodic right-hand sides -----------------------------------------------

@pytest.mark.parametrize("N", [1, 3])
def test_no_boundary_faces_is_the_periodic_rhs(N):
    d = box_disc(2, N)
    q = isentropic_vortex(d.xyz, 0.0)
    q = uniform_perturbation(q, 1e-3, seed=1)
    assert _rel(bd.rhs_euler_bc(d.ref, d.geo, d.conn, q, GAS), rhs_strong(d.ref, d.geo, d.conn, q, GAS)) <= 1e-14
    assert _rel(bd.rhs_ns_bc(d.ref, d.geo, d.conn, q, GAS, MU, PR), rhs_ns(d.ref, d.geo, d.conn, q, GAS, MU, PR)) <= 1e-13


# --- uniform states that satisfy the boundary conditions --------------------------------------

CHANNEL = {(0, 0): INFLOW, (0, 1): OUTFLOW, (1, 0): SLIP, (1, 1): SLIP}


def _freestream_holds(N=2):
    d = bc_disc((2, 2, 1), N, CHANNEL)
    one = np.ones(d.xyz.shape[:-1])
    q = _state(1.2 * one, 2.0 * one, 0.0 * one, 0.3 * one, 0.9 * one)  # tangent to the walls
    q_in = q[:, 0, 0]
    r = bd.rhs_euler_bc(d.ref, d.geo, d.conn, q, GAS, q_in=q_in)
    return np.abs(r).max() <= 1e-12


def _rest_state_holds(N=2):
    d = bc_disc((2, 2, 2), N, {(0, 0): INFLOW, (0, 1): OUTFLOW, (1, 0): NOSLIP, (1, 1): NOSLIP,
                               (2, 0): SLIP, (2, 1): NOSLIP})
    one = np.ones(d.xyz.shape[:-1])
    q = _state(one, 0 * one, 0 * one, 0 * one, 0.8 * one)
    r = bd.rhs_ns_bc(d.ref, d.geo, d.conn, q, GAS, MU, PR, q_in=q[:, 0, 0])
    return np.abs(r).max() <= 1e-12


def test_uniform_states_are_steady():
    assert _freestream_holds()
    assert _rest_state_holds()


# --- conservation in closed boxes -------------------------------------------------------------

def _walls(code):
    return {(a, e): code for a in range(3) for e in (0, 1)}


def _closed_box_conserves(code, ns, N=2):
    d = bc_disc((2, 2, 2), N, _walls(code))
    q = _smooth(d.xyz)
    if ns:
        r = bd.rhs_ns_bc(d.ref, d.geo, d.conn, q, GAS, MU, PR)
    else:
        r = bd.rhs_euler_bc(d.ref, d.geo, d.conn, q, GAS)
    ok = True
    for v in (0, 4):  # mass and total energy
        ok &= abs(d.integrate(r[v])) <= 1e-12 * d.abs_integral(r[v])
    return bool(ok)


def test_closed_boxes_conserve_mass_and_energy():
    assert _closed_box_conserves(SLIP, ns=False)
    assert _closed_box_conserves(SLIP, ns=True)
    assert _closed_box_conserves(NOSLIP, ns=True)


def test_momentum_balance_of_a_slip_wall_box():
    """With slip walls the total momentum changes only through the wall faces, where the
    Lax-Friedrichs flux of the mirror state is (p + (m.n)(u.n) + lambda (m.n)) n: the integral of
    the rhs equals the face integral of minus that, computed here face by face."""
    d = bc_disc((2, 2, 2), 2, _walls(SLIP))
    q = _smooth(d.xyz)
    r = bd.rhs_euler_bc(d.ref, d.geo, d.conn, q, GAS)
    from oracle.euler import face_normals, gather
    n = face_normals(d.geo, d.ref.Nfp)
    qM = gather(q, d.conn.vmapM)
    p, c = GAS.pressure_sound_speed(qM)
    un = (qM[1] * n[0] + qM[2] * n[1] + qM[3] * n[2]) / qM[0]
    lam = np.abs(un) + c
    mn = qM[1] * n[0] + qM[2] * n[1] + qM[3] * n[2]
    # the integral of a lifted face term is exactly its face integral (M LIFT = E)
    from oracle.euler import lift
    wall = d.conn.bc != 0  # the wall face nodes; interior faces cancel in pairs
    flux = np.stack([-(p + mn * un + lam * mn) * n[dd] * wall for dd in range(3)])  # [3][K][4 Nfp]
    want = [d.integrate(lift(d.ref, d.geo, flux[dd][None])[0]) for dd in range(3)]
    got = [d.integrate(r[1 + dd]) for dd in range(3)]
    scale = max(d.abs_integral(r[1 + dd]) for dd in range(3))
    assert np.abs(np.array(got) - np.array(want)).max() <= 1e-12 * scale


# --- slip wall = mirror-image periodic problem -----------------------------------------------

def _mirror_vertices(v):
    m = np.array(v, copy=True)
    m[..., 1] = -m[..., 1]
    m[:, [2, 3]] = m[:, [3, 2]]  # keep the orientation positive
    return m


def _mirror_matches(code=SLIP, N=2):
    """Walls at y = 0 and y = 1 against the doubled box y in [-1, 1] (period 2 in y) holding the
    state and its mirror image: the neighbour trace at a wall node is then the ghost state."""
    n = (2, 2, 1)
    v, per = box_mesh(n, 1.0)
    wall = bc_disc(n, N, {(1, 0): code, (1, 1): code})
    vm = _mirror_vertices(v)
    big = Disc(np.concatenate([v, vm]), (per[0], 2.0, per[2]), N)
    K = v.shape[0]
    xyz = affine_nodes(np.concatenate([v, vm]), big.ref.nodes)
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    ya = np.abs(y)
    rho = 1.0 + 0.1 * np.sin(2 * np.pi * x) * np.cos(1.3 * ya + 0.2)
    u = 0.2 * np.cos(2 * np.pi * z) + 0.1 * ya
    vy = 0.15 * np.sin(np.pi * ya) * np.cos(2 * np.pi * x)
    w = 0.1 * np.sin(2 * np.pi * x + 0.3)
    p = 0.7 + 0.05 * np.cos(2 * np.pi * z) * np.sin(0.9 * ya)
    sgn = np.where(np.arange(2 * K)[:, None] < K, 1.0, -1.0)
    if code == SLIP:  # mirror image: normal (y) velocity odd in y
        q = _state(rho, u, sgn * vy, w, p)
    else:  # the no-slip ghost: all velocity components odd across the wall
        q = _state(rho, sgn * u, sgn * vy, sgn * w, p)
    r_big = rhs_strong(big.ref, big.geo, big.conn, q, GAS)
    r_wall = bd.rhs_euler_bc(wall.ref, wall.geo, wall.conn, q[:, :K], GAS)
    return _rel(r_wall, r_big[:, :K]) <= 1e-12


def test_slip_wall_is_the_mirror_image():
    assert _mirror_matches(SLIP)


def test_noslip_inviscid_ghost_is_the_odd_image():
    assert _mirror_matches(NOSLIP)


# --- supersonic inflow / outflow: an entropy wave leaves the channel ---------------------------

U0 = 2.0  # c = 1 (rho = 1, p = 1/gamma): Mach 2


def _entropy_wave(xyz, t):
    x = xyz[..., 0] - U0 * t
    one = np.ones_like(x)
    rho = 1.0 + 0.2 * np.exp(-((x - 0.45) / 0.12) ** 2)
    return _state(rho, U0 * one, 0 * one, 0 * one, one / 1.4)


def _wave_error(n, N, T=0.15):
    d = bc_disc((n, 1, 1), N, CHANNEL)
    q = _entropy_wave(d.xyz, 0.0)
    q_in = _state(np.array(1.0), np.array(U0), np.array(0.0), np.array(0.0), np.array(1 / 1.4))
    f = lambda u: bd.rhs_euler_bc(d.ref, d.geo, d.conn, u, GAS, q_in=q_in)
    dt0 = 0.3 * (1.0 / n) / ((N + 1) ** 2 * (U0 + 1.0))
    steps = int(np.ceil(T / dt0))
    for _ in range(steps):
        q = lsrk4_step(q, T / steps, f)
    return d.l2(q[0] - _entropy_wave(d.xyz, T)[0])


def _wave_converges(N=2):
    return np.log2(_wave_error(4, N) / _wave_error(8, N)) >= N


def _wave_leaves():
    """At t = 0.3 the bump's centre (0.45 + 0.6) has passed x = 1: at N = 3 on 8 cells the error
    stays at the discretisation level (2.4e-4); an outflow that imposes the inflow state instead
    leaves 4.3e-3."""
    return _wave_error(8, 3, T=0.3) <= 5e-4


def test_entropy_wave_leaves_through_the_outflow():
    """At t = 0.15 the density bump (centre 0.45 -> 0.75, width 0.12) reaches x = 1; the
    boundaries must neither reflect it nor disturb the inflow: error rates >= N at N = 2, 3, and
    the error after the bump has left stays at the discretisation level."""
    assert _wave_converges(2)
    assert np.log2(_wave_error(4, 3) / _wave_error(8, 3)) >= 3
    assert _wave_leaves()


# --- strong = weak -------------------------------------------------------------------------------

def _strong_equals_weak(N=2):
    d = bc_disc((2, 2, 2), N, {(0, 0): INFLOW, (0, 1): OUTFLOW, (1, 0): SLIP, (1, 1): NOSLIP})
    q = _smooth(d.xyz)
    q_in = q[:, 0, 0]
    ok = True
    for fn, args in ((bd.rhs_euler_bc, ()), (bd.rhs_ns_bc, (MU, PR))):
        rs = fn(d.ref, d.geo, d.conn, q, GAS, *args, q_in=q_in, form="strong")
        rw = fn(d.ref, d.geo, d.conn, q, GAS, *args, q_in=q_in, form="weak")
        ok &= _rel(rw, rs) <= 1e-12
    return bool(ok)


def test_strong_equals_weak_with_boundaries():
    assert _strong_equals_weak()


# --- planted mistakes ----------------------------------------------------------------------------

def _all_pins_hold():
    return (_freestream_holds() and _rest_state_holds() and _closed_box_conserves(SLIP, False)
            and _closed_box_conserves(NOSLIP, True) and _mirror_matches(SLIP) and _wave_converges()
            and _wave_leaves())


def _plant(kind):
    orig = bd.exterior_state

    def bad(qM, qPi, bc, n, q_in=None):
        qP = orig(qM, qPi, bc, n, q_in)
        if kind == "no_reflection":  # slip wall copies the interior state
            qP = np.where((bc == SLIP)[None], qM, qP)
        elif kind == "wrong_sign":  # m + 2 (m.n) n
            mn = qM[1] * n[0] + qM[2] * n[1] + qM[3] * n[2]
            for dd in range(3):
                qP[1 + dd] = np.where(bc == SLIP, qM[1 + dd] + 2 * mn * n[dd], qP[1 + dd])
        elif kind == "outflow_as_inflow":
            for v in range(qM.shape[0]):
                qP[v] = np.where(bc == OUTFLOW, q_in[v] if q_in is not None else qP[v], qP[v])
        return qP
    return bad


@pytest.mark.parametrize("kind", ["no_reflection", "wrong_sign", "outflow_as_inflow"])
def test_planted_ghost_mistake_fails_a_pin(kind, monkeypatch):
    monkeypatch.setattr(bd, "exterior_state", _plant(kind))
    assert not _all_pins_hold()


def test_planted_heat_leak_fails_a_pin(monkeypatch):
    """No-slip wall without the adiabatic condition (Q+ = Q-): energy leaks through the walls."""
    orig = bd.rhs_ns_bc
    import oracle.boundary as mod

    def leaky(ref, geo, conn, q, gas, mu, Pr, q_in=None, form="strong"):
        bc = conn.bc.copy()
        conn.bc = np.where(bc == NOSLIP, -1, bc)  # code -1: ghost as no-slip, viscous flux copied
        try:
            return orig(ref, geo, conn, q, gas, mu, Pr, q_in=q_in, form=form)
        finally:
            conn.bc = bc
    mono = mod.exterior_state

    def ghost(qM, qPi, bc, n, q_in=None):
        return mono(qM, qPi, np.where(bc == -1, NOSLIP, bc), n, q_in)
    monkeypatch.setattr(mod, "rhs_ns_bc", leaky)
    monkeypatch.setattr(mod, "exterior_state", ghost)
    assert not _closed_box_conserves(NOSLIP, True)
