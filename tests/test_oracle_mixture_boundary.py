"""Pins of the mixture boundary-condition oracle (oracle/boundary.py: rhs_mixture_bc) against what
the mathematics fixes:
* one species of constant heat capacity is a perfect gas: the right-hand side is the perfect-gas
  one of the same (gamma, R), and the species row is the density row;
* the species rows sum to the density row (sum_k Y_k = 1 is kept by every flux and ghost state);
* boxes closed by slip or no-slip walls conserve mass, every species and total energy;
* a wall ghost has the node's internal energy, so the Newton temperature of the ghost state is
  the node's (the reading T+ = T- at walls);
* a slip wall is the mirror-image periodic problem and a no-slip wall the odd-velocity image
  (the periodic mixture right-hand side on the doubled box);
* an inflow face is an interior face whose neighbour holds the constant state q_in at T_in (the
  periodic-face code on a box twice as long);
* uniform states that satisfy the boundary conditions are steady;
* strong = weak form.
Planted mistakes in the oracle must break at least one pin."""

import numpy as np
import pytest

import oracle.boundary as bd
from oracle.euler import rhs_strong
from oracle.geometry import affine_nodes
from oracle.thermo import Nasa7Gas, PerfectGas
from tests._oracle_case import Disc, bc_disc
from workloads import box_mesh
from workloads.gas import seeded_nasa7_mixture
from workloads.mesh import box_face_bc

SLIP, NOSLIP, INFLOW, OUTFLOW = bd.SLIP_WALL, bd.NOSLIP_WALL, bd.INFLOW, bd.OUTFLOW
MIX = seeded_nasa7_mixture(7, seed=5)
GAS = Nasa7Gas(W=MIX.W, coeffs=MIX.coeffs)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _mixture_state(xyz, gas, fold=lambda y: y, seed=0):
    """A smooth non-uniform mixture: T in about [900, 1500] K, 7 species, p near 1 bar, 20 m/s
    flow across the box.  fold(y) replaces y in every field that must be even across y = 0 (the
    mirror pins pass abs); the y velocity is returned separately so a caller can make it odd."""
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    yy = fold(y)
    rng = np.random.default_rng(seed)
    ns = gas.nspecies
    a, b, c = rng.uniform(0.5, 2.5, (3, ns))
    Yr = np.stack([1.0 + 0.4 * np.sin(a[k] * x + b[k] * yy + c[k] * z + k) for k in range(ns)])
    Y = Yr / Yr.sum(axis=0)
    T = 1200.0 + 300.0 * np.sin(1.7 * x + 0.3) * np.cos(1.1 * yy - 0.4 * z)
    p = 1.0e5 * (1.0 + 0.05 * np.cos(2.1 * z + 0.9 * x) * np.sin(0.7 * yy + 0.1))
    rho = p / (gas.R_mix(Y) * T)
    u = 20.0 + 5.0 * np.cos(1.3 * yy + 0.5 * z)
    v = 8.0 * np.sin(2.3 * x + 0.2) * np.sin(0.9 * yy + 0.6)
    w = 6.0 * np.cos(1.1 * x + 1.9 * yy)
    return rho, u, v, w, Y, T


def _conserved(gas, rho, u, v, w, Y, T):
    return gas.conserved(rho, np.stack([u, v, w]), Y, T)


def _inflow_state(gas):
    """q_in and its temperature: a uniform state at 1000 K entering through x = 0."""
    Y = np.linspace(1.0, 2.0, gas.nspecies)
    Y = Y / Y.sum()
    T = 1000.0
    rho = 1.0e5 / (gas.R_mix(Y) * T)
    return gas.conserved(np.array(rho), np.array([30.0, 2.0, -1.0]), Y, np.array(T)), T


def _newton_T(gas, q, T0=1500.0):
    rho, vel, Y, e = gas.split_state(q)
    T, _, ok = gas.newton_temperature(e, Y, np.full(e.shape, T0), tol=1e-9, max_it=100)
    assert ok.all()
    return T


# --- one species of constant heat capacity is the perfect gas --------------------------------

def _one_species_matches(N=2):
    """NASA-7 with a1 = gamma/(gamma-1) and no other term is e = R T/(gamma-1), the perfect gas."""
    g = PerfectGas(1.4, 287.0)
    one = Nasa7Gas(W=np.array([8314.462618 / 287.0]), coeffs=np.array([[3.5, 0, 0, 0, 0, 0, 0]]))
    sides = {(0, 0): INFLOW, (0, 1): OUTFLOW, (1, 0): SLIP, (1, 1): NOSLIP, (2, 0): SLIP, (2, 1): OUTFLOW}
    d = bc_disc((2, 2, 2), N, sides)
    rho, u, v, w, _, T = _mixture_state(d.xyz, GAS)
    p = rho * 287.0 * T
    E = p / 0.4 + 0.5 * rho * (u * u + v * v + w * w)
    q5 = np.stack([rho, rho * u, rho * v, rho * w, E])
    q6 = np.concatenate([q5, rho[None]])
    rin, Tin = 1.1, 1000.0
    qin5 = np.array([rin, rin * 30.0, rin * 2.0, -rin, rin * 287.0 * Tin / 0.4 + 0.5 * rin * (900 + 4 + 1)])
    qin6 = np.concatenate([qin5, [rin]])
    want = bd.rhs_euler_bc(d.ref, d.geo, d.conn, q5, g, q_in=qin5)
    got = bd.rhs_mixture_bc(d.ref, d.geo, d.conn, q6, one, T, q_in=qin6, T_in=Tin)
    return _rel(got[:5], want) <= 1e-13 and _rel(got[5], want[0]) <= 1e-13


def test_one_species_constant_cp_is_the_perfect_gas():
    assert _one_species_matches()


# --- species rows, conservation ------------------------------------------------------------------

def _species_sum_holds(N=2):
    sides = {(0, 0): INFLOW, (0, 1): OUTFLOW, (1, 0): SLIP, (1, 1): NOSLIP}
    d = bc_disc((2, 2, 1), N, sides)
    q = _conserved(GAS, *_mixture_state(d.xyz, GAS))
    q_in, T_in = _inflow_state(GAS)
    r = bd.rhs_mixture_bc(d.ref, d.geo, d.conn, q, GAS, _newton_T(GAS, q), q_in=q_in, T_in=T_in)
    return _rel(r[5:].sum(axis=0), r[0]) <= 1e-12


def test_species_rows_sum_to_the_mass_row():
    assert _species_sum_holds()


def _closed_box_conserves(code, N=2):
    d = bc_disc((2, 2, 2), N, {(a, e): code for a in range(3) for e in (0, 1)})
    q = _conserved(GAS, *_mixture_state(d.xyz, GAS))
    r = bd.rhs_mixture_bc(d.ref, d.geo, d.conn, q, GAS, _newton_T(GAS, q))
    return all(abs(d.integrate(r[v])) <= 1e-12 * d.abs_integral(r[v]) for v in [0, 4] + list(range(5, r.shape[0])))


def test_closed_boxes_conserve_mass_species_and_energy():
    assert _closed_box_conserves(SLIP)
    assert _closed_box_conserves(NOSLIP)


def test_wall_ghosts_keep_the_node_temperature():
    d = bc_disc((2, 1, 1), 2, {(1, 0): SLIP, (1, 1): NOSLIP})
    q = _conserved(GAS, *_mixture_state(d.xyz, GAS))
    T = _newton_T(GAS, q)
    n, qM, qP = bd._traces(d.conn, d.geo, d.ref, q, None)
    wall = d.conn.bc != 0
    from oracle.euler import gather
    TM = gather(T[None], d.conn.vmapM)[0]
    TP = _newton_T(GAS, qP[:, wall])
    assert np.abs(TP - TM[wall]).max() <= 1e-9 * TM.max()
    assert np.abs(qP[:, wall][:4] - qM[:, wall][:4]).max() > 0  # the ghosts do differ from q-


# --- slip wall = mirror image, no-slip wall = odd image ------------------------------------------

def _mirror_vertices(v):
    m = np.array(v, copy=True)
    m[..., 1] = -m[..., 1]
    m[:, [2, 3]] = m[:, [3, 2]]  # keep the orientation positive
    return m


def _mirror_matches(code, N=2):
    """Walls at y = 0 and y = 1 against the doubled box y in [-1, 1] (period 2 in y) holding the
    state and its image: the neighbour trace at a wall node is then the ghost state."""
    n = (2, 2, 1)
    v, per = box_mesh(n, 1.0)
    wall = bc_disc(n, N, {(1, 0): code, (1, 1): code})
    vm = _mirror_vertices(v)
    big = Disc(np.concatenate([v, vm]), (per[0], 2.0, per[2]), wall.N)
    K = v.shape[0]
    xyz = affine_nodes(np.concatenate([v, vm]), big.ref.nodes)
    rho, u, vy, w, Y, T = _mixture_state(xyz, GAS, fold=np.abs)
    sgn = np.where(np.arange(2 * K)[:, None] < K, 1.0, -1.0)
    if code == SLIP:
        q = _conserved(GAS, rho, u, sgn * vy, w, Y, T)
    else:
        q = _conserved(GAS, rho, sgn * u, sgn * vy, sgn * w, Y, T)
    r_big = rhs_strong(big.ref, big.geo, big.conn, q, GAS, T=T)
    r_wall = bd.rhs_mixture_bc(wall.ref, wall.geo, wall.conn, q[:, :K], GAS, T[:K])
    return _rel(r_wall, r_big[:, :K]) <= 1e-12


def test_slip_wall_is_the_mirror_image():
    assert _mirror_matches(SLIP)


def test_noslip_wall_is_the_odd_image():
    assert _mirror_matches(NOSLIP)


# --- inflow = a neighbour holding q_in ------------------------------------------------------------

def _inflow_matches(N=2):
    """The box [0, 1]^3 with inflow at x = 0 against [-1, 1] x [0, 1]^2 whose left half holds q_in
    at T_in: the right half's right-hand side is the same (outflow at x = 1 on both)."""
    n = (2, 2, 1)
    v, per = box_mesh(n, 1.0)
    small = Disc(v, (0.0, per[1], per[2]), N, face_bc=box_face_bc(v, 1.0, sides={(0, 0): INFLOW, (0, 1): OUTFLOW}))
    vl = np.array(v, copy=True)
    vl[..., 0] -= 1.0
    vb = np.concatenate([v, vl])
    bbc = box_face_bc(vb, (2.0, 1.0, 1.0), origin=(-1.0, 0.0, 0.0), sides={(0, 0): OUTFLOW, (0, 1): OUTFLOW})
    big = Disc(vb, (0.0, per[1], per[2]), N, face_bc=bbc)
    K = v.shape[0]
    q = _conserved(GAS, *_mixture_state(small.xyz, GAS))
    T = _newton_T(GAS, q)
    q_in, T_in = _inflow_state(GAS)
    qb = np.concatenate([q, np.broadcast_to(q_in[:, None, None], q.shape)], axis=1)
    Tb = np.concatenate([T, np.full(T.shape, T_in)])
    r_big = bd.rhs_mixture_bc(big.ref, big.geo, big.conn, qb, GAS, Tb)
    r = bd.rhs_mixture_bc(small.ref, small.geo, small.conn, q, GAS, T, q_in=q_in, T_in=T_in)
    return _rel(r, r_big[:, :K]) <= 1e-12


def test_inflow_is_a_neighbour_holding_the_inflow_state():
    assert _inflow_matches()


def test_inflow_temperature_is_the_newton_root():
    q_in, T_in = _inflow_state(GAS)
    assert abs(_newton_T(GAS, q_in[:, None])[0] - T_in) <= 1e-9 * T_in


# --- uniform states, strong = weak ------------------------------------------------------------------

def _freestream_holds(N=2):
    d = bc_disc((2, 2, 1), N, {(0, 0): INFLOW, (0, 1): OUTFLOW, (1, 0): SLIP, (1, 1): SLIP})
    q_in, T_in = _inflow_state(GAS)
    q_in = q_in.copy()
    q_in[2] = 0.0  # tangent to the walls at y = 0, 1
    rho, vel, Y, e = GAS.split_state(q_in)
    q_in[4] = rho * (GAS.mixture_e(np.array(T_in), Y) + 0.5 * np.sum(vel[[0, 2]] ** 2))
    q = np.broadcast_to(q_in[:, None, None], (q_in.shape[0],) + d.xyz.shape[:-1]).copy()
    r = bd.rhs_mixture_bc(d.ref, d.geo, d.conn, q, GAS, np.full(d.xyz.shape[:-1], T_in), q_in=q_in, T_in=T_in)
    scale = np.abs(q).max() * 30.0 / 0.5  # flux / element size
    return np.abs(r).max() <= 1e-12 * scale


def test_uniform_state_is_steady():
    assert _freestream_holds()


def test_strong_equals_weak_with_boundaries():
    sides = {(0, 0): INFLOW, (0, 1): OUTFLOW, (1, 0): SLIP, (1, 1): NOSLIP, (2, 0): NOSLIP, (2, 1): SLIP}
    d = bc_disc((2, 2, 2), 2, sides)
    q = _conserved(GAS, *_mixture_state(d.xyz, GAS))
    T = _newton_T(GAS, q)
    q_in, T_in = _inflow_state(GAS)
    a = bd.rhs_mixture_bc(d.ref, d.geo, d.conn, q, GAS, T, q_in=q_in, T_in=T_in)
    b = bd.rhs_mixture_bc(d.ref, d.geo, d.conn, q, GAS, T, q_in=q_in, T_in=T_in, form="weak")
    assert _rel(a, b) <= 1e-11


# --- planted mistakes --------------------------------------------------------------------------------

def _all_pins_hold():
    return (_one_species_matches() and _species_sum_holds() and _closed_box_conserves(SLIP)
            and _closed_box_conserves(NOSLIP) and _mirror_matches(SLIP) and _mirror_matches(NOSLIP)
            and _inflow_matches() and _freestream_holds())


def test_pins_hold_unplanted():
    assert _all_pins_hold()


def _exterior_species_swapped_at_walls(qM, qP_interior, bc, n, q_in=None):
    """A transposed species index in the wall ghosts (every value stays physical)."""
    qP = _EXTERIOR(qM, qP_interior, bc, n, q_in)
    wall = (bc == SLIP) | (bc == NOSLIP)
    if qM.shape[0] > 6:
        qP[5], qP[6] = np.where(wall, qM[6], qP[5]), np.where(wall, qM[5], qP[6])
    return qP


def _exterior_inflow_species_dropped(qM, qP_interior, bc, n, q_in=None):
    qP = _EXTERIOR(qM, qP_interior, bc, n, q_in)
    for v in range(5, qM.shape[0]):
        qP[v] = np.where(bc == INFLOW, qM[v], qP[v])
    return qP


_EXTERIOR = bd.exterior_state


@pytest.mark.parametrize("plant", ["species_walls", "inflow_species"])
def test_planted_ghost_mistake_fails_a_pin(plant, monkeypatch):
    fn = {"species_walls": _exterior_species_swapped_at_walls,
          "inflow_species": _exterior_inflow_species_dropped}[plant]
    monkeypatch.setattr(bd, "exterior_state", fn)
    assert not _all_pins_hold()


def test_planted_inflow_temperature_mistake_fails_a_pin(monkeypatch):
    """The inflow ghost evaluated at the node's own temperature instead of T_in."""
    real = bd.rhs_mixture_bc

    def planted(ref, geo, conn, q, gas, T, q_in=None, T_in=None, form="strong"):
        if T_in is None:
            return real(ref, geo, conn, q, gas, T, q_in=q_in, T_in=None, form=form)
        from oracle.euler import gather
        TM = gather(T[None], conn.vmapM)[0]
        return real(ref, geo, conn, q, gas, T, q_in=q_in, T_in=np.where(conn.bc == INFLOW, TM, T_in), form=form)

    monkeypatch.setattr(bd, "rhs_mixture_bc", planted)
    assert not _inflow_matches()
