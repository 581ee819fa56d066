"""Pins of the viscous-mixture boundary oracle (oracle/mixture_ns.py: rhs_ns_mixture_bc) against
what the mathematics fixes:
* without boundary faces it is the periodic viscous-mixture right-hand side;
* one species of constant heat capacity is the perfect gas: the result is the single-gas
  Navier-Stokes right-hand side with the same walls and inflow, and the species row is the
  density row (the corrected diffusion flux of one species vanishes);
* the species rows sum to the density row;
* boxes closed by no-slip or slip walls conserve mass, every species and total energy (adiabatic,
  impermeable walls);
* a mixture at rest with uniform temperature, composition and pressure between no-slip walls is
  steady.
The viscosity is large enough that the viscous, heat and diffusion terms are of the size of the
convective ones, so a mistake in them shows at the pins' tolerances.  Planted mistakes in the
oracle must break at least one pin."""

import numpy as np
import pytest

import oracle.boundary as bd
import oracle.mixture_ns as mns
from oracle.thermo import Nasa7Gas, PerfectGas
from tests._oracle_case import bc_disc, box_disc
from tests.test_oracle_mixture_boundary import GAS, _conserved, _inflow_state, _mixture_state

SLIP, NOSLIP, INFLOW, OUTFLOW = bd.SLIP_WALL, bd.NOSLIP_WALL, bd.INFLOW, bd.OUTFLOW
MU, PR, SC = 5.0, 0.71, 0.7
SIDES = {(0, 0): INFLOW, (0, 1): OUTFLOW, (1, 0): SLIP, (1, 1): NOSLIP, (2, 0): NOSLIP, (2, 1): SLIP}


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _newton_T(gas, q, T0=1500.0):
    rho, vel, Y, e = gas.split_state(q)
    T, _, ok = gas.newton_temperature(e, Y, np.full(e.shape, T0), tol=1e-9, max_it=100)
    assert ok.all()
    return T


def _periodic_reduction(N=2):
    d = box_disc(2, N)
    q = _conserved(GAS, *_mixture_state(d.xyz, GAS))
    T = _newton_T(GAS, q)
    a = mns.rhs_ns_mixture_bc(d.ref, d.geo, d.conn, q, GAS, T, MU, PR, SC)
    b = mns.rhs_ns_mixture(d.ref, d.geo, d.conn, q, GAS, T, MU, PR, SC)
    return _rel(a, b) <= 1e-13


def test_no_boundary_faces_is_the_periodic_rhs():
    assert _periodic_reduction(2)


def _one_species_matches(N=2):
    """NASA-7 with a1 = gamma/(gamma - 1) and nothing else is the perfect gas of the same R."""
    g = PerfectGas(1.4, 287.0)
    one = Nasa7Gas(W=np.array([8314.462618 / 287.0]), coeffs=np.array([[3.5, 0, 0, 0, 0, 0, 0]]))
    d = bc_disc((2, 2, 2), N, SIDES)
    rho, u, v, w, _, T = _mixture_state(d.xyz, GAS)
    p = rho * 287.0 * T
    q5 = np.stack([rho, rho * u, rho * v, rho * w, p / 0.4 + 0.5 * rho * (u * u + v * v + w * w)])
    q6 = np.concatenate([q5, rho[None]])
    rin, Tin = 1.1, 1000.0
    qin5 = np.array([rin, rin * 30.0, rin * 2.0, -rin, rin * 287.0 * Tin / 0.4 + 0.5 * rin * (900 + 4 + 1)])
    want = bd.rhs_ns_bc(d.ref, d.geo, d.conn, q5, g, MU, PR, q_in=qin5)
    got = mns.rhs_ns_mixture_bc(d.ref, d.geo, d.conn, q6, one, T, MU, PR, SC,
                                q_in=np.concatenate([qin5, [rin]]), T_in=Tin)
    return _rel(got[:5], want) <= 1e-12 and _rel(got[5], want[0]) <= 1e-12


def test_one_species_constant_cp_is_the_perfect_gas():
    assert _one_species_matches(2)
    assert _one_species_matches(3)


def _species_sum_holds(N=2):
    d = bc_disc((2, 2, 1), N, SIDES)
    q = _conserved(GAS, *_mixture_state(d.xyz, GAS))
    q_in, T_in = _inflow_state(GAS)
    r = mns.rhs_ns_mixture_bc(d.ref, d.geo, d.conn, q, GAS, _newton_T(GAS, q), MU, PR, SC, q_in=q_in, T_in=T_in)
    return _rel(r[5:].sum(axis=0), r[0]) <= 1e-12


def test_species_rows_sum_to_the_mass_row():
    assert _species_sum_holds()


def _closed_box_conserves(code, N=2):
    d = bc_disc((2, 2, 2), N, {(a, e): code for a in range(3) for e in (0, 1)})
    q = _conserved(GAS, *_mixture_state(d.xyz, GAS))
    r = mns.rhs_ns_mixture_bc(d.ref, d.geo, d.conn, q, GAS, _newton_T(GAS, q), MU, PR, SC)
    return all(abs(d.integrate(r[v])) <= 1e-12 * d.abs_integral(r[v]) for v in [0, 4] + list(range(5, r.shape[0])))


def test_closed_boxes_conserve_mass_species_and_energy():
    assert _closed_box_conserves(NOSLIP)
    assert _closed_box_conserves(SLIP)


def _rest_holds(N=2):
    d = bc_disc((2, 2, 2), N, {(a, e): NOSLIP for a in range(3) for e in (0, 1)})
    one = np.ones(d.xyz.shape[:-1])
    Y = np.linspace(1.0, 2.0, GAS.nspecies)[:, None, None] * one[None]
    Y = Y / Y.sum(axis=0)
    T = 1100.0 * one
    rho = 1.0e5 / (GAS.R_mix(Y) * T)
    q = GAS.conserved(rho, np.zeros((3,) + one.shape), Y, T)
    r = mns.rhs_ns_mixture_bc(d.ref, d.geo, d.conn, q, GAS, T, MU, PR, SC)
    # rounding scales: the state's size x |D| ~ (N+1)^2 / h, and the heat conduction of the uniform
    # temperature, kappa T |D|^2
    kappa = MU * GAS.mixture_cp(T, Y).max() / PR
    scale = np.abs(q).max() * (N + 1) ** 2 / 0.5 + kappa * 1100.0 * ((N + 1) ** 2 / 0.5) ** 2
    return np.abs(r).max() <= 1e-13 * scale


def test_rest_state_between_walls_is_steady():
    assert _rest_holds(2)
    assert _rest_holds(3)


# --- planted mistakes ---------------------------------------------------------------------------------

def _all_pins_hold():
    return (_periodic_reduction() and _one_species_matches() and _species_sum_holds()
            and _closed_box_conserves(NOSLIP) and _closed_box_conserves(SLIP) and _rest_holds())


def test_pins_hold_unplanted():
    assert _all_pins_hold()


_EXTERIOR = mns.exterior_viscous


def _permeable_walls(nvM, nvP, bc, n):
    """Walls that let species diffuse through (s+ = s-)."""
    out = _EXTERIOR(nvM, nvP, bc, n)
    wall = (bc == SLIP) | (bc == NOSLIP)
    for v in range(5, nvM.shape[0]):
        out[v] = np.where(wall, nvM[v], out[v])
    return out


def _conducting_walls(nvM, nvP, bc, n):
    """Walls that let heat through (e+ = e-)."""
    out = _EXTERIOR(nvM, nvP, bc, n)
    wall = (bc == SLIP) | (bc == NOSLIP)
    out[4] = np.where(wall, nvM[4], out[4])
    return out


def _slip_takes_the_full_traction(nvM, nvP, bc, n):
    out = _EXTERIOR(nvM, nvP, bc, n)
    for i in range(3):
        out[1 + i] = np.where(bc == SLIP, nvM[1 + i], out[1 + i])
    return out


@pytest.mark.parametrize("plant", [_permeable_walls, _conducting_walls, _slip_takes_the_full_traction])
def test_planted_wall_mistake_fails_a_pin(plant, monkeypatch):
    monkeypatch.setattr(mns, "exterior_viscous", plant)
    assert not _all_pins_hold()
