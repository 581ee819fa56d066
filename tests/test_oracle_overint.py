"""Pins of the tetrahedral over-integration oracle (oracle/overint.py) against what the mathematics
fixes:
* the Stroud rule with q points per direction integrates every monomial of total degree <= 2q - 1
  exactly (exact rational integrals) and misses one of degree 2q; its weights are positive and its
  points interior;
* when the flux is itself a degree-N polynomial (uniform density and velocity), over-integration
  changes nothing: the result is the collocated strong-form right-hand side;
* with rho = 1 and degree-N velocity and pressure the flux has degree <= 2N, so the default rule
  (exact for degree 3N - 1) agrees with a far finer rule, while a rule exact only to degree N
  aliases;
* periodic meshes conserve mass, momentum and energy; a uniform flow tangent to slip walls with a
  matching inflow stays steady;
* the right-hand side of the translating isentropic vortex converges to its exact time derivative
  at order >= N - 0.9 (the same consistency bar as the collocated form);
* Navier-Stokes: with a degree-N convective flux it is the collocated Navier-Stokes right-hand side
  (walls included); periodic boxes conserve mass, momentum and energy and boxes closed by no-slip
  walls mass and energy; the rest state between no-slip walls is steady;
* the artificial-viscosity flux, a degree-N field, integrated on the rule in weak form with its
  central face flux is the collocated strong AV term.
Planted mistakes in the oracle must break at least one pin."""

import dataclasses

import numpy as np
import pytest

import oracle.boundary as bd
import oracle.overint as oi
from oracle.euler import rhs_strong
from oracle.refelem import exponents3, tet_monomial_integral
from oracle.thermo import PerfectGas
from tests._oracle_case import Disc, bc_disc, box_disc
from workloads import box_mesh, isentropic_vortex, uniform_perturbation

GAS = PerfectGas(1.4, 1.0)
SLIP, NOSLIP, INFLOW, OUTFLOW = bd.SLIP_WALL, bd.NOSLIP_WALL, bd.INFLOW, bd.OUTFLOW


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _state(rho, u, v, w, p):
    E = p / (GAS.gamma - 1) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E])


# --- the rule ---------------------------------------------------------------------------------------

def _rule_exact(q):
    pts, w = oi.tet_rule(q)
    worst = 0.0
    for (a, b, c) in exponents3(2 * q - 1):
        want = float(tet_monomial_integral(a, b, c))
        got = np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
        worst = max(worst, abs(got - want))
    miss = abs(np.sum(w * pts[:, 2] ** (2 * q)) - float(tet_monomial_integral(0, 0, 2 * q)))
    return worst <= 1e-14, miss > 1e-10


@pytest.mark.parametrize("q", [1, 2, 3, 5, 6, 8])
def test_rule_is_exact_to_degree_2q_minus_1(q):
    exact, misses = _rule_exact(q)
    assert exact and misses
    pts, w = oi.tet_rule(q)
    assert np.all(w > 0) and abs(w.sum() - 4.0 / 3.0) <= 1e-15
    assert np.all(pts > -1) and np.all(pts.sum(axis=1) < -1)  # strictly inside the tetrahedron


def test_default_points():
    assert [oi.default_points(N) for N in (1, 2, 3, 4)] == [2, 3, 5, 6]


# --- reductions -------------------------------------------------------------------------------------

def _poly_flux_is_collocated(N=3):
    """Uniform rho and u and a degree-N pressure: every flux is a degree-N polynomial in each element
    (the periodic seam only adds jumps, which both forms treat with the same face flux)."""
    d = box_disc(2, N)
    x, y, z = d.xyz[..., 0], d.xyz[..., 1], d.xyz[..., 2]
    one = np.ones_like(x)
    p = 1.0 + 0.1 * (x - 0.5) ** N + 0.05 * y * z
    q = _state(one, 0.3 * one, -0.2 * one, 0.1 * one, p)
    a = oi.rhs_overint(d.ref, d.geo, d.conn, q, GAS)
    b = rhs_strong(d.ref, d.geo, d.conn, q, GAS)
    return _rel(a, b) <= 1e-12


def test_polynomial_flux_reduces_to_the_collocated_rhs():
    assert _poly_flux_is_collocated(2)
    assert _poly_flux_is_collocated(3)


def _exact_integration(N=3):
    """rho = 1 with degree-N velocity and pressure: the mass and momentum fluxes have degree <= 2N
    (integrand 3N - 1, within the default rule), the energy flux degree 3N (integrand 4N - 1,
    within Q = 2N).  Both agree with a 12-point rule where they are exact; Q = N aliases."""
    d = box_disc(2, N)
    x, y, z = d.xyz[..., 0], d.xyz[..., 1], d.xyz[..., 2]
    one = np.ones_like(x)
    u = 0.3 + 0.2 * x ** N - 0.1 * y
    v = -0.2 + 0.15 * y ** (N - 1) * z
    w = 0.1 * x * z
    p = 1.0 + 0.1 * (x * y) ** (N // 2) * z ** (N - 2 * (N // 2))
    q = _state(one, u, v, w, p)
    fine = oi.rhs_overint(d.ref, d.geo, d.conn, q, GAS, Q=12)
    dflt = oi.rhs_overint(d.ref, d.geo, d.conn, q, GAS)
    full = oi.rhs_overint(d.ref, d.geo, d.conn, q, GAS, Q=2 * N)
    coarse = oi.rhs_overint(d.ref, d.geo, d.conn, q, GAS, Q=N)
    return (_rel(dflt[:4], fine[:4]) <= 1e-12 and _rel(full, fine) <= 1e-12
            and _rel(coarse, fine) > 1e-8)


def test_rules_integrate_polynomial_fluxes_exactly():
    assert _exact_integration(2)
    assert _exact_integration(3)


# --- conservation and steady states -------------------------------------------------------------------

def _conserves(N=3):
    d = box_disc(2, N)
    q = uniform_perturbation(isentropic_vortex(d.xyz, 0.0), 1e-2, seed=4)
    r = oi.rhs_overint(d.ref, d.geo, d.conn, q, GAS)
    return all(abs(d.integrate(r[v])) <= 1e-12 * d.abs_integral(r[v]) for v in range(5))


def test_periodic_mesh_conserves():
    assert _conserves(2)
    assert _conserves(3)


def _freestream_holds(N=2):
    d = bc_disc((2, 2, 1), N, {(0, 0): INFLOW, (0, 1): OUTFLOW, (1, 0): SLIP, (1, 1): SLIP})
    one = np.ones(d.xyz.shape[:-1])
    q = _state(1.2 * one, 2.0 * one, 0.0 * one, 0.3 * one, 0.9 * one)
    r = oi.rhs_overint(d.ref, d.geo, d.conn, q, GAS, q_in=q[:, 0, 0])
    scale = np.abs(q).max() * 2.0 * (N + 1) ** 2 / 0.5  # flux size x |D| ~ (N+1)^2 / h
    return np.abs(r).max() <= 1e-13 * scale


def test_uniform_flow_between_walls_is_steady():
    assert _freestream_holds(2)
    assert _freestream_holds(3)


# --- Navier-Stokes ---------------------------------------------------------------------------------------

MU, PR = 2e-2, 0.71
WALLS = {(1, 0): NOSLIP, (1, 1): SLIP}


def _ns_poly_flux_is_collocated(N=3):
    """Uniform rho and u with a degree-N pressure between a no-slip and a slip wall: the convective
    flux is a degree-N polynomial and the viscous one a nodal field, so over-integration gives the
    collocated Navier-Stokes right-hand side."""
    d = bc_disc((2, 2, 2), N, WALLS)
    x, y, z = d.xyz[..., 0], d.xyz[..., 1], d.xyz[..., 2]
    one = np.ones_like(x)
    p = 1.0 + 0.1 * (x - 0.5) ** N + 0.05 * y * z
    q = _state(one, 0.3 * one, -0.2 * one, 0.1 * one, p)
    a = oi.rhs_overint_ns(d.ref, d.geo, d.conn, q, GAS, MU, PR)
    b = bd.rhs_ns_bc(d.ref, d.geo, d.conn, q, GAS, MU, PR)
    return _rel(a, b) <= 1e-12


def test_ns_polynomial_flux_reduces_to_the_collocated_rhs():
    assert _ns_poly_flux_is_collocated(2)
    assert _ns_poly_flux_is_collocated(3)


def _ns_conserves(N=2):
    d = box_disc(2, N)
    q = uniform_perturbation(isentropic_vortex(d.xyz, 0.0), 1e-2, seed=6)
    r = oi.rhs_overint_ns(d.ref, d.geo, d.conn, q, GAS, MU, PR)
    periodic = all(abs(d.integrate(r[v])) <= 1e-12 * d.abs_integral(r[v]) for v in range(5))
    b = bc_disc((2, 2, 2), N, {(a, e): NOSLIP for a in range(3) for e in (0, 1)})
    x, y, z = b.xyz[..., 0], b.xyz[..., 1], b.xyz[..., 2]
    qb = uniform_perturbation(_state(np.ones_like(x), 0.1 * np.sin(3 * y), 0.05 * np.cos(2 * x), 0 * x,
                                     0.8 + 0.05 * z), 1e-3, seed=7)
    rb = oi.rhs_overint_ns(b.ref, b.geo, b.conn, qb, GAS, MU, PR)
    closed = all(abs(b.integrate(rb[v])) <= 1e-12 * b.abs_integral(rb[v]) for v in (0, 4))
    return periodic and closed


def test_ns_conserves_in_periodic_and_closed_boxes():
    assert _ns_conserves(2)


def _ns_rest_holds(N=2):
    d = bc_disc((2, 2, 2), N, {(a, e): NOSLIP for a in range(3) for e in (0, 1)})
    one = np.ones(d.xyz.shape[:-1])
    q = _state(one, 0 * one, 0 * one, 0 * one, 0.8 * one)
    r = oi.rhs_overint_ns(d.ref, d.geo, d.conn, q, GAS, MU, PR)
    return np.abs(r).max() <= 1e-12


def test_ns_rest_state_between_walls_is_steady():
    assert _ns_rest_holds(2)
    assert _ns_rest_holds(3)


# --- the artificial-viscosity flux on the rule ----------------------------------------------------------

def _av_weak_is_strong(N=3):
    """The AV flux sigma = eps grad_h q integrated on the rule in weak form, with the central face
    flux n.(sigma- + sigma+)/2, equals the collocated strong AV term of oracle/av.py (integration by
    parts is exact for the degree-N field sigma)."""
    import oracle.av as av
    from oracle.euler import face_normals, gather, lift, normal_flux
    d = bc_disc((3, 2, 2), N, {(0, 0): INFLOW, (0, 1): OUTFLOW, (1, 0): SLIP, (1, 1): NOSLIP})
    x, y, z = d.xyz[..., 0], d.xyz[..., 1], d.xyz[..., 2]
    q = uniform_perturbation(_state(1.0 + 0.2 * np.sin(3 * x), 0.3 + 0 * x, 0.1 * np.cos(2 * y), 0 * x,
                                    0.9 + 0.1 * z), 1e-2, seed=9)
    q_in = q[:, 0, 0]
    eps = np.linspace(0.0, 0.03, d.K)
    sigma = eps[None, None, :, None] * av.br1_gradient(d.ref, d.geo, d.conn, q, q_in)  # [3][5][K][Np]
    vol = (oi.overint_volume(d.ref, d.geo, q, GAS, 4, Fv=sigma) - oi.overint_volume(d.ref, d.geo, q, GAS, 4))
    n = face_normals(d.geo, d.ref.Nfp)
    sM = np.stack([gather(sigma[k], d.conn.vmapM) for k in range(3)])
    sP = np.stack([gather(sigma[k], d.conn.vmapP) for k in range(3)])
    sP = np.where((d.conn.bc != 0)[None, None], sM, sP)
    weak = vol + lift(d.ref, d.geo, 0.5 * (normal_flux(sM, n) + normal_flux(sP, n)))
    return _rel(weak, av.rhs_av(d.ref, d.geo, d.conn, q, eps, q_in)) <= 1e-11


def test_av_flux_weak_on_the_rule_is_the_strong_term():
    assert _av_weak_is_strong(2)
    assert _av_weak_is_strong(3)


# --- consistency with the vortex ------------------------------------------------------------------

_L, _R = 10.0, 1.0


def _consistency(n, N):
    v, per = box_mesh((n, n, 1), (_L, _L, _L / n))
    d = Disc(v, per, N)
    kw = dict(center=(5.0, 5.0), radius=_R, u_inf=(1.0, 0.0), period=per)
    q = isentropic_vortex(d.xyz, 0.0, **kw)
    dqdt = np.imag(isentropic_vortex(d.xyz, 1e-30j, **kw)) / 1e-30
    return np.linalg.norm(d.l2(oi.rhs_overint(d.ref, d.geo, d.conn, q, GAS) - dqdt))


def _converges(N=2):
    return np.log2(_consistency(8, N) / _consistency(16, N)) >= N - 0.9


@pytest.mark.slow
def test_vortex_consistency_converges():
    assert _converges(2)


# --- planted mistakes -----------------------------------------------------------------------------------

def _all_pins_hold():
    return (_poly_flux_is_collocated(2) and _exact_integration(2) and _exact_integration(3)
            and _conserves(2) and _freestream_holds(2) and _ns_poly_flux_is_collocated(2)
            and _ns_conserves(2) and _ns_rest_holds(2))


def test_pins_hold_unplanted():
    assert _all_pins_hold()


def _uniform_weights(q):
    pts, w = _RULE(q)
    return pts, np.full_like(w, w.sum() / w.size)


_RULE = oi.tet_rule


def _planted_volume_transposed(ref, geo, q, gas, Q, Fv=None):
    """The r and s derivative operators exchanged in the volume term."""
    return _VOLUME(dataclasses.replace(ref, Dr=ref.Ds, Ds=ref.Dr), geo, q, gas, Q, Fv)


def _planted_no_metric(ref, geo, q, gas, Q, Fv=None):
    """The contravariant flux taken as the Cartesian one (dr_a/dx_d dropped)."""
    class Unit:
        def drdx(self):
            K = geo.drdx().shape[2]
            return np.broadcast_to(np.eye(3)[:, :, None], (3, 3, K))
    return _VOLUME(ref, Unit(), q, gas, Q, Fv)


_VOLUME = oi.overint_volume


def _planted_no_viscous_volume(ref, geo, q, gas, Q, Fv=None):
    """The viscous flux left out of the integrand at the points."""
    return _VOLUME(ref, geo, q, gas, Q)


@pytest.mark.parametrize("plant", ["uniform_weights", "transposed", "no_metric", "no_viscous_volume"])
def test_planted_mistake_fails_a_pin(plant, monkeypatch):
    if plant == "uniform_weights":
        monkeypatch.setattr(oi, "tet_rule", _uniform_weights)
    elif plant == "transposed":
        monkeypatch.setattr(oi, "overint_volume", _planted_volume_transposed)
    elif plant == "no_metric":
        monkeypatch.setattr(oi, "overint_volume", _planted_no_metric)
    else:
        monkeypatch.setattr(oi, "overint_volume", _planted_no_viscous_volume)
    assert not _all_pins_hold()
