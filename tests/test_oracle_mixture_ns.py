"""Pins of the mixture Navier-Stokes oracle with species diffusion (oracle/mixture_ns.py): it
reduces to the single-gas Navier-Stokes right-hand side for one species of constant heat
capacity; a binary mixture at rest with equal molar masses diffuses its species (and, with
unequal heat capacities, its enthalpy) as the closed-form Laplacians while mass and momentum
stay at rest; it conserves every variable on periodic meshes and the species equations add up to
the continuity equation.  Planted mistakes must break a pin."""

import numpy as np
import pytest

import oracle.mixture_ns as mns
from oracle.ns import rhs_ns
from oracle.thermo import Nasa7Gas, PerfectGas
from tests._oracle_case import box_disc
from workloads import taylor_green, uniform_perturbation

MU, PR, SC = 0.05, 0.71, 0.6
RU = 8314.462618


def _gas(W, a1, a6=None):
    ns = len(W)
    c = np.zeros((ns, 7))
    c[:, 0] = a1
    if a6 is not None:
        c[:, 5] = a6
    return Nasa7Gas(W=np.array(W, dtype=float), coeffs=c)


def _single_species_reduces(N=2):
    d = box_disc(2, N)
    W = 28.0
    gas = _gas([W], [3.5])
    R = RU / W
    pg = PerfectGas(1.4, R)
    q5 = taylor_green(d.xyz, gamma=1.4, mach=0.3, noise=0.02, seed=2)  # rho ~ 1, c ~ 1 (T ~ 1/(1.4 R))
    q = np.concatenate([q5, q5[0:1]])
    T = pg.temperature(q5)
    r = mns.rhs_ns_mixture(d.ref, d.geo, d.conn, q, gas, T, MU, PR, SC)
    want = rhs_ns(d.ref, d.geo, d.conn, q5, pg, MU, PR)
    scale = np.abs(want).max(axis=(1, 2))
    ok = np.all(np.abs(r[:5] - want).max(axis=(1, 2)) <= 1e-12 * scale)
    return bool(ok and np.abs(r[5] - r[0]).max() <= 1e-12 * scale[0])


def _binary_at_rest(d, a1, T0=800.0, p0=1e5):
    gas = _gas([20.0, 20.0], a1)
    x = d.xyz[..., 0]
    Y1 = 0.5 + 0.2 * np.sin(2 * np.pi * x)
    Y = np.stack([Y1, 1.0 - Y1])
    T = np.full(x.shape, T0)
    rho = p0 / (gas.R_mix(Y) * T)
    q = gas.conserved(rho, np.zeros((3,) + x.shape), Y, T)
    return gas, q, T, Y1, rho


def _species_diffuse(N=3):
    """Equal molar masses and heat capacities, at rest, uniform T and p: only rho Y_1 and rho Y_2
    move, as (mu/Sc) Y_1'' and its negative; BR1's pointwise rate ~ N - 1 (0.45 -> 0.10 at N = 3)."""
    errs, rest = [], []
    for n in (2, 4):
        d = box_disc((n, 1, 1), N)
        gas, q, T, Y1, rho = _binary_at_rest(d, [3.5, 3.5])
        r = mns.rhs_ns_mixture(d.ref, d.geo, d.conn, q, gas, T, MU, PR, SC)
        exact = -(MU / SC) * (2 * np.pi) ** 2 * 0.2 * np.sin(2 * np.pi * d.xyz[..., 0])
        errs.append(d.l2(r[5] - exact) / d.l2(exact))
        # mass, momentum and energy stay at rest up to rounding of p ~ 1e5 and E ~ 2.5e5 times a
        # derivative scale (N + 1)^2 / h < 1e3; the two species move oppositely
        p0, E0 = 1e5, np.abs(q[4]).max()
        rest.append(np.abs(r[0]).max() <= 1e-12 and np.abs(r[1:4]).max() <= 1e-12 * p0 * 1e3
                    and np.abs(r[4]).max() <= 1e-12 * E0 * 1e3
                    and np.abs(r[5] + r[6]).max() <= 1e-9 * np.abs(r[5]).max())
    return all(rest) and np.log2(errs[0] / errs[1]) >= 1.5 and errs[1] < 0.15


def _enthalpy_diffuses(N=3):
    """Unequal heat capacities (a1 = 3.5, 2.5) at uniform T: the energy moves by
    (h_1 - h_2) (mu/Sc) Y_1'' (enthalpy carried by the diffusion fluxes)."""
    errs = []
    for n in (2, 4):
        d = box_disc((n, 1, 1), N)
        gas, q, T, Y1, rho = _binary_at_rest(d, [3.5, 2.5])
        r = mns.rhs_ns_mixture(d.ref, d.geo, d.conn, q, gas, T, MU, PR, SC)
        h = gas.h_species(T)
        exact = (h[0] - h[1]) * (MU / SC) * (-(2 * np.pi) ** 2 * 0.2 * np.sin(2 * np.pi * d.xyz[..., 0]))
        errs.append(d.l2(r[4] - exact) / d.l2(exact))
    return np.log2(errs[0] / errs[1]) >= 1.5 and errs[1] < 0.15


def _random_mixture(d, ns=4, seed=0):
    rng = np.random.default_rng(seed)
    W = rng.uniform(2.0, 40.0, ns)
    c = np.zeros((ns, 7))
    c[:, 0] = rng.uniform(2.5, 4.5, ns)
    c[:, 1] = rng.uniform(0, 1e-3, ns)
    c[:, 5] = rng.uniform(-1e3, 1e3, ns)
    gas = Nasa7Gas(W=W, coeffs=c)
    x, y, z = d.xyz[..., 0], d.xyz[..., 1], d.xyz[..., 2]
    k = 2 * np.pi
    raw = np.stack([1.0 + 0.3 * np.sin(k * (x + i * y) + i) for i in range(ns)])
    Y = raw / raw.sum(axis=0)
    T = 900.0 + 50.0 * np.cos(k * z) * np.sin(k * x)
    vel = np.stack([10 * np.sin(k * y), 5 * np.cos(k * z), 3 * np.sin(k * x)])
    rho = 1e5 / (gas.R_mix(Y) * T)
    return gas, gas.conserved(rho, vel, Y, T), T


def _conserves(N=2):
    d = box_disc(2, N)
    gas, q, T = _random_mixture(d)
    r = mns.rhs_ns_mixture(d.ref, d.geo, d.conn, q, gas, T, MU, PR, SC)
    return all(abs(d.integrate(r[v])) <= 1e-12 * d.abs_integral(r[v]) for v in range(r.shape[0]))


def _species_sum_is_continuity(N=2):
    d = box_disc(2, N)
    gas, q, T = _random_mixture(d, seed=3)
    r = mns.rhs_ns_mixture(d.ref, d.geo, d.conn, q, gas, T, MU, PR, SC)
    return np.abs(r[5:].sum(axis=0) - r[0]).max() <= 1e-10 * np.abs(r[0]).max()


def _all_pins_hold():
    return (_single_species_reduces() and _species_diffuse() and _enthalpy_diffuses() and _conserves()
            and _species_sum_is_continuity())


def test_single_species_reduces_to_navier_stokes():
    assert _single_species_reduces()


@pytest.mark.parametrize("N", [1, 3])
def test_single_species_other_orders(N):
    assert _single_species_reduces(N)


def test_binary_species_diffusion():
    assert _species_diffuse()


def test_binary_enthalpy_diffusion():
    assert _enthalpy_diffuses()


def test_conservation_and_species_sum():
    assert _conserves()
    assert _species_sum_is_continuity()


def _plant(kind):
    orig = mns.viscous_flux_mixture

    def bad(q, T, grad, gas, mu, Pr, Sc):
        Fv = orig(q, T, grad, gas, mu, Pr, Sc)
        if kind == "species_sign":
            Fv[:, 5:] = -Fv[:, 5:]
        elif kind == "no_enthalpy_diffusion":
            rho, vel, Y, _ = gas.split_state(q)
            gY = grad[:, 5:]
            J = -(mu / Sc) * (gY - Y[None] * gY.sum(axis=1)[:, None])
            Fv[:, 4] += np.sum(gas.h_species(T)[None] * J, axis=1)
        elif kind == "no_heat_conduction":
            rho, vel, Y, _ = gas.split_state(q)
            Fv[:, 4] -= (mu * gas.mixture_cp(T, Y) / Pr)[None] * grad[:, 4]
        return Fv
    return bad


@pytest.mark.parametrize("kind", ["species_sign", "no_enthalpy_diffusion", "no_heat_conduction"])
def test_planted_mistake_fails_a_pin(kind, monkeypatch):
    monkeypatch.setattr(mns, "viscous_flux_mixture", _plant(kind))
    assert not _all_pins_hold()
