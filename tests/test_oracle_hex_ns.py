"""Pins of the hexahedral Navier-Stokes oracle (oracle/hex.py, hex_gradient / hex_rhs_ns): it
reduces to the Euler right-hand side at zero viscosity, leaves a uniform state at rest, conserves
every variable on periodic boxes, and its viscous part converges to the closed forms of shear,
compression and heat conduction; planted mistakes must break a pin."""

import numpy as np
import pytest

import oracle.hex as hx
from oracle.thermo import PerfectGas
from workloads import isentropic_vortex, uniform_perturbation
from workloads.hexmesh import gll_nodes, hex_box, hex_nodes

GAS = PerfectGas(1.4, 1.0)
MU, PR = 0.05, 0.71
KAPPA = MU * GAS.cp / PR
K2PI = 2 * np.pi


def _state(rho, u, v, w, p):
    E = p / (GAS.gamma - 1) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E])


def _case(n, N, L=1.0):
    box = hex_box(n, L)
    x = gll_nodes(N)
    return box, hx.hex_reference(x), hex_nodes(box, x)


def _zero_viscosity_is_euler(N=3):
    box, ref, xyz = _case((3, 2, 2), N)
    q = uniform_perturbation(isentropic_vortex(xyz, 0.0, center=(0.45, 0.55), radius=0.15, period=box["L"]), 1e-2)
    return np.abs(hx.hex_rhs_ns(ref, box, q, GAS, 0.0, PR) - hx.hex_rhs_strong(ref, box, q, GAS)).max() == 0.0


def _rest_is_steady(N=3):
    box, ref, xyz = _case((2, 2, 2), N)
    one = np.ones(xyz.shape[:-1])
    q = _state(1.1 * one, 0 * one, 0 * one, 0 * one, 0.9 * one)
    return np.abs(hx.hex_rhs_ns(ref, box, q, GAS, MU, PR)).max() <= 1e-13


def _conserves(N=3):
    box, ref, xyz = _case((3, 2, 2), N)
    q = uniform_perturbation(isentropic_vortex(xyz, 0.0, center=(0.45, 0.55), radius=0.15, period=box["L"]), 1e-2)
    r = hx.hex_rhs_ns(ref, box, q, GAS, MU, PR)
    tot, scale = hx.hex_integrate(ref, box, r), hx.hex_integrate(ref, box, np.abs(r))
    return bool(np.all(np.abs(tot) <= 1e-12 * scale))


def _closed_form(name, xyz):
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    one, zero = np.ones_like(x), np.zeros_like(x)
    A, B, k = 0.2, 0.1, K2PI
    if name == "shear_y":  # u = A sin(ky): tau_xy = mu u'
        u, du, d2u = A * np.sin(k * y), A * k * np.cos(k * y), -A * k * k * np.sin(k * y)
        return _state(one, u, zero, zero, one), (1, MU * d2u)
    if name == "compress_x":  # u = A sin(kx): tau_xx = 4/3 mu u'
        u, d2u = A * np.sin(k * x), -A * k * k * np.sin(k * x)
        return _state(one, u, zero, zero, one), (1, 4 / 3 * MU * d2u)
    if name == "heat_z":  # at rest, T = p / rho = 1 + B sin(kz)
        p = 1 + B * np.sin(k * z)
        return _state(one, zero, zero, zero, p), (4, -KAPPA * B * k * k * np.sin(k * z))
    raise ValueError(name)


def _viscous_converges(name, N=3):
    errs = []
    for n in (4, 8):
        box, ref, xyz = _case((n, n, n) if name == "heat_z" else (n, n, 1), N,
                              1.0 if name == "heat_z" else (1.0, 1.0, 1.0 / n))
        q, (v, exact) = _closed_form(name, xyz)
        r = hx.hex_rhs_ns(ref, box, q, GAS, MU, PR) - hx.hex_rhs_strong(ref, box, q, GAS)
        errs.append(np.sqrt(hx.hex_integrate(ref, box, ((r[v] - exact) ** 2)[None])[0]
                            / hx.hex_integrate(ref, box, (exact ** 2)[None])[0]))
    return np.log2(errs[0] / errs[1]) >= 2.0 and errs[1] < 0.05


def _gradient_integrates_to_zero(N=2):
    """The central flux makes the discrete gradient of any periodic field, continuous or not,
    integrate to zero over the box (a jump weight other than 1/2 leaves sum (1 - 2a)[w] n)."""
    box, ref, xyz = _case((3, 2, 2), N)
    w = np.random.default_rng(5).uniform(-1, 1, (2,) + xyz.shape[:-1])
    g = hx.hex_gradient(ref, box, w)
    return all(np.abs(hx.hex_integrate(ref, box, g[d])).max() <= 1e-12 * hx.hex_integrate(ref, box, np.abs(g[d])).max()
               for d in range(3))


def _all_pins_hold():
    return (_zero_viscosity_is_euler() and _rest_is_steady() and _conserves() and _gradient_integrates_to_zero()
            and all(_viscous_converges(c) for c in ("shear_y", "compress_x")))


def test_zero_viscosity_is_euler():
    assert _zero_viscosity_is_euler()


def test_rest_and_conservation():
    assert _rest_is_steady()
    assert _conserves()
    assert _gradient_integrates_to_zero()


@pytest.mark.parametrize("name", ["shear_y", "compress_x", "heat_z"])
def test_viscous_terms_converge_to_closed_forms(name):
    """Rates >= 2 at N = 3 (shear: 0.053 -> 0.0071 from 4 to 8 cells)."""
    assert _viscous_converges(name)


@pytest.mark.parametrize("N", [1, 2, 4])
def test_conservation_other_orders(N):
    assert _conserves(N) and _rest_is_steady(N)


# --- walls -----------------------------------------------------------------------------------------

import oracle.boundary as bd  # noqa: E402


def _ns_mirror_matches(code, N=3):
    """Navier-Stokes walls at y = 0 and y = 1 against the doubled periodic box holding the folded
    state: the slip wall (shear-free, adiabatic) is the even image, the no-slip wall's inviscid and
    gradient ghosts are the odd image; for the no-slip wall the viscous ghost differs from the odd
    image, so only the slip wall is compared in full."""
    box = hex_box((2, 2, 2), 1.0)
    box["bc"] = ((0, 0), (code, code), (0, 0))
    x = gll_nodes(N)
    ref = hx.hex_reference(x)
    xyz = hex_nodes(box, x)
    big = hex_box((2, 4, 2), (1.0, 2.0, 1.0))
    xyz2 = hex_nodes(big, x)
    e = np.arange(16)
    lower = ((e // 2) % 4) < 2

    def folded(pts, upper):
        xx, y, z = pts[..., 0], pts[..., 1], pts[..., 2]
        yf = np.where(upper[:, None], 2.0 - y, y)
        s = np.where(upper[:, None], -1.0, 1.0)
        rho = 1.0 + 0.1 * np.sin(2 * np.pi * xx) * np.cos(1.3 * yf + 0.2)
        u = 0.2 * np.cos(2 * np.pi * z) + 0.1 * yf
        v = 0.15 * np.sin(np.pi * yf) * np.cos(2 * np.pi * xx)
        w = 0.1 * np.sin(2 * np.pi * xx + 0.3)
        p = 0.7 + 0.05 * np.cos(2 * np.pi * z) * np.sin(0.9 * yf)
        return _state(rho, u, s * v, w, p)

    r_wall = hx.hex_rhs_ns(ref, box, folded(xyz, np.zeros(8, dtype=bool)), GAS, MU, PR)
    r_big = hx.hex_rhs_ns(ref, big, folded(xyz2, ~lower), GAS, MU, PR)
    return np.abs(r_wall - r_big[:, lower]).max() <= 1e-11 * np.abs(r_big).max()


def _noslip_box_conserves(N=3):
    box = hex_box((2, 2, 2), 1.0)
    box["bc"] = ((bd.NOSLIP_WALL,) * 2, (bd.NOSLIP_WALL,) * 2, (bd.SLIP_WALL,) * 2)
    x = gll_nodes(N)
    ref = hx.hex_reference(x)
    xyz = hex_nodes(box, x)
    q = uniform_perturbation(isentropic_vortex(xyz, 0.0, center=(0.45, 0.55), radius=0.15), 1e-2)
    r = hx.hex_rhs_ns(ref, box, q, GAS, MU, PR)
    tot, scale = hx.hex_integrate(ref, box, r), hx.hex_integrate(ref, box, np.abs(r))
    return abs(tot[0]) <= 1e-12 * scale[0] and abs(tot[4]) <= 1e-12 * scale[4]


def test_slip_wall_is_the_mirror_image_with_viscosity():
    assert _ns_mirror_matches(bd.SLIP_WALL)


def test_walled_box_conserves_mass_and_energy():
    """Adiabatic no-slip and slip walls: no mass and no energy (heat or work) cross them."""
    assert _noslip_box_conserves()


def test_planted_heat_leak_at_walls_fails(monkeypatch):
    orig = hx.hex_rhs_ns

    def leaky(ref, box, q, gas, mu, Pr, q_in=None):  # walls that pass the interior energy flux
        bc = box["bc"]
        box2 = dict(box)
        box2["bc"] = tuple(tuple(bd.OUTFLOW if c in (bd.SLIP_WALL, bd.NOSLIP_WALL) else c for c in ax) for ax in bc)
        # inviscid and gradient ghosts of the walls kept, viscous exterior flux = interior one:
        # the difference of the two right-hand sides is the walls' viscous correction
        r_out = orig(ref, box2, q, gas, mu, Pr, q_in)
        r_out_inv = orig(ref, box2, q, gas, 0.0, Pr, q_in)
        r_wall_inv = orig(ref, box, q, gas, 0.0, Pr, q_in)
        return r_wall_inv + (r_out - r_out_inv)
    monkeypatch.setattr(hx, "hex_rhs_ns", leaky)
    assert not _noslip_box_conserves()


def test_planted_full_jump_fails(monkeypatch):
    orig = hx.hex_gradient

    def bad(ref, box, w, *rest):  # jump (w+ - w-) instead of half of it
        g = orig(ref, box, w, *rest)
        N = ref.N
        vol = np.stack([(2.0 / box["h"][d]) * hx._along(ref.D, w.reshape(w.shape[0], w.shape[1], N + 1, N + 1, N + 1),
                                                        d).reshape(w.shape) for d in range(3)])
        return 2 * g - vol
    monkeypatch.setattr(hx, "hex_gradient", bad)
    assert not _all_pins_hold()


def test_planted_viscous_face_sign_fails(monkeypatch):
    orig_ns = hx.hex_rhs_ns

    def bad(ref, box, q, gas, mu, Pr):  # the viscous face term -n.(Fv- - Fv+)/2 with its sign flipped
        return orig_ns(ref, box, q, gas, mu, Pr) + _face_only(ref, box, q, gas, mu, Pr)
    monkeypatch.setattr(hx, "hex_rhs_ns", bad)
    assert not _all_pins_hold()


def _face_only(ref, box, q, gas, mu, Pr):
    """Lifted +n.(Fv- - Fv+) at the face nodes: minus twice the viscous face term."""
    from oracle.ns import viscous_flux
    N = ref.N
    T = gas.temperature(q)
    w = np.stack([q[0], q[1], q[2], q[3], T])
    Fv = viscous_flux(q, T, hx.hex_gradient(ref, box, w), mu, mu * gas.cp / Pr)
    Fv5 = Fv.reshape((3, 5, q.shape[1], N + 1, N + 1, N + 1))
    out = np.zeros((5, q.shape[1], N + 1, N + 1, N + 1))
    for d in range(3):
        for end in (0, 1):
            nd = -1.0 if end == 0 else 1.0
            nb = hx._neighbour(box, d, -1 if end == 0 else 1)
            sel = hx._face_slices(N, d, end)
            lift = (2.0 / box["h"][d]) / ref.w[0 if end == 0 else N]
            out[sel] += lift * nd * (Fv5[d][sel] - Fv5[d][:, nb][hx._face_slices(N, d, 1 - end)])
    return out.reshape(q.shape)
