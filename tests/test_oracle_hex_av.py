"""Pins of the hexahedral artificial viscosity (oracle/hex.py: hex_indicator, hex_rhs_av): the
indicator against closed forms (a pure top Legendre mode, Q_{N-1} fields, alpha + beta L_N with
the GLL norms 2 and 2/N: S = beta^2 / (N alpha^2 + beta^2)), and the BR1 operator against zero on
constants, conservation and the discrete energy identity; planted mistakes must break a pin."""

import numpy as np
import pytest

import oracle.hex as hx
from workloads.hexmesh import gll_nodes, hex_box, hex_nodes


def _ref(N):
    return hx.hex_reference(gll_nodes(N))


def _legendre(a, x):
    return np.polynomial.legendre.Legendre.basis(a)(x)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_indicator_closed_forms(N):
    ref = _ref(N)
    x = ref.nodes
    k, j, i = np.meshgrid(x, x, x, indexing="ij")  # node order [k][j][i]
    top = _legendre(N, j)  # a pure top mode along y
    assert abs(hx.hex_indicator(ref, top.reshape(1, -1))[0] - 1.0) <= 1e-13
    if N > 1:
        low = 1.0 + 0.3 * _legendre(N - 1, i) * _legendre(N - 1, k) - 0.2 * _legendre(1, j)
        assert hx.hex_indicator(ref, low.reshape(1, -1))[0] <= 1e-26
    alpha, beta = 1.3, 0.4
    u = alpha + beta * _legendre(N, k)
    want = beta ** 2 / (N * alpha ** 2 + beta ** 2)
    assert abs(hx.hex_indicator(ref, u.reshape(1, -1))[0] - want) <= 1e-13


def _case(N=3, seed=0):
    box = hex_box((3, 2, 2), 1.0)
    ref = _ref(N)
    xyz = hex_nodes(box, ref.nodes)
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    k = 2 * np.pi
    q = np.stack([1 + 0.2 * np.sin(k * x) * np.cos(k * z), 0.3 * np.cos(k * y), 0.1 * np.sin(k * (x + z)),
                  0.05 * np.cos(k * x), 2.5 + 0.3 * np.sin(k * y)])
    q = q + 1e-2 * np.random.default_rng(seed).uniform(-1, 1, q.shape)
    eps = np.random.default_rng(seed + 1).uniform(0, 1e-2, q.shape[1])
    return box, ref, q, eps


def _constant_steady():
    box, ref, q, eps = _case()
    c = np.ones_like(q) * np.array([1.0, 0.2, -0.1, 0.3, 2.0])[:, None, None]
    return np.abs(hx.hex_rhs_av(ref, box, c, eps)).max() <= 1e-13


def _conserves():
    box, ref, q, eps = _case()
    r = hx.hex_rhs_av(ref, box, q, eps)
    return bool(np.all(np.abs(hx.hex_integrate(ref, box, r)) <= 1e-12 * hx.hex_integrate(ref, box, np.abs(r))))


def _energy_identity(N=3):
    """(q, div_h(eps grad_h q)) = -sum_e eps_e ||grad_h q||^2 in the GLL-weighted inner product."""
    box, ref, q, eps = _case(N)
    r = hx.hex_rhs_av(ref, box, q, eps)
    g = hx.hex_gradient_state(ref, box, q)
    lhs = hx.hex_integrate(ref, box, q * r).sum()
    rhs = -sum(hx.hex_integrate(ref, box, eps[None, :, None] * g[d] ** 2).sum() for d in range(3))
    return abs(lhs - rhs) <= 1e-11 * abs(rhs) and rhs < 0


def _all_pins_hold():
    return _constant_steady() and _conserves() and _energy_identity()


def test_av_operator_pins():
    assert _constant_steady()
    assert _conserves()
    assert _energy_identity()


@pytest.mark.parametrize("N", [1, 2, 4])
def test_energy_identity_other_orders(N):
    assert _energy_identity(N)


def test_planted_full_jump_fails(monkeypatch):
    orig = hx.hex_gradient_state

    def bad(ref, box, q, q_in=None):
        g = orig(ref, box, q, q_in)
        N = ref.N
        q5 = np.asarray(q).reshape(q.shape[0], q.shape[1], N + 1, N + 1, N + 1)
        vol = np.stack([(2.0 / box["h"][d]) * hx._along(ref.D, q5, d).reshape(np.shape(q)) for d in range(3)])
        return 2 * g - vol
    monkeypatch.setattr(hx, "hex_gradient_state", bad)
    assert not _all_pins_hold()


def test_planted_sign_fails(monkeypatch):
    orig = hx.hex_rhs_av
    monkeypatch.setattr(hx, "hex_rhs_av", lambda *a, **k: -orig(*a, **k))
    assert not _all_pins_hold()
