"""GPU parity of the artificial viscosity: element viscosities (smoothness indicator + ramp) and
the FP64 right-hand sides with the artificial-viscosity flux, through the C ABI, against the
oracle (oracle/av.py with oracle/boundary.py) at 1e-11; the mixed-precision form with AV at its
bars (right-hand side 1e-4 per field, state after RK4 steps 1e-6 per field)."""

import numpy as np
import pytest

import oracle.av as av
import oracle.boundary as bd
from oracle.lsrk import lsrk4_step
from oracle.thermo import PerfectGas
from tests._gpu import field_err, rel_err, torch_cuda
from tests._oracle_case import bc_disc, box_disc
from workloads import equispaced_tet_nodes

pytestmark = pytest.mark.gpu
TOL = 1e-11
GAS = PerfectGas(1.4, 1.0)
MU, PR = 2e-2, 0.71
EPS0 = 1e-2


def _front(xyz, seed=0):
    """A steep front across x = 0.5 (width 0.04) on a smooth background: the indicator spans zero,
    the ramp and eps0 over the mesh."""
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    th = np.tanh((x - 0.5) / 0.04)
    rho = 1.5 + 0.5 * th + 0.05 * np.sin(2 * np.pi * y)
    u = 0.3 - 0.2 * th
    v = 0.05 * np.cos(2 * np.pi * z)
    w = 0.02 * np.sin(2 * np.pi * x)
    p = 1.2 + 0.4 * th
    E = p / 0.4 + 0.5 * rho * (u * u + v * v + w * w)
    q = np.stack([rho, rho * u, rho * v, rho * w, E])
    return q + 1e-4 * np.random.default_rng(seed).uniform(-1, 1, q.shape)


def _thresholds(d, q):
    """s0 and kappa placed within the upper spread of the state's indicator, so that the
    elements fall in all three regimes of the ramp."""
    s = np.log10(av.smoothness_indicator(d.ref, q[0]))
    s0 = np.percentile(s, 80)
    return s0, 0.4 * (s.max() - s0)


def _setup(d, N, viscous, q_in=None):
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    mesh = dg.Mesh(d.vertices, d.period, N, equispaced_tet_nodes(N), face_bc=d.face_bc)
    if q_in is not None:
        mesh.set_inflow(q_in)
    s0, kappa = _thresholds(d, _front(d.xyz))
    mesh.set_av(EPS0, s0, kappa)
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=MU if viscous else 0.0, Pr=PR)
    return torch, dg, mesh, gas, (s0, kappa)


def _want(d, q, viscous, th, q_in=None):
    eps = av.element_viscosity(d.ref, q, EPS0, th[0], th[1])
    base = (bd.rhs_ns_bc(d.ref, d.geo, d.conn, q, GAS, MU, PR, q_in=q_in) if viscous
            else bd.rhs_euler_bc(d.ref, d.geo, d.conn, q, GAS, q_in=q_in))
    return base + av.rhs_av(d.ref, d.geo, d.conn, q, eps, q_in=q_in)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_element_viscosity(N):
    d = box_disc((4, 2, 2), N)
    torch, dg, mesh, gas, s0 = _setup(d, N, False)
    q0 = _front(d.xyz)
    eps = torch.empty(d.K, dtype=torch.float64, device="cuda")
    mesh.av_viscosity(torch.tensor(q0, device="cuda"), eps)
    want = av.element_viscosity(d.ref, q0, EPS0, s0[0], s0[1])
    got = eps.cpu().numpy()
    assert np.abs(got - want).max() <= 1e-11 * EPS0
    assert (want == 0).any() and (want == EPS0).any() and ((want > 0) & (want < EPS0)).any()


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_rhs_with_artificial_viscosity(N, viscous):
    d = box_disc((4, 2, 2), N)
    torch, dg, mesh, gas, s0 = _setup(d, N, viscous)
    q0 = _front(d.xyz)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs)
    assert rel_err(rhs.cpu().numpy(), _want(d, q0, viscous, s0)) <= TOL
    assert mesh.status() == 0


@pytest.mark.parametrize("viscous", [False, True])
def test_rhs_with_artificial_viscosity_and_boundaries(viscous):
    sides = {(0, 0): bd.INFLOW, (0, 1): bd.OUTFLOW, (1, 0): bd.SLIP_WALL, (1, 1): bd.NOSLIP_WALL}
    d = bc_disc((4, 2, 2), 2, sides)
    q0 = _front(d.xyz)
    q_in = q0[:, 0, 0].copy()
    torch, dg, mesh, gas, s0 = _setup(d, 2, viscous, q_in=q_in)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs)
    assert rel_err(rhs.cpu().numpy(), _want(d, q0, viscous, s0, q_in=q_in)) <= TOL


def test_two_rk4_steps_with_artificial_viscosity():
    d = box_disc((4, 2, 2), 2)
    torch, dg, mesh, gas, s0 = _setup(d, 2, False)
    q0 = _front(d.xyz, seed=4)
    dt = 5e-4
    q = torch.tensor(q0, device="cuda")
    dg.lsrk4_step(mesh, gas, q, dt, steps=2)
    f = lambda u: _want(d, u, False, s0)
    want = lsrk4_step(lsrk4_step(q0, dt, f), dt, f)
    assert rel_err(q.cpu().numpy() - q0, want - q0) <= TOL


def test_artificial_viscosity_off_and_rejections():
    """A mixture with AV is refused before any launch; AV off gives the plain right-hand side."""
    from workloads.gas import seeded_nasa7_mixture
    d = box_disc(2, 2)
    torch, dg, mesh, gas, s0 = _setup(d, 2, False)
    from paper_2512_17101_gb300 import capi
    q0 = _front(d.xyz)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    mix = seeded_nasa7_mixture(2, seed=0)
    mgas = dg.Gas(model="nasa7", W=mix.W, nasa7=mix.coeffs)
    qm = torch.zeros((7,) + tuple(q.shape[1:]), device="cuda", dtype=torch.float64)
    T = torch.full(tuple(q.shape[1:]), 1000.0, device="cuda", dtype=torch.float64)
    with pytest.raises(capi.DGError):
        dg.dg_rhs(mesh, mgas, qm, torch.empty_like(qm), T_io=T)
    mesh.set_av(0.0)
    dg.dg_rhs(mesh, gas, q, rhs)
    assert rel_err(rhs.cpu().numpy(), bd.rhs_euler_bc(d.ref, d.geo, d.conn, q0, GAS)) <= TOL
    with pytest.raises(capi.DGError):
        mesh.set_av(1e-2, 0.0, -1.0)


# --- the mixed-precision form with artificial viscosity ------------------------------------------

MIXED_RHS_TOL = 1e-4  # per field, as for the mixed form without AV (tests/test_gpu_mixed.py)


def _mixed(dg):
    from paper_2512_17101_gb300 import capi
    return dg._opts(precision=capi.DG_PREC_MIXED)


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_mixed_rhs_with_artificial_viscosity(N, viscous):
    d = box_disc((4, 2, 2), N)
    torch, dg, mesh, gas, s0 = _setup(d, N, viscous)
    q0 = _front(d.xyz)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs, opts=_mixed(dg))
    err = field_err(rhs.cpu().numpy(), _want(d, q0, viscous, s0))
    assert err <= MIXED_RHS_TOL, err
    assert mesh.status() == 0


@pytest.mark.parametrize("viscous", [False, True])
def test_mixed_rhs_with_artificial_viscosity_and_boundaries(viscous):
    sides = {(0, 0): bd.INFLOW, (0, 1): bd.OUTFLOW, (1, 0): bd.SLIP_WALL, (1, 1): bd.NOSLIP_WALL}
    d = bc_disc((4, 2, 2), 3, sides)
    q0 = _front(d.xyz)
    q_in = q0[:, 0, 0].copy()
    torch, dg, mesh, gas, s0 = _setup(d, 3, viscous, q_in=q_in)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs, opts=_mixed(dg))
    err = field_err(rhs.cpu().numpy(), _want(d, q0, viscous, s0, q_in=q_in))
    assert err <= MIXED_RHS_TOL, err


@pytest.mark.parametrize("N", [2, 3])
def test_mixed_rk4_steps_with_artificial_viscosity(N):
    """Two RK4 steps of the mixed form with AV against the oracle: state error <= 1e-6 per field."""
    d = box_disc((4, 2, 2), N)
    torch, dg, mesh, gas, s0 = _setup(d, N, True)
    q0 = _front(d.xyz, seed=4)
    dt = 2e-4
    q = torch.tensor(q0, device="cuda")
    dg.lsrk4_step(mesh, gas, q, dt, steps=2, opts=_mixed(dg))
    f = lambda u: _want(d, u, True, s0)
    want = lsrk4_step(lsrk4_step(q0, dt, f), dt, f)
    err = field_err(q.cpu().numpy(), want)
    assert err <= 1e-6, err
    assert mesh.status() == 0


@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("regime", ["none", "all"])
def test_av_element_list_extremes(regime, mixed):
    """Thresholds under which no element and every element has eps > 0: the flux pass's element
    list is empty or holds all K elements; the right-hand sides match the oracle."""
    from paper_2512_17101_gb300 import capi
    d = box_disc((4, 2, 2), 3)
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    mesh = dg.Mesh(d.vertices, d.period, 3, equispaced_tet_nodes(3))
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=MU, Pr=PR)
    q0 = _front(d.xyz)
    th = (50.0, 1.0) if regime == "none" else (-50.0, 1.0)
    mesh.set_av(EPS0, th[0], th[1])
    eps = av.element_viscosity(d.ref, q0, EPS0, th[0], th[1])
    assert (eps == 0).all() if regime == "none" else (eps == EPS0).all()
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    opts = dg._opts(precision=capi.DG_PREC_MIXED) if mixed else None
    for _ in range(2):  # twice: the list is rebuilt, not appended to
        dg.dg_rhs(mesh, gas, q, rhs, opts=opts)
    want = _want(d, q0, True, th)
    if mixed:
        assert field_err(rhs.cpu().numpy(), want) <= MIXED_RHS_TOL
    else:
        assert rel_err(rhs.cpu().numpy(), want) <= TOL
    assert mesh.status() == 0
