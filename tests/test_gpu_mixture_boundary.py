"""GPU parity of the mixture right-hand side on meshes with boundary faces (slip and no-slip walls,
inflow, outflow): 7 NASA-7 species, through the C ABI, against the mixture boundary oracle
(oracle/boundary.py: rhs_mixture_bc) with the oracle's own Newton temperatures.  FP64 form at
1e-11 per conserved variable; the mixed-precision form at its right-hand-side bar (1e-4 per field)
and its state bar after RK4 steps (1e-6 per field)."""

import numpy as np
import pytest

import oracle.boundary as bd
from oracle.lsrk import lsrk4_step
from tests._gpu import field_err, rel_err, torch_cuda
from tests._oracle_case import bc_disc
from tests.test_oracle_mixture_boundary import GAS, MIX, _conserved, _inflow_state, _mixture_state
from workloads import equispaced_tet_nodes

pytestmark = pytest.mark.gpu
TOL = 1e-11
MIXED_RHS_TOL = 1e-4
MIXED_STATE_TOL = 1e-6
SLIP, NOSLIP, INFLOW, OUTFLOW = bd.SLIP_WALL, bd.NOSLIP_WALL, bd.INFLOW, bd.OUTFLOW
T_SEED = 1500.0

SIDES = {
    "slip_y": {(1, 0): SLIP, (1, 1): SLIP},
    "noslip_y_slip_z": {(1, 0): NOSLIP, (1, 1): NOSLIP, (2, 0): SLIP, (2, 1): SLIP},
    "in_out_x_walls_y": {(0, 0): INFLOW, (0, 1): OUTFLOW, (1, 0): SLIP, (1, 1): NOSLIP},
    "closed_box": {(a, e): NOSLIP for a in range(3) for e in (0, 1)},
}
Q_IN, T_IN = _inflow_state(GAS)


def _setup(n, N, sides, mu=0.0):
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    d = bc_disc(n, N, sides)
    mesh = dg.Mesh(d.vertices, d.period, N, equispaced_tet_nodes(N), face_bc=d.face_bc)
    if any(c == INFLOW for c in sides.values()):
        mesh.set_inflow(Q_IN)
    gas = dg.Gas(model="nasa7", W=MIX.W, nasa7=MIX.coeffs, newton_tol=1e-10, newton_max_it=50, mu=mu)
    return torch, dg, d, mesh, gas


def _newton(q):
    rho, vel, Y, e = GAS.split_state(q)
    T, _, ok = GAS.newton_temperature(e, Y, np.full(e.shape, T_SEED))
    assert ok.all()
    return T


def _want(d, q):
    return bd.rhs_mixture_bc(d.ref, d.geo, d.conn, q, GAS, _newton(q), q_in=Q_IN, T_in=T_IN)


def _mixed(dg):
    from paper_2512_17101_gb300 import capi
    return dg._opts(precision=capi.DG_PREC_MIXED)


@pytest.mark.parametrize("name", list(SIDES))
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_mixture_rhs_with_boundaries(N, name):
    torch, dg, d, mesh, gas = _setup((3, 2, 2), N, SIDES[name])
    q0 = _conserved(GAS, *_mixture_state(d.xyz, GAS))
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    T = torch.full(q0.shape[1:], T_SEED, device="cuda", dtype=torch.float64)
    dg.dg_rhs(mesh, gas, q, rhs, T_io=T)
    assert np.abs(T.cpu().numpy() - _newton(q0)).max() < 1e-9
    got = rhs.cpu().numpy()
    assert rel_err(got, _want(d, q0)) <= TOL
    assert rel_err(got[5:].sum(axis=0)[None], got[0][None]) <= 1e-12  # the species sum is the mass row
    assert mesh.status() == 0 and gas.status() == 0


def test_mixture_rk4_steps_with_boundaries():
    torch, dg, d, mesh, gas = _setup((3, 3, 2), 2, SIDES["in_out_x_walls_y"])
    q0 = _conserved(GAS, *_mixture_state(d.xyz, GAS, seed=3))
    dt = 1e-5  # a CFL of about 0.1: c + |u| ~ 700 m/s, h ~ 0.3 m, N = 2
    q = torch.tensor(q0, device="cuda")
    T = torch.full(q0.shape[1:], T_SEED, device="cuda", dtype=torch.float64)
    dg.lsrk4_step(mesh, gas, q, dt, steps=2, T_io=T)
    f = lambda u: _want(d, u)
    want = lsrk4_step(lsrk4_step(q0, dt, f), dt, f)
    assert rel_err(q.cpu().numpy() - q0, want - q0) <= TOL
    assert mesh.status() == 0 and gas.status() == 0


@pytest.mark.parametrize("name", list(SIDES))
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_mixed_mixture_rhs_with_boundaries(N, name):
    torch, dg, d, mesh, gas = _setup((3, 2, 2), N, SIDES[name])
    q0 = _conserved(GAS, *_mixture_state(d.xyz, GAS))
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    T = torch.full(q0.shape[1:], T_SEED, device="cuda", dtype=torch.float64)
    dg.dg_rhs(mesh, gas, q, rhs, T_io=T, opts=_mixed(dg))
    assert np.abs(T.cpu().numpy() - _newton(q0)).max() < 1e-9  # the temperature stays FP64 Newton
    err = field_err(rhs.cpu().numpy(), _want(d, q0))
    assert err <= MIXED_RHS_TOL, err
    assert mesh.status() == 0 and gas.status() == 0


def test_mixed_mixture_rk4_steps_with_boundaries():
    torch, dg, d, mesh, gas = _setup((3, 3, 2), 3, SIDES["in_out_x_walls_y"])
    q0 = _conserved(GAS, *_mixture_state(d.xyz, GAS, seed=3))
    dt = 1e-5
    q = torch.tensor(q0, device="cuda")
    T = torch.full(q0.shape[1:], T_SEED, device="cuda", dtype=torch.float64)
    dg.lsrk4_step(mesh, gas, q, dt, steps=2, T_io=T, opts=_mixed(dg))
    f = lambda u: _want(d, u)
    want = lsrk4_step(lsrk4_step(q0, dt, f), dt, f)
    err = field_err(q.cpu().numpy(), want)
    assert err <= MIXED_STATE_TOL, err
    assert mesh.status() == 0 and gas.status() == 0


def test_boundary_mixture_errors():
    """An inflow state of the wrong length or without a temperature is refused before any launch."""
    from paper_2512_17101_gb300 import capi
    torch, dg, d, mesh, gas = _setup((2, 2, 2), 1, SIDES["in_out_x_walls_y"])
    q0 = _conserved(GAS, *_mixture_state(d.xyz, GAS))
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    T = torch.full(q0.shape[1:], T_SEED, device="cuda", dtype=torch.float64)
    mesh.set_inflow(Q_IN[:5])  # a perfect-gas inflow state for a 7-species gas
    with pytest.raises(capi.DGError):
        dg.dg_rhs(mesh, gas, q, rhs, T_io=T)
    bad = Q_IN.copy()
    bad[4] = -1.0e12  # an internal energy below every temperature's
    mesh.set_inflow(bad)
    with pytest.raises(capi.DGError):
        dg.dg_rhs(mesh, gas, q, rhs, T_io=T)
    mesh.set_inflow(Q_IN)
    dg.dg_rhs(mesh, gas, q, rhs, T_io=T)  # and the mesh still works
    assert rel_err(rhs.cpu().numpy(), _want(d, q0)) <= TOL
