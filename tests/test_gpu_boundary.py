"""GPU parity of the boundary conditions: the FP64 Euler and Navier-Stokes right-hand sides on
meshes with slip walls, no-slip adiabatic walls, supersonic inflow and outflow, through the C ABI,
against the boundary-condition oracle (oracle/boundary.py) at 1e-11 per conserved variable."""

import numpy as np
import pytest

import oracle.boundary as bd
from oracle.lsrk import lsrk4_step
from oracle.thermo import PerfectGas
from tests._gpu import component_err, field_err, rel_err, torch_cuda
from tests._oracle_case import bc_disc
from workloads import equispaced_tet_nodes, uniform_perturbation

pytestmark = pytest.mark.gpu
TOL = 1e-11
GAS = PerfectGas(1.4, 1.0)
MU, PR = 2e-2, 0.71
SLIP, NOSLIP, INFLOW, OUTFLOW = bd.SLIP_WALL, bd.NOSLIP_WALL, bd.INFLOW, bd.OUTFLOW

SIDES = {
    "slip_y": {(1, 0): SLIP, (1, 1): SLIP},
    "noslip_y_slip_z": {(1, 0): NOSLIP, (1, 1): NOSLIP, (2, 0): SLIP, (2, 1): SLIP},
    "in_out_x_walls_y": {(0, 0): INFLOW, (0, 1): OUTFLOW, (1, 0): SLIP, (1, 1): NOSLIP},
    "closed_box": {(a, e): NOSLIP for a in range(3) for e in (0, 1)},
}


def _state(rho, u, v, w, p):
    E = p / (GAS.gamma - 1) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E])


def _smooth(xyz, seed=0):
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    rho = 1.0 + 0.1 * np.sin(2.1 * x + 0.7 * y) * np.cos(1.3 * z)
    u = 1.5 + 0.1 * np.cos(1.7 * y + 0.4 * z)
    v = 0.1 * np.sin(2.3 * x) * np.sin(0.9 * z + 0.2)
    w = 0.1 + 0.1 * np.cos(1.1 * x + 1.9 * y)
    p = 1.0 / 1.4 + 0.1 * np.sin(0.8 * x - 1.4 * z)
    return uniform_perturbation(_state(rho, u, v, w, p), 1e-3, seed=seed)


Q_IN = _state(np.array(1.1), np.array(1.8), np.array(0.05), np.array(-0.02), np.array(0.75))


def _setup(n, N, sides, viscous):
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    d = bc_disc(n, N, sides)
    mesh = dg.Mesh(d.vertices, d.period, N, equispaced_tet_nodes(N), face_bc=d.face_bc)
    if any(c == INFLOW for c in sides.values()):
        mesh.set_inflow(Q_IN)
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=MU if viscous else 0.0, Pr=PR)
    return torch, dg, d, mesh, gas


def _want(d, q, viscous):
    if viscous:
        return bd.rhs_ns_bc(d.ref, d.geo, d.conn, q, GAS, MU, PR, q_in=Q_IN)
    return bd.rhs_euler_bc(d.ref, d.geo, d.conn, q, GAS, q_in=Q_IN)


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("name", list(SIDES))
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_rhs_with_boundaries(N, name, viscous):
    torch, dg, d, mesh, gas = _setup((3, 2, 2), N, SIDES[name], viscous)
    q0 = _smooth(d.xyz)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs)
    assert rel_err(rhs.cpu().numpy(), _want(d, q0, viscous)) <= TOL
    assert mesh.status() == 0


@pytest.mark.parametrize("viscous", [False, True])
def test_two_rk4_steps_with_boundaries(viscous):
    torch, dg, d, mesh, gas = _setup((3, 3, 2), 2, SIDES["in_out_x_walls_y"], viscous)
    q0 = _smooth(d.xyz, seed=3)
    dt = 1e-3
    q = torch.tensor(q0, device="cuda")
    dg.lsrk4_step(mesh, gas, q, dt, steps=2)
    f = lambda u: _want(d, u, viscous)
    want = lsrk4_step(lsrk4_step(q0, dt, f), dt, f)
    assert rel_err(q.cpu().numpy() - q0, want - q0) <= TOL


def test_boundary_meshes_need_their_inflow_state():
    torch, dg, d, mesh, gas = _setup((2, 2, 2), 2, SIDES["in_out_x_walls_y"], True)
    from paper_2512_17101_gb300 import capi
    q = torch.tensor(_smooth(d.xyz), device="cuda")
    rhs = torch.empty_like(q)
    bare = dg.Mesh(d.vertices, d.period, 2, equispaced_tet_nodes(2), face_bc=d.face_bc)
    with pytest.raises(capi.DGError):  # inflow faces without an inflow state
        dg.dg_rhs(bare, gas, q, rhs)


def test_ghost_states_flag_a_nonphysical_inflow():
    """An inflow state with negative pressure is caught by the status word, not by a fault."""
    torch, dg, d, mesh, gas = _setup((2, 2, 2), 1, SIDES["in_out_x_walls_y"], False)
    bad = Q_IN.copy()
    bad[4] = 0.1  # E below the kinetic energy: p < 0
    mesh.set_inflow(bad)
    q = torch.tensor(_smooth(d.xyz), device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs)
    from paper_2512_17101_gb300 import capi
    assert mesh.status() & capi.DG_STATUS_NONPHYSICAL


@pytest.mark.slow
def test_channel_full_size_stage():
    """The wall-bounded benchmark workload (24^3 x 6 = 82,944 tets, N = 3, no-slip walls at
    y = 0, 1): the stage the benchmark times."""
    from workloads.configs import build_case, get_config
    from tests._oracle_case import Disc
    cfg = get_config("ns_channel")
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    case = build_case(cfg)
    d = Disc(case["vertices"], case["period"], cfg.N, face_bc=case["face_bc"])
    mesh = dg.Mesh(case["vertices"], case["period"], cfg.N, case["ref_nodes"], face_bc=case["face_bc"])
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=1e-3, Pr=0.71)
    q0 = case["q"]
    q_in = torch.tensor(q0, device="cuda")
    q_out, k = torch.empty_like(q_in), torch.zeros_like(q_in)
    dg.dg_rk_stage(mesh, gas, 0, cfg.dt, q_in, q_out, k)
    want = bd.rhs_ns_bc(d.ref, d.geo, d.conn, q0, GAS, 1e-3, 0.71)
    assert rel_err(k.cpu().numpy(), cfg.dt * want) <= TOL
    assert mesh.status() == 0


# --- the mixed-precision form with boundaries ------------------------------------------------------


MIXED_RHS_TOL = 1e-4  # per field, as for the periodic mixed form (tests/test_gpu_mixed.py)


def _mixed_opts(dg):
    from paper_2512_17101_gb300 import capi
    return dg._opts(precision=capi.DG_PREC_MIXED)


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("name", list(SIDES))
@pytest.mark.parametrize("N", [2, 3])
def test_mixed_rhs_with_boundaries(N, name, viscous):
    torch, dg, d, mesh, gas = _setup((3, 2, 2), N, SIDES[name], viscous)
    q0 = _smooth(d.xyz)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs, opts=_mixed_opts(dg))
    err = field_err(rhs.cpu().numpy(), _want(d, q0, viscous))
    assert err <= MIXED_RHS_TOL, err
    assert mesh.status() == 0


@pytest.mark.parametrize("viscous", [False, True])
def test_mixed_rk4_steps_with_boundaries(viscous):
    """Two RK4 steps of the mixed form against the oracle: state error <= 1e-6 per field."""
    torch, dg, d, mesh, gas = _setup((3, 3, 2), 3, SIDES["in_out_x_walls_y"], viscous)
    q0 = _smooth(d.xyz, seed=3)
    dt = 1e-3
    q = torch.tensor(q0, device="cuda")
    dg.lsrk4_step(mesh, gas, q, dt, steps=2, opts=_mixed_opts(dg))
    f = lambda u: _want(d, u, viscous)
    want = lsrk4_step(lsrk4_step(q0, dt, f), dt, f)
    err = field_err(q.cpu().numpy(), want)
    assert err <= 1e-6, err
    assert component_err(q.cpu().numpy(), want) <= 1e-4
