"""GPU parity of the viscous mixture (species diffusion, enthalpy diffusion, heat conduction) on
meshes with boundary faces: the FP64 right-hand side through the C ABI against the oracle
(oracle/mixture_ns.py: rhs_ns_mixture_bc), temperatures from Newton on both sides, at 1e-11 per
conserved variable, and the viscous part on its own (minus the inviscid boundary right-hand side)
at 1e-9.  Orders 1-4 on four boundary layouts, and two RK4 steps."""

import numpy as np
import pytest

import oracle.boundary as bd
import oracle.mixture_ns as mns
from oracle.lsrk import lsrk4_step
from tests._gpu import rel_err, torch_cuda
from tests._oracle_case import bc_disc
from tests.test_oracle_mixture_boundary import GAS, MIX, _conserved, _inflow_state, _mixture_state
from workloads import equispaced_tet_nodes

pytestmark = pytest.mark.gpu
TOL = 1e-11
MU, PR, SC = 0.5, 0.71, 0.6
SLIP, NOSLIP, INFLOW, OUTFLOW = bd.SLIP_WALL, bd.NOSLIP_WALL, bd.INFLOW, bd.OUTFLOW
T_SEED = 1500.0
SIDES = {
    "slip_y": {(1, 0): SLIP, (1, 1): SLIP},
    "noslip_y_slip_z": {(1, 0): NOSLIP, (1, 1): NOSLIP, (2, 0): SLIP, (2, 1): SLIP},
    "in_out_x_walls_y": {(0, 0): INFLOW, (0, 1): OUTFLOW, (1, 0): SLIP, (1, 1): NOSLIP},
    "closed_box": {(a, e): NOSLIP for a in range(3) for e in (0, 1)},
}
Q_IN, T_IN = _inflow_state(GAS)


def _setup(n, N, sides):
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    d = bc_disc(n, N, sides)
    mesh = dg.Mesh(d.vertices, d.period, N, equispaced_tet_nodes(N), face_bc=d.face_bc)
    if any(c == INFLOW for c in sides.values()):
        mesh.set_inflow(Q_IN)
    gas = dg.Gas(model="nasa7", W=MIX.W, nasa7=MIX.coeffs, newton_tol=1e-10, newton_max_it=50, mu=MU, Pr=PR,
                 Sc=SC)
    return torch, dg, d, mesh, gas


def _newton(q):
    rho, vel, Y, e = GAS.split_state(q)
    T, _, ok = GAS.newton_temperature(e, Y, np.full(e.shape, T_SEED))
    assert ok.all()
    return T


def _want(d, q):
    return mns.rhs_ns_mixture_bc(d.ref, d.geo, d.conn, q, GAS, _newton(q), MU, PR, SC, q_in=Q_IN, T_in=T_IN)


@pytest.mark.parametrize("name", list(SIDES))
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_viscous_mixture_rhs_with_boundaries(N, name):
    torch, dg, d, mesh, gas = _setup((3, 2, 2), N, SIDES[name])
    q0 = _conserved(GAS, *_mixture_state(d.xyz, GAS))
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    T = torch.full(q0.shape[1:], T_SEED, device="cuda", dtype=torch.float64)
    dg.dg_rhs(mesh, gas, q, rhs, T_io=T)
    got, want = rhs.cpu().numpy(), _want(d, q0)
    assert rel_err(got, want) <= TOL
    inviscid = bd.rhs_mixture_bc(d.ref, d.geo, d.conn, q0, GAS, _newton(q0), q_in=Q_IN, T_in=T_IN)
    assert rel_err(got - inviscid, want - inviscid) <= 1e-9
    assert mesh.status() == 0 and gas.status() == 0


def test_viscous_mixture_rk4_steps_with_boundaries():
    torch, dg, d, mesh, gas = _setup((3, 3, 2), 2, SIDES["in_out_x_walls_y"])
    q0 = _conserved(GAS, *_mixture_state(d.xyz, GAS, seed=3))
    dt = 2e-6
    q = torch.tensor(q0, device="cuda")
    T = torch.full(q0.shape[1:], T_SEED, device="cuda", dtype=torch.float64)
    dg.lsrk4_step(mesh, gas, q, dt, steps=2, T_io=T)
    f = lambda u: _want(d, u)
    want = lsrk4_step(lsrk4_step(q0, dt, f), dt, f)
    assert rel_err(q.cpu().numpy() - q0, want - q0) <= TOL
    assert mesh.status() == 0 and gas.status() == 0
