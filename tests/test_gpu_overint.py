"""GPU parity of over-integration on tetrahedra: the weak-form Euler and Navier-Stokes right-hand
sides with the volume term on the Stroud rule (dg_mesh_set_overint), through the C ABI, against
oracle/overint.py at 1e-11 per conserved variable.  Orders 1-4, periodic and walled / inflow /
outflow boxes, the default and other point counts, ragged last element groups and blocks that
loop over several groups, two RK4 steps, artificial viscosity on top, switching it off, and the
combinations the library refuses."""

import numpy as np
import pytest

import oracle.boundary as bd
import oracle.overint as oi
from oracle.euler import rhs_strong
from oracle.lsrk import lsrk4_step
from oracle.thermo import PerfectGas
from tests._gpu import rel_err, torch_cuda
from tests._oracle_case import bc_disc, box_disc
from workloads import equispaced_tet_nodes, isentropic_vortex, uniform_perturbation

pytestmark = pytest.mark.gpu
TOL = 1e-11
GAS = PerfectGas(1.4, 1.0)
MU, PR = 2e-2, 0.71
SLIP, NOSLIP, INFLOW, OUTFLOW = bd.SLIP_WALL, bd.NOSLIP_WALL, bd.INFLOW, bd.OUTFLOW
SIDES = {
    "periodic": None,
    "in_out_x_walls_y": {(0, 0): INFLOW, (0, 1): OUTFLOW, (1, 0): SLIP, (1, 1): NOSLIP},
}


def _state(rho, u, v, w, p):
    E = p / (GAS.gamma - 1) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E])


Q_IN = _state(np.array(1.1), np.array(1.8), np.array(0.05), np.array(-0.02), np.array(0.75))


def _smooth(xyz, seed=0):
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    rho = 1.0 + 0.2 * np.sin(2.1 * x + 0.7 * y) * np.cos(1.3 * z)
    u = 1.5 + 0.3 * np.cos(1.7 * y + 0.4 * z)
    v = 0.2 * np.sin(2.3 * x) * np.sin(0.9 * z + 0.2)
    w = 0.1 + 0.2 * np.cos(1.1 * x + 1.9 * y)
    p = 1.0 / 1.4 + 0.2 * np.sin(0.8 * x - 1.4 * z)
    return uniform_perturbation(_state(rho, u, v, w, p), 1e-3, seed=seed)


def _setup(n, N, sides, q=None, viscous=False):
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    d = box_disc(n, N) if sides is None else bc_disc(n, N, sides)
    mesh = dg.Mesh(d.vertices, d.period, N, equispaced_tet_nodes(N), face_bc=d.face_bc)
    if sides and any(c == INFLOW for c in sides.values()):
        mesh.set_inflow(Q_IN)
    mesh.set_overint(-1 if q is None else q)
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=MU if viscous else 0.0, Pr=PR)
    return torch, dg, d, mesh, gas


def _want(d, q0, Q=None, viscous=False):
    if viscous:
        return oi.rhs_overint_ns(d.ref, d.geo, d.conn, q0, GAS, MU, PR, Q=Q, q_in=Q_IN)
    return oi.rhs_overint(d.ref, d.geo, d.conn, q0, GAS, Q=Q, q_in=Q_IN)


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("name", list(SIDES))
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_overint_rhs(N, name, viscous):
    n = 3 if SIDES[name] is None else (3, 2, 2)
    torch, dg, d, mesh, gas = _setup(n, N, SIDES[name], viscous=viscous)
    q0 = _smooth(d.xyz)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs)
    assert rel_err(rhs.cpu().numpy(), _want(d, q0, viscous=viscous)) <= TOL
    assert mesh.status() == 0


def test_overint_ns_closed_box():
    """No-slip walls on every side (adiabatic, shear at the walls)."""
    sides = {(a, e): NOSLIP for a in range(3) for e in (0, 1)}
    torch, dg, d, mesh, gas = _setup((2, 2, 2), 3, sides, viscous=True)
    q0 = _smooth(d.xyz, seed=8)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs)
    assert rel_err(rhs.cpu().numpy(), _want(d, q0, viscous=True)) <= TOL


@pytest.mark.parametrize("N,Q", [(1, 1), (2, 2), (2, 4), (3, 6), (4, 7)])
def test_overint_other_point_counts(N, Q):
    torch, dg, d, mesh, gas = _setup((3, 2, 2), N, SIDES["in_out_x_walls_y"], q=Q)
    q0 = _smooth(d.xyz, seed=2)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs)
    assert rel_err(rhs.cpu().numpy(), _want(d, q0, Q=Q)) <= TOL


@pytest.mark.parametrize("N", [2, 3])
def test_overint_many_groups_per_block(N):
    """Enough elements that every persistent block loops over several element groups."""
    torch, dg, d, mesh, gas = _setup(6, N, None)
    q0 = uniform_perturbation(isentropic_vortex(d.xyz, 0.0), 1e-3, seed=5)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs)
    assert rel_err(rhs.cpu().numpy(), _want(d, q0)) <= TOL


@pytest.mark.parametrize("viscous", [False, True])
def test_overint_rk4_steps(viscous):
    torch, dg, d, mesh, gas = _setup((3, 3, 2), 3, SIDES["in_out_x_walls_y"], viscous=viscous)
    q0 = _smooth(d.xyz, seed=3)
    dt = 2e-4 if viscous else 1e-3  # the viscous steps at N = 3 with walls need the smaller step
    q = torch.tensor(q0, device="cuda")
    dg.lsrk4_step(mesh, gas, q, dt, steps=2)
    f = lambda u: _want(d, u, viscous=viscous)
    want = lsrk4_step(lsrk4_step(q0, dt, f), dt, f)
    assert rel_err(q.cpu().numpy() - q0, want - q0) <= TOL
    assert mesh.status() == 0


def test_overint_off_is_the_collocated_form():
    torch, dg, d, mesh, gas = _setup(3, 2, None)
    q0 = _smooth(d.xyz, seed=4)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    mesh.set_overint(0)
    dg.dg_rhs(mesh, gas, q, rhs)
    assert rel_err(rhs.cpu().numpy(), rhs_strong(d.ref, d.geo, d.conn, q0, GAS)) <= TOL
    mesh.set_overint(-1)
    dg.dg_rhs(mesh, gas, q, rhs)
    assert rel_err(rhs.cpu().numpy(), _want(d, q0)) <= TOL


def test_overint_flags_a_nonphysical_state():
    torch, dg, d, mesh, gas = _setup(2, 2, None)
    q0 = _smooth(d.xyz)
    q0[4, 3, :] = 0.01  # energy below the kinetic energy in one element: p < 0 at its points
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs)
    from paper_2512_17101_gb300 import capi
    assert mesh.status() & capi.DG_STATUS_NONPHYSICAL


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("name", list(SIDES))
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_overint_with_artificial_viscosity(N, name, viscous):
    """Over-integration plus the AV term on a steep front whose elements span all three regimes of
    the viscosity ramp (the front and thresholds of tests/test_gpu_av.py), with a z velocity of
    the size of the x velocity.  (On that test's own front rho w is 1/700 of rho u; the weak form
    cancels terms several hundred times that row's result across the reference directions, and
    at N = 4 the row keeps 3e-11 of its own maximum in rounding, against an extended-precision
    evaluation, while the FP64 oracle keeps 1e-12.)"""
    import oracle.av as av
    from tests.test_gpu_av import EPS0, _front, _thresholds
    sides = SIDES[name]
    torch, dg, d, mesh, gas = _setup((4, 2, 2), N, sides, viscous=viscous)
    q0 = _front(d.xyz)
    w = 0.2 + 0.1 * np.cos(2 * np.pi * d.xyz[..., 1])  # rho w of the size of rho u, E to match
    q0[4] += 0.5 * ((q0[0] * w) ** 2 - q0[3] ** 2) / q0[0]
    q0[3] = q0[0] * w
    s0, kappa = _thresholds(d, q0)
    mesh.set_av(EPS0, s0, kappa)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs)
    eps = av.element_viscosity(d.ref, q0, EPS0, s0, kappa)
    assert (eps == 0).any() and (eps > 0).any()
    want = oi.rhs_overint_av(d.ref, d.geo, d.conn, q0, GAS, eps, mu=MU if viscous else 0.0, Pr=PR, q_in=Q_IN)
    assert rel_err(rhs.cpu().numpy(), want) <= TOL
    assert mesh.status() == 0


def test_overint_refusals():
    """A mixture, the mixed form, element ranges and point counts whose tables do not fit are
    refused; the mesh keeps working, with and without artificial viscosity."""
    from paper_2512_17101_gb300 import capi
    from workloads.gas import seeded_nasa7_mixture
    torch, dg, d, mesh, gas = _setup(2, 4, None)
    q0 = _smooth(d.xyz)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    mix = seeded_nasa7_mixture(2, seed=0)
    mgas = dg.Gas(model="nasa7", W=mix.W, nasa7=mix.coeffs)
    qm = torch.zeros((7,) + tuple(q.shape[1:]), device="cuda", dtype=torch.float64)
    T = torch.full(tuple(q.shape[1:]), 1000.0, device="cuda", dtype=torch.float64)
    with pytest.raises(capi.DGError):
        dg.dg_rhs(mesh, mgas, qm, torch.empty_like(qm), T_io=T)
    with pytest.raises(capi.DGError):
        dg.dg_rhs(mesh, gas, q, rhs, opts=dg._opts(precision=capi.DG_PREC_MIXED))
    with pytest.raises(capi.DGError):
        dg.dg_rhs(mesh, gas, q, rhs, opts=dg._opts(elems=(0, 6)))
    with pytest.raises(capi.DGError):
        mesh.set_overint(capi.DG_MAX_OVERINT_POINTS)  # N = 4: 1728 points do not fit
    with pytest.raises(capi.DGError):
        mesh.set_overint(-2)
    dg.dg_rhs(mesh, gas, q, rhs)
    assert rel_err(rhs.cpu().numpy(), _want(d, q0)) <= TOL


@pytest.mark.parametrize("av_on", [False, True])
def test_overint_diffusive_fluxes_need_n_plus_one_points(av_on):
    """The viscous and AV fluxes take the exact weak form of a degree-N nodal field, which the rule
    reproduces only from N + 1 points per direction: with N points the right-hand side is
    refused, with N + 1 it matches the oracle on that rule, and Euler still runs with N points."""
    from paper_2512_17101_gb300 import capi
    from tests.test_gpu_av import EPS0
    N = 3
    torch, dg, d, mesh, gas = _setup((3, 2, 2), N, SIDES["in_out_x_walls_y"], q=N, viscous=not av_on)
    q0 = _smooth(d.xyz, seed=6)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    if av_on:
        mesh.set_av(EPS0, -40.0, 1.0)  # a threshold far below the smooth state's indicator: eps0 everywhere
    with pytest.raises(capi.DGError):
        dg.dg_rhs(mesh, gas, q, rhs)
    if not av_on:
        euler = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=0.0, Pr=PR)
        dg.dg_rhs(mesh, euler, q, rhs)
        assert rel_err(rhs.cpu().numpy(), _want(d, q0, Q=N)) <= TOL
    mesh.set_overint(N + 1)
    dg.dg_rhs(mesh, gas, q, rhs)
    if av_on:
        import oracle.av as av
        eps = av.element_viscosity(d.ref, q0, EPS0, -40.0, 1.0)
        assert (eps > 0).all()
        want = oi.rhs_overint_av(d.ref, d.geo, d.conn, q0, GAS, eps, Q=N + 1, q_in=Q_IN)
    else:
        want = _want(d, q0, Q=N + 1, viscous=True)
    assert rel_err(rhs.cpu().numpy(), want) <= TOL
    assert mesh.status() == 0


@pytest.mark.parametrize("N,Q,viscous", [(2, 11, False), (3, 10, True), (4, 9, False), (4, 9, True)])
def test_overint_largest_point_counts(N, Q, viscous):
    """The largest point counts that fit: one element per block, even and odd Q (the folded
    a-sum with and without a middle point), Q >= 2N, so that the rule is exact for the cubic
    energy flux of a degree-N state too."""
    torch, dg, d, mesh, gas = _setup((3, 2, 2), N, SIDES["in_out_x_walls_y"], q=Q, viscous=viscous)
    q0 = _smooth(d.xyz, seed=7)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs)
    assert rel_err(rhs.cpu().numpy(), _want(d, q0, Q=Q, viscous=viscous)) <= TOL
    assert mesh.status() == 0
