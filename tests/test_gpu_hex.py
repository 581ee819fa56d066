"""Tensor-product hexahedra: the CUDA path through the C ABI against the hexahedron oracle
(FP64, 1e-11 relative per conserved variable)."""

import numpy as np
import pytest

import oracle.hex as hx
from oracle.lsrk import lsrk4_stage, lsrk4_step
from oracle.thermo import PerfectGas
from tests._gpu import rel_err, torch_cuda
from workloads import isentropic_vortex, uniform_perturbation
from workloads.hexmesh import gll_nodes, hex_box, hex_nodes

pytestmark = pytest.mark.gpu
TOL = 1e-11
GAS = PerfectGas(1.4, 1.0)


def _setup(n, N, L=1.0, noise=1e-3, seed=0):
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    box = hex_box(n, L)
    x = gll_nodes(N)
    ref = hx.hex_reference(x)
    q0 = isentropic_vortex(hex_nodes(box, x), 0.0, center=(0.45, 0.55), radius=0.15, period=box["L"])
    q0 = uniform_perturbation(q0, noise, seed=seed)
    mesh = dg.HexMesh(box["n"], box["L"], N, x)
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0)
    return torch, dg, box, ref, q0, mesh, gas


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_hex_operators_match_oracle(N):
    torch, dg, box, ref, q0, mesh, gas = _setup(1, N)
    D, w = mesh.operators()
    assert np.abs(D - ref.D).max() <= 1e-13 * max(1.0, np.abs(ref.D).max())
    assert np.abs(w - ref.w).max() <= 1e-15


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [1, (3, 2, 2), (5, 1, 3)])
def test_hex_rhs(n, N):
    torch, dg, box, ref, q0, mesh, gas = _setup(n, N)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_hex_rhs(mesh, gas, q, rhs)
    want = hx.hex_rhs_strong(ref, box, q0, GAS)
    assert rel_err(rhs.cpu().numpy(), want) <= TOL
    assert mesh.status() == 0


def test_hex_two_rk4_steps():
    torch, dg, box, ref, q0, mesh, gas = _setup((4, 3, 2), 3)
    dt = 2e-3
    q = torch.tensor(q0, device="cuda")
    dg.hex_lsrk4_step(mesh, gas, q, dt, steps=2)
    f = lambda u: hx.hex_rhs_strong(ref, box, u, GAS)
    want = lsrk4_step(lsrk4_step(q0, dt, f), dt, f)
    assert rel_err(q.cpu().numpy() - q0, want - q0) <= TOL


def test_hex_rejects_what_it_does_not_solve():
    torch, dg, box, ref, q0, mesh, gas = _setup(2, 2)
    from paper_2512_17101_gb300 import capi
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    mix = dg.Gas(model="nasa7", W=np.array([28.0]), nasa7=np.array([[3.5, 0, 0, 0, 0, 0, 0]]))
    with pytest.raises(capi.DGError):  # a perfect gas only
        dg.dg_hex_rhs(mesh, mix, q, rhs)
    with pytest.raises(capi.DGError):
        dg.dg_hex_rhs(mesh, gas, q, q)
    with pytest.raises(capi.DGError):
        dg.HexMesh(2, 1.0, 2, np.array([-1.0, 0.5, 0.2]))


def test_hex_status_flags_without_fault():
    torch, dg, box, ref, q0, mesh, gas = _setup(2, 2)
    q0 = q0.copy()
    q0[0, 3, 1] = -1.0
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_hex_rhs(mesh, gas, q, rhs)
    from paper_2512_17101_gb300 import capi
    assert mesh.status() & capi.DG_STATUS_NONPHYSICAL


@pytest.mark.slow
def test_hex_vortex_full_size_stage():
    """The hexahedral benchmark workload (32^3 hexahedra, N = 4): the stage the benchmark times."""
    from workloads.configs import build_hex_case, get_config
    cfg = get_config("hex_vortex")
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    case = build_hex_case(cfg)
    ref = hx.hex_reference(case["nodes1d"])
    mesh = dg.HexMesh(case["box"]["n"], case["box"]["L"], cfg.N, case["nodes1d"])
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0)
    q_in = torch.tensor(case["q"], device="cuda")
    q_out, k = torch.empty_like(q_in), torch.zeros_like(q_in)
    dg.dg_hex_rk_stage(mesh, gas, 0, cfg.dt, q_in, q_out, k)
    want = hx.hex_rhs_strong(ref, case["box"], case["q"], GAS)
    assert rel_err(k.cpu().numpy(), cfg.dt * want) <= TOL
    assert mesh.status() == 0


# --- scalar advection -------------------------------------------------------------------------------

VELOCITIES = [(1.0, -0.5, 0.25), (0.0, 0.0, -2.0), (-1.0, 0.3, 0.0)]


def _adv_setup(n, N, noise=1e-3, seed=0):
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    from workloads import advected_wave
    box = hex_box(n, 1.0)
    x = gll_nodes(N)
    ref = hx.hex_reference(x)
    u0 = advected_wave(hex_nodes(box, x))
    u0 = u0 + noise * np.random.default_rng(seed).uniform(-1.0, 1.0, u0.shape)
    mesh = dg.HexMesh(box["n"], box["L"], N, x)
    return torch, dg, box, ref, u0, mesh


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [1, (3, 2, 2), (5, 1, 3)])
@pytest.mark.parametrize("vel", VELOCITIES)
def test_hex_advection_rhs(n, N, vel):
    torch, dg, box, ref, u0, mesh = _adv_setup(n, N)
    u = torch.tensor(u0, device="cuda")
    rhs = torch.empty_like(u)
    dg.dg_hex_advection_rhs(mesh, vel, u, rhs)
    want = hx.hex_advection_rhs_strong(ref, box, u0, vel)
    assert _rel(rhs.cpu().numpy(), want) <= TOL


def test_hex_advection_many_blocks_ragged():
    """More elements than one block holds, with a ragged last block (5 x 7 x 3 = 105 elements)."""
    torch, dg, box, ref, u0, mesh = _adv_setup((5, 7, 3), 1)
    u = torch.tensor(u0, device="cuda")
    rhs = torch.empty_like(u)
    dg.dg_hex_advection_rhs(mesh, VELOCITIES[0], u, rhs)
    assert _rel(rhs.cpu().numpy(), hx.hex_advection_rhs_strong(ref, box, u0, VELOCITIES[0])) <= TOL


def test_hex_advection_two_rk4_steps():
    torch, dg, box, ref, u0, mesh = _adv_setup((4, 3, 2), 2)
    dt, vel = 2e-3, VELOCITIES[0]
    u = torch.tensor(u0, device="cuda")
    dg.hex_advection_lsrk4_step(mesh, vel, u, dt, steps=2)
    f = lambda v: hx.hex_advection_rhs_strong(ref, box, v, vel)
    want = lsrk4_step(lsrk4_step(u0, dt, f), dt, f)
    assert _rel(u.cpu().numpy() - u0, want - u0) <= TOL


def test_hex_advection_rejects_bad_arguments():
    torch, dg, box, ref, u0, mesh = _adv_setup(2, 2)
    from paper_2512_17101_gb300 import capi
    u = torch.tensor(u0, device="cuda")
    rhs = torch.empty_like(u)
    with pytest.raises(capi.DGError):
        dg.dg_hex_advection_rhs(mesh, (np.nan, 0.0, 0.0), u, rhs)
    with pytest.raises(capi.DGError):
        dg.dg_hex_advection_rhs(mesh, VELOCITIES[0], u, u)
    with pytest.raises(ValueError):
        dg.dg_hex_advection_rhs(mesh, VELOCITIES[0], u[:-1], rhs[:-1])
    with pytest.raises(ValueError):
        dg.dg_hex_advection_rhs(mesh, (1.0, 0.0), u, rhs)


@pytest.mark.slow
def test_hex_advection_full_size_stage():
    """The advection benchmark workload (128^3 hexahedra, N = 1): the stage the benchmark times."""
    from workloads.configs import build_hex_advection_case, get_config
    cfg = get_config("hex_advection")
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    case = build_hex_advection_case(cfg)
    ref = hx.hex_reference(case["nodes1d"])
    mesh = dg.HexMesh(case["box"]["n"], case["box"]["L"], cfg.N, case["nodes1d"])
    u_in = torch.tensor(case["u"], device="cuda")
    u_out, k = torch.empty_like(u_in), torch.zeros_like(u_in)
    dg.dg_hex_advection_rk_stage(mesh, case["velocity"], 0, cfg.dt, u_in, u_out, k)
    f = lambda v: hx.hex_advection_rhs_strong(ref, case["box"], v, case["velocity"])
    want_u, want_k = lsrk4_stage(case["u"], np.zeros_like(case["u"]), 0, cfg.dt, f)
    assert _rel(k.cpu().numpy(), want_k) <= TOL
    assert _rel(u_out.cpu().numpy() - case["u"], want_u - case["u"]) <= TOL


# --- box-face boundary conditions ------------------------------------------------------------------

import oracle.boundary as bd  # noqa: E402

HEX_BC = {
    "channel": ((bd.INFLOW, bd.OUTFLOW), (bd.SLIP_WALL, bd.SLIP_WALL), (0, 0)),
    "closed": ((bd.SLIP_WALL, bd.SLIP_WALL), (bd.NOSLIP_WALL, bd.NOSLIP_WALL), (bd.SLIP_WALL, bd.OUTFLOW)),
}


def _bc_setup(n, N, bc):
    torch, dg, box, ref, q0, mesh, gas = _setup(n, N)
    box["bc"] = bc
    mesh = dg.HexMesh(box["n"], box["L"], N, gll_nodes(N), bc=bc)
    q_in = q0[:, 0, 0].copy()
    mesh.set_inflow(q_in)
    return torch, dg, box, ref, q0, mesh, gas, q_in


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("name", list(HEX_BC))
def test_hex_rhs_with_boundaries(name, N):
    torch, dg, box, ref, q0, mesh, gas, q_in = _bc_setup((3, 2, 2), N, HEX_BC[name])
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_hex_rhs(mesh, gas, q, rhs)
    want = hx.hex_rhs_strong(ref, box, q0, GAS, q_in=q_in)
    assert rel_err(rhs.cpu().numpy(), want) <= TOL
    assert mesh.status() == 0


def test_hex_two_rk4_steps_with_boundaries():
    torch, dg, box, ref, q0, mesh, gas, q_in = _bc_setup((4, 3, 2), 3, HEX_BC["channel"])
    dt = 2e-3
    q = torch.tensor(q0, device="cuda")
    dg.hex_lsrk4_step(mesh, gas, q, dt, steps=2)
    f = lambda u: hx.hex_rhs_strong(ref, box, u, GAS, q_in=q_in)
    want = lsrk4_step(lsrk4_step(q0, dt, f), dt, f)
    assert rel_err(q.cpu().numpy() - q0, want - q0) <= TOL


def test_hex_boundary_arguments():
    torch, dg, box, ref, q0, mesh, gas = _setup(2, 2)
    from paper_2512_17101_gb300 import capi
    with pytest.raises(capi.DGError):  # periodic at one end only
        dg.HexMesh(2, 1.0, 2, gll_nodes(2), bc=((bd.SLIP_WALL, 0), (0, 0), (0, 0)))
    m = dg.HexMesh(2, 1.0, 2, gll_nodes(2), bc=HEX_BC["channel"])
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    with pytest.raises(capi.DGError):  # inflow face without its state
        dg.dg_hex_rhs(m, gas, q, rhs)
    u = torch.zeros(m.K * m.Np, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.DGError):  # the advection runs on periodic boxes
        dg.dg_hex_advection_rhs(m, (1.0, 0.0, 0.0), u, torch.empty_like(u))


# --- Navier-Stokes on periodic boxes ---------------------------------------------------------------

NS_MU, NS_PR = 2e-2, 0.71


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [1, (3, 2, 2)])
def test_hex_navier_stokes_rhs(n, N):
    torch, dg, box, ref, q0, mesh, gas = _setup(n, N)
    ns = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=NS_MU, Pr=NS_PR)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_hex_rhs(mesh, ns, q, rhs)
    want = hx.hex_rhs_ns(ref, box, q0, GAS, NS_MU, NS_PR)
    got = rhs.cpu().numpy()
    assert rel_err(got, want) <= TOL
    euler = hx.hex_rhs_strong(ref, box, q0, GAS)
    assert rel_err(got - euler, want - euler) <= 1e-9  # the viscous part on its own
    assert mesh.status() == 0


def test_hex_navier_stokes_two_rk4_steps():
    torch, dg, box, ref, q0, mesh, gas = _setup((4, 3, 2), 3)
    ns = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=NS_MU, Pr=NS_PR)
    dt = 1e-3
    q = torch.tensor(q0, device="cuda")
    dg.hex_lsrk4_step(mesh, ns, q, dt, steps=2)
    f = lambda u: hx.hex_rhs_ns(ref, box, u, GAS, NS_MU, NS_PR)
    want = lsrk4_step(lsrk4_step(q0, dt, f), dt, f)
    assert rel_err(q.cpu().numpy() - q0, want - q0) <= TOL


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("name", list(HEX_BC))
def test_hex_navier_stokes_with_walls(name, N):
    torch, dg, box, ref, q0, mesh, gas, q_in = _bc_setup((3, 2, 2), N, HEX_BC[name])
    ns = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=NS_MU, Pr=NS_PR)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_hex_rhs(mesh, ns, q, rhs)
    want = hx.hex_rhs_ns(ref, box, q0, GAS, NS_MU, NS_PR, q_in=q_in)
    got = rhs.cpu().numpy()
    assert rel_err(got, want) <= TOL
    euler = hx.hex_rhs_strong(ref, box, q0, GAS, q_in=q_in)
    assert rel_err(got - euler, want - euler) <= 1e-9


# --- artificial viscosity --------------------------------------------------------------------------

AV_EPS0 = 1e-2


def _front_state(xyz):
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    th = np.tanh((x - 0.5) / 0.04)
    rho = 1.5 + 0.5 * th + 0.05 * np.sin(2 * np.pi * y)
    u = 0.3 - 0.2 * th
    v = 0.05 * np.cos(2 * np.pi * z)
    w = 0.02 * np.sin(2 * np.pi * x)
    p = 1.2 + 0.4 * th
    return np.stack([rho, rho * u, rho * v, rho * w, p / 0.4 + 0.5 * rho * (u * u + v * v + w * w)])


def _av_thresholds(ref, q):
    """s0 at the second-largest indicator value of the state and kappa half its distance to the
    nearest other value: elements fall on zero, on the ramp and on eps0."""
    u = np.unique(np.round(np.log10(hx.hex_indicator(ref, q[0])), 9))
    s0 = u[-2]
    return s0, 0.5 * min(u[-1] - s0, s0 - u[-3])


def _av_setup(N, bc=None):
    torch, dg, box, ref, q0, mesh, gas = _setup((4, 2, 2), N)
    q0 = _front_state(hex_nodes(box, gll_nodes(N)))
    if bc is not None:
        box["bc"] = bc
        mesh = dg.HexMesh(box["n"], box["L"], N, gll_nodes(N), bc=bc)
        mesh.set_inflow(q0[:, 0, 0])
    s0, kappa = _av_thresholds(ref, q0)
    mesh.set_av(AV_EPS0, s0, kappa)
    return torch, dg, box, ref, q0, mesh, gas, (s0, kappa)


def _av_eps(ref, q, th):
    import oracle.av as oav
    return oav.viscosity(hx.hex_indicator(ref, q[0]), AV_EPS0, th[0], th[1])


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_hex_element_viscosity(N):
    torch, dg, box, ref, q0, mesh, gas, th = _av_setup(N)
    eps = torch.empty(mesh.K, dtype=torch.float64, device="cuda")
    mesh.av_viscosity(torch.tensor(q0, device="cuda"), eps)
    want = _av_eps(ref, q0, th)
    assert np.abs(eps.cpu().numpy() - want).max() <= 1e-11 * AV_EPS0
    assert (want == 0).any() and (want == AV_EPS0).any() and ((want > 0) & (want < AV_EPS0)).any()


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_hex_rhs_with_artificial_viscosity(N, viscous):
    torch, dg, box, ref, q0, mesh, gas, th = _av_setup(N)
    g = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=NS_MU if viscous else 0.0, Pr=NS_PR)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_hex_rhs(mesh, g, q, rhs)
    base = hx.hex_rhs_ns(ref, box, q0, GAS, NS_MU, NS_PR) if viscous else hx.hex_rhs_strong(ref, box, q0, GAS)
    want = base + hx.hex_rhs_av(ref, box, q0, _av_eps(ref, q0, th))
    assert rel_err(rhs.cpu().numpy(), want) <= TOL
    assert mesh.status() == 0


def test_hex_artificial_viscosity_with_walls():
    torch, dg, box, ref, q0, mesh, gas, th = _av_setup(3, bc=HEX_BC["channel"])
    g = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=NS_MU, Pr=NS_PR)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_hex_rhs(mesh, g, q, rhs)
    q_in = q0[:, 0, 0]
    want = (hx.hex_rhs_ns(ref, box, q0, GAS, NS_MU, NS_PR, q_in=q_in)
            + hx.hex_rhs_av(ref, box, q0, _av_eps(ref, q0, th), q_in=q_in))
    assert rel_err(rhs.cpu().numpy(), want) <= TOL


# --- over-integration -------------------------------------------------------------------------------

def _q32(N):
    return int(np.ceil(3 * (N + 1) / 2))


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [1, (3, 2, 2), (5, 1, 3)])
def test_hex_overintegrated_rhs(n, N):
    torch, dg, box, ref, q0, mesh, gas = _setup(n, N)
    mesh.set_overintegration(True)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_hex_rhs(mesh, gas, q, rhs)
    want = hx.hex_rhs_overint(ref, box, q0, GAS, _q32(N))
    assert rel_err(rhs.cpu().numpy(), want) <= TOL
    assert mesh.status() == 0


def test_hex_overintegrated_with_boundaries_and_rk_steps():
    torch, dg, box, ref, q0, mesh, gas, q_in = _bc_setup((4, 3, 2), 3, HEX_BC["channel"])
    mesh.set_overintegration(True)
    dt = 2e-3
    q = torch.tensor(q0, device="cuda")
    dg.hex_lsrk4_step(mesh, gas, q, dt, steps=2)
    f = lambda u: hx.hex_rhs_overint(ref, box, u, GAS, _q32(3), q_in=q_in)
    want = lsrk4_step(lsrk4_step(q0, dt, f), dt, f)
    assert rel_err(q.cpu().numpy() - q0, want - q0) <= TOL


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("bc", [None, "closed"])
def test_hex_overintegrated_ns_rhs(N, bc):
    """Navier-Stokes with over-integration: periodic, and closed by no-slip and slip walls."""
    if bc is None:
        torch, dg, box, ref, q0, mesh, gas = _setup((3, 2, 2), N)
        q_in = None
    else:
        torch, dg, box, ref, q0, mesh, gas, q_in = _bc_setup((3, 2, 2), N, HEX_BC[bc])
    mesh.set_overintegration(True)
    ns = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=NS_MU, Pr=NS_PR)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_hex_rhs(mesh, ns, q, rhs)
    want = hx.hex_rhs_overint_ns(ref, box, q0, GAS, NS_MU, NS_PR, _q32(N), q_in=q_in)
    assert rel_err(rhs.cpu().numpy(), want) <= TOL
    assert mesh.status() == 0


def test_hex_overintegrated_ns_channel_rk_steps():
    torch, dg, box, ref, q0, mesh, gas, q_in = _bc_setup((4, 3, 2), 3, HEX_BC["channel"])
    mesh.set_overintegration(True)
    ns = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=NS_MU, Pr=NS_PR)
    dt = 1e-3
    q = torch.tensor(q0, device="cuda")
    dg.hex_lsrk4_step(mesh, ns, q, dt, steps=2)
    f = lambda u: hx.hex_rhs_overint_ns(ref, box, u, GAS, NS_MU, NS_PR, _q32(3), q_in=q_in)
    want = lsrk4_step(lsrk4_step(q0, dt, f), dt, f)
    assert rel_err(q.cpu().numpy() - q0, want - q0) <= TOL


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_hex_overintegrated_with_artificial_viscosity(N, viscous):
    """Over-integration with the AV term on the steep front (all three regimes of the ramp), and
    with walls at N = 3."""
    torch, dg, box, ref, q0, mesh, gas, th = _av_setup(N)
    mesh.set_overintegration(True)
    g = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=NS_MU if viscous else 0.0, Pr=NS_PR)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_hex_rhs(mesh, g, q, rhs)
    want = hx.hex_rhs_overint_av(ref, box, q0, GAS, _av_eps(ref, q0, th), _q32(N),
                                 mu=NS_MU if viscous else 0.0, Pr=NS_PR)
    assert rel_err(rhs.cpu().numpy(), want) <= TOL
    assert mesh.status() == 0


def test_hex_overintegrated_with_artificial_viscosity_and_walls():
    torch, dg, box, ref, q0, mesh, gas, th = _av_setup(3, bc=HEX_BC["channel"])
    mesh.set_overintegration(True)
    g = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=NS_MU, Pr=NS_PR)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_hex_rhs(mesh, g, q, rhs)
    want = hx.hex_rhs_overint_av(ref, box, q0, GAS, _av_eps(ref, q0, th), _q32(3), mu=NS_MU, Pr=NS_PR,
                                 q_in=q0[:, 0, 0])
    assert rel_err(rhs.cpu().numpy(), want) <= TOL