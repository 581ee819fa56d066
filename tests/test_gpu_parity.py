"""GPU parity: libdg's CUDA kernels (through the C ABI) against the FP64 oracle.

Bar: max-norm relative error per conserved variable <= 1e-11 for the FP64 path
(rounding-order differences only; both sides compute in float64).
"""

import numpy as np
import pytest

from oracle.euler import rhs_strong
from oracle.lsrk import lsrk4_step
from oracle.ns import rhs_ns
from oracle.thermo import Nasa7Gas, PerfectGas
from tests._gpu import rel_err, torch_cuda
from tests._oracle_case import Disc
from workloads import (box_mesh, equispaced_tet_nodes, isentropic_vortex, taylor_green, uniform_perturbation)
from workloads.gas import mixture_primitive_state, seeded_nasa7_mixture

pytestmark = pytest.mark.gpu
TOL = 1e-11


def _setup(n, N, L=1.0):
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    v, per = box_mesh(n, L)
    d = Disc(v, per, N)
    mesh = dg.Mesh(v, per, N, equispaced_tet_nodes(N))
    return torch, dg, d, mesh


def _vortex(d, noise=1e-3, seed=0):
    q = isentropic_vortex(d.xyz, 0.0, center=(0.45, 0.55), radius=0.15, period=d.period)
    return uniform_perturbation(q, noise, seed=seed)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [1, (3, 2, 2)])
def test_euler_rhs(n, N):
    torch, dg, d, mesh = _setup(n, N)
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0)
    q0 = _vortex(d)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs)
    want = rhs_strong(d.ref, d.geo, d.conn, q0, PerfectGas(1.4, 1.0))
    assert rel_err(rhs.cpu().numpy(), want) <= TOL
    assert mesh.status() == 0


def test_euler_small_config_one_rk4_step():
    """Single-species Euler, 4^3 x 6 = 384 tets, N = 2, vortex + U(+-1e-3), one RK4 step, dt = 1e-3."""
    torch, dg, d, mesh = _setup(4, 2)
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0)
    q0 = isentropic_vortex(d.xyz, 0.0, gamma=1.4, period=d.period)
    q0 = uniform_perturbation(q0, 1e-3, seed=0)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs)
    f = lambda u: rhs_strong(d.ref, d.geo, d.conn, u, PerfectGas(1.4, 1.0))
    assert rel_err(rhs.cpu().numpy(), f(q0)) <= TOL
    dg.lsrk4_step(mesh, gas, q, 1e-3, steps=1)
    want = lsrk4_step(q0, 1e-3, f)
    assert rel_err(q.cpu().numpy() - q0, want - q0) <= TOL  # the step's increment, not the state
    assert rel_err(q.cpu().numpy(), want) <= 1e-13


def test_rk_stage_semantics():
    """Each fused stage equals k <- a k + dt rhs, q_out <- q_in + b k on the oracle side."""
    torch, dg, d, mesh = _setup((2, 3, 2), 3)
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0)
    from oracle.lsrk import RK4A, RK4B
    q0 = _vortex(d, noise=1e-2, seed=4)
    k0 = np.random.default_rng(2).normal(size=q0.shape)
    f = lambda u: rhs_strong(d.ref, d.geo, d.conn, u, PerfectGas(1.4, 1.0))
    for s in range(5):
        q_in = torch.tensor(q0, device="cuda")
        q_out = torch.empty_like(q_in)
        k = torch.tensor(k0, device="cuda")
        dt = 2e-3
        dg.dg_rk_stage(mesh, gas, s, dt, q_in, q_out, k)
        k_want = RK4A[s] * k0 + dt * f(q0)
        assert rel_err(k.cpu().numpy(), k_want) <= TOL
        assert rel_err(q_out.cpu().numpy() - q0, RK4B[s] * k_want) <= TOL


def test_stage_zero_ignores_k_content():
    torch, dg, d, mesh = _setup(2, 2)
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0)
    q0 = _vortex(d)
    q_in = torch.tensor(q0, device="cuda")
    out1, out2 = torch.empty_like(q_in), torch.empty_like(q_in)
    k1 = torch.full_like(q_in, float("nan"))
    k2 = torch.zeros_like(q_in)
    dg.dg_rk_stage(mesh, gas, 0, 1e-3, q_in, out1, k1)
    dg.dg_rk_stage(mesh, gas, 0, 1e-3, q_in, out2, k2)
    assert torch.equal(out1, out2) and torch.equal(k1, k2)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_navier_stokes_rhs(N):
    torch, dg, d, mesh = _setup((3, 2, 2), N)
    mu, Pr = 2e-2, 0.71
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=mu, Pr=Pr)
    q0 = uniform_perturbation(taylor_green(d.xyz, mach=0.3, noise=0.01, seed=1), 1e-3, seed=5)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs)
    want = rhs_ns(d.ref, d.geo, d.conn, q0, PerfectGas(1.4, 1.0), mu, Pr)
    assert rel_err(rhs.cpu().numpy(), want) <= TOL
    assert mesh.status() == 0


def test_navier_stokes_reduced_config_two_steps():
    """The viscous config (TGV Mach 0.1 + 1% noise, mu = 1e-3, Pr = 0.71, N = 3) on 6^3 x 6 tets, 2 RK4 steps."""
    from workloads.configs import _tgv_dt
    torch, dg, d, mesh = _setup(6, 3)
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=1e-3, Pr=0.71)
    q0 = taylor_green(d.xyz, mach=0.1, noise=0.01, seed=0)
    dt = _tgv_dt(6, 3)
    q = torch.tensor(q0, device="cuda")
    dg.lsrk4_step(mesh, gas, q, dt, steps=2)
    f = lambda u: rhs_ns(d.ref, d.geo, d.conn, u, PerfectGas(1.4, 1.0), 1e-3, 0.71)
    want = lsrk4_step(lsrk4_step(q0, dt, f), dt, f)
    assert rel_err(q.cpu().numpy() - q0, want - q0) <= TOL


@pytest.mark.slow
def test_navier_stokes_full_size_stage():
    """Full-size viscous workload (24^3 x 6 = 82,944 tets, N = 3), the stage call the benchmark times."""
    from workloads.configs import get_config, build_case
    cfg = get_config("ns_viscous")
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    case = build_case(cfg)
    d = Disc(case["vertices"], case["period"], cfg.N)
    mesh = dg.Mesh(case["vertices"], case["period"], cfg.N, case["ref_nodes"])
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=1e-3, Pr=0.71)
    q0 = case["q"]
    q_in = torch.tensor(q0, device="cuda")
    q_out = torch.empty_like(q_in)
    k = torch.zeros_like(q_in)
    dg.dg_rk_stage(mesh, gas, 0, cfg.dt, q_in, q_out, k)
    rhs_want = rhs_ns(d.ref, d.geo, d.conn, q0, PerfectGas(1.4, 1.0), 1e-3, 0.71)
    assert rel_err(k.cpu().numpy(), cfg.dt * rhs_want) <= TOL
    assert mesh.status() == 0


def _mixture_setup(n, N, seed=0):
    torch, dg, d, mesh = _setup(n, N)
    mix = seeded_nasa7_mixture(7, seed=seed)
    gas_o = Nasa7Gas(W=mix.W, coeffs=mix.coeffs)
    gas = dg.Gas(model="nasa7", W=mix.W, nasa7=mix.coeffs, newton_tol=1e-10, newton_max_it=50)
    Y, T, vel, p0 = mixture_primitive_state(d.xyz, 7, seed=seed)
    rho = p0 / (gas_o.R_mix(Y) * T)
    q0 = gas_o.conserved(rho, vel, Y, T)
    return torch, dg, d, mesh, gas, gas_o, q0, T


def test_temperature_newton():
    torch, dg, d, mesh, gas, gas_o, q0, T_true = _mixture_setup(3, 2)
    n = q0.shape[1] * q0.shape[2]
    q = torch.tensor(q0.reshape(q0.shape[0], n), device="cuda")
    T = torch.full((n,), 1500.0, device="cuda", dtype=torch.float64)
    it = torch.zeros(n, device="cuda", dtype=torch.int32)
    dg.dg_temperature(gas, q, T, it)
    rho, vel, Y, e = gas_o.split_state(q0.reshape(q0.shape[0], n))
    Tw, itw, ok = gas_o.newton_temperature(e, Y, np.full(n, 1500.0))
    assert ok.all() and gas.status() == 0
    assert np.abs(T.cpu().numpy() - Tw).max() < 1e-9
    assert np.abs(T.cpu().numpy() - T_true.ravel()).max() < 1e-8
    assert np.abs(it.cpu().numpy() - itw).max() <= 1


def test_mixture_energy_inverts_temperature():
    torch, dg, d, mesh, gas, gas_o, q0, T_true = _mixture_setup(2, 1)
    rng = np.random.default_rng(3)
    n = 4096
    T = rng.uniform(300, 3000, n)
    Y = rng.dirichlet(np.ones(7), size=n).T.copy()
    e = torch.empty(n, device="cuda", dtype=torch.float64)
    dg.dg_mixture_energy(gas, torch.tensor(T, device="cuda"), torch.tensor(Y, device="cuda"), e)
    want = gas_o.mixture_e(T, Y)
    assert np.abs(e.cpu().numpy() - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("N", [1, 2, 3])
def test_mixture_rhs(N):
    # a 3^3 box: on a 2-cell lattice sin(2 pi y) vanishes at every N=1 node and the x/y-momentum
    # right-hand side degenerates to rounding noise of the uniform pressure
    torch, dg, d, mesh, gas, gas_o, q0, T_true = _mixture_setup(3, N, seed=1)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    T = torch.full(q0.shape[1:], 1650.0, device="cuda", dtype=torch.float64)
    dg.dg_rhs(mesh, gas, q, rhs, T_io=T)
    rho, vel, Y, e = gas_o.split_state(q0)
    Tw, _, ok = gas_o.newton_temperature(e, Y, np.full(e.shape, 1650.0))
    want = rhs_strong(d.ref, d.geo, d.conn, q0, gas_o, T=Tw)
    assert ok.all()
    assert np.abs(T.cpu().numpy() - Tw).max() < 1e-9
    got = rhs.cpu().numpy()
    per_var = [float(np.abs(got[v] - want[v]).max() / np.abs(want[v]).max()) for v in range(want.shape[0])]
    worst = np.unravel_index(np.argmax(np.abs(got[4] - want[4])), want[4].shape)
    assert rel_err(got, want) <= TOL, (per_var, worst, got[:, worst[0], worst[1]], want[:, worst[0], worst[1]])


def test_status_flags_without_fault():
    torch, dg, d, mesh = _setup(2, 1)
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0)
    q0 = _vortex(d)
    q0[0, 3, 1] = -1.0  # negative density at one node
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs)
    from paper_2512_17101_gb300 import capi
    assert mesh.status() & capi.DG_STATUS_NONPHYSICAL
    assert mesh.status() == 0  # cleared by the previous read
    # Newton capped at one update
    mix = seeded_nasa7_mixture(7, seed=0)
    g2 = dg.Gas(model="nasa7", W=mix.W, nasa7=mix.coeffs, newton_tol=1e-10, newton_max_it=1)
    gas_o = Nasa7Gas(W=mix.W, coeffs=mix.coeffs)
    Y = np.full((7, 8), 1 / 7)
    T = np.full(8, 2500.0)
    qm = gas_o.conserved(np.ones(8), np.zeros((3, 8)), Y, T)
    Tt = torch.full((8,), 300.0, device="cuda", dtype=torch.float64)
    dg.dg_temperature(g2, torch.tensor(qm, device="cuda"), Tt)
    assert g2.status() & capi.DG_STATUS_NO_CONVERGENCE


def test_bitwise_deterministic():
    torch, dg, d, mesh = _setup((3, 3, 2), 3)
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=1e-3, Pr=0.71)
    q = torch.tensor(uniform_perturbation(taylor_green(d.xyz, mach=0.2), 1e-3, seed=7), device="cuda")
    a, b = torch.empty_like(q), torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, a)
    dg.dg_rhs(mesh, gas, q, b)
    assert torch.equal(a, b)


def test_overlapping_output_rejected():
    torch, dg, d, mesh = _setup(1, 1)
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0)
    q = torch.tensor(_vortex(d), device="cuda")
    from paper_2512_17101_gb300.capi import DGError
    with pytest.raises(DGError):
        dg.dg_rhs(mesh, gas, q, q)


def test_discrete_conservation_on_gpu():
    torch, dg, d, mesh = _setup(3, 3)
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=5e-3, Pr=0.71)
    q = torch.tensor(uniform_perturbation(taylor_green(d.xyz, mach=0.3), 1e-2, seed=3), device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs)
    r = rhs.cpu().numpy()
    assert np.all(np.abs(d.integrate(r)) <= 1e-12 * d.abs_integral(r))


@pytest.mark.slow
def test_mixture_learned_full_size_stage():
    """Full-size learned-form workload (32^3 x 6 = 196,608 tets, N = 2, 7 species): the FP64 stage
    against the oracle, temperatures from Newton on both sides."""
    from workloads.configs import build_case, get_config
    cfg = get_config("mixture_learned")
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    case = build_case(cfg)
    d = Disc(case["vertices"], case["period"], cfg.N)
    mesh = dg.Mesh(case["vertices"], case["period"], cfg.N, case["ref_nodes"])
    mix = case["mixture"]
    gas_o = Nasa7Gas(W=mix.W, coeffs=mix.coeffs)
    gas = dg.Gas(model="nasa7", W=mix.W, nasa7=mix.coeffs, newton_tol=1e-10, newton_max_it=50)
    rho = case["p0"] / (gas_o.R_mix(case["Y"]) * case["T"])
    q0 = gas_o.conserved(rho, case["vel"], case["Y"], case["T"])
    q_in = torch.tensor(q0, device="cuda")
    q_out, k = torch.empty_like(q_in), torch.zeros_like(q_in)
    T = torch.full(q0.shape[1:], 1650.0, device="cuda", dtype=torch.float64)
    dg.dg_rk_stage(mesh, gas, 0, cfg.dt, q_in, q_out, k, T_io=T)
    _, _, Y, e = gas_o.split_state(q0)
    Tw, _, ok = gas_o.newton_temperature(e, Y, np.full(e.shape, 1650.0))
    assert ok.all()
    rhs_want = rhs_strong(d.ref, d.geo, d.conn, q0, gas_o, T=Tw)
    assert rel_err(k.cpu().numpy(), cfg.dt * rhs_want) <= TOL
    assert mesh.status() == 0 and gas.status() == 0
