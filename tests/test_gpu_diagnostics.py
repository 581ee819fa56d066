"""GPU parity of the global reductions (csrc/k_diag.cu) through the C ABI against the oracle
(oracle/diagnostics.py): conservation integrals and the stability rate, over whole meshes, over
leading element ranges and over partitions combined with the in-process router."""

import numpy as np
import pytest

import oracle.diagnostics as dgn
from oracle.thermo import PerfectGas
from tests._gpu import torch_cuda
from tests._oracle_case import Disc
from workloads import box_mesh, equispaced_tet_nodes, isentropic_vortex, uniform_perturbation

pytestmark = pytest.mark.gpu
GAS = PerfectGas(1.4, 1.0)


def _setup(n, N, mu=0.0, L=1.0):
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    v, per = box_mesh(n, L)
    d = Disc(v, per, N)
    mesh = dg.Mesh(v, per, N, equispaced_tet_nodes(N))
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=mu, Pr=0.71)
    q = uniform_perturbation(isentropic_vortex(d.xyz, 0.0, period=d.period), 1e-2, seed=N)
    return torch, dg, d, mesh, gas, q


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_integrals_match_the_oracle(N):
    torch, dg, d, mesh, gas, q0 = _setup((4, 3, 3), N, L=1.7)
    q = torch.tensor(q0, device="cuda")
    scale = dgn.integrals(d.ref, d.geo, np.abs(q0))
    got = dg.dg_integrals(mesh, q).cpu().numpy()
    assert np.all(np.abs(got - dgn.integrals(d.ref, d.geo, q0)) <= 1e-14 * scale)
    for kc in (0, 1, 37, d.K - 1):  # leading element ranges
        got = dg.dg_integrals(mesh, q, nvar=3, K_count=kc).cpu().numpy()
        want = np.einsum("vki,i,k->v", q0[:3, :kc], dgn.mass_weights(d.ref), d.geo.J[:kc])
        assert np.all(np.abs(got - want) <= 1e-14 * scale[:3]), kc
    again = dg.dg_integrals(mesh, q).cpu().numpy()
    assert np.array_equal(again, dg.dg_integrals(mesh, q).cpu().numpy())  # fixed reduction order


@pytest.mark.parametrize("N", [1, 3, 4])
@pytest.mark.parametrize("mu", [0.0, 0.02])
def test_stability_rate_matches_the_oracle(N, mu):
    torch, dg, d, mesh, gas, q0 = _setup((3, 4, 2), N, mu=mu)
    q = torch.tensor(q0, device="cuda")
    want = dgn.max_rate(d.ref, d.geo, q0, GAS, mu, 0.71)
    got = float(dg.dg_max_rate(mesh, gas, q).item())
    assert abs(got - want) <= 1e-14 * want
    rates = dgn.element_rates(d.ref, d.geo, q0, GAS, mu, 0.71)
    for kc in (1, 50, d.K):
        assert abs(float(dg.dg_max_rate(mesh, gas, q, K_count=kc).item()) - rates[:kc].max()) <= 1e-14 * want
    assert float(dg.dg_max_rate(mesh, gas, q, K_count=0).item()) == 0.0
    assert abs(dg.stable_dt(mesh, gas, q, 0.5) - 0.5 / want) <= 1e-14 / want
    assert mesh.status() == 0


def test_rate_closed_form_and_a_nonphysical_node():
    torch, dg, d, mesh, gas, q0 = _setup(4, 2, mu=0.03)
    rho, u, p = 1.3, np.array([0.4, -0.2, 0.1]), 0.9
    qu = np.empty_like(q0)
    qu[0] = rho
    qu[1:4] = (rho * u)[:, None, None]
    qu[4] = p / 0.4 + 0.5 * rho * (u @ u)
    h = 0.25
    speed = np.linalg.norm(u) + np.sqrt(1.4 * p / rho)
    want = 9 * np.sqrt(2.0) * speed / h + 81 * 2.0 * (0.03 / rho * (1.4 / 0.71)) / h ** 2
    q = torch.tensor(qu, device="cuda")
    assert abs(float(dg.dg_max_rate(mesh, gas, q).item()) - want) <= 1e-13 * want
    qb = qu.copy()
    qb[4, 5, 2] = 0.1 * qb[4, 5, 2] - 0.5  # negative pressure at one node
    r = float(dg.dg_max_rate(mesh, gas, torch.tensor(qb, device="cuda")).item())
    from paper_2512_17101_gb300 import capi
    assert r == float("inf") and mesh.status() & capi.DG_STATUS_NONPHYSICAL


def test_mixtures_and_bad_ranges_are_refused():
    torch, dg, d, mesh, gas, q0 = _setup(2, 1)
    from paper_2512_17101_gb300 import capi
    q = torch.tensor(q0, device="cuda")
    with pytest.raises(capi.DGError):
        dg.dg_integrals(mesh, q, K_count=d.K + 1)
    with pytest.raises(capi.DGError):
        dg.dg_max_rate(mesh, gas, q, K_count=-1)
    from workloads.gas import seeded_nasa7_mixture
    m7 = seeded_nasa7_mixture(3, seed=0)
    mix = dg.Gas(model="nasa7", W=m7.W, nasa7=m7.coeffs)
    with pytest.raises(capi.DGError):
        dg.dg_max_rate(mesh, mix, q)


@pytest.mark.parametrize("mu", [0.0, 0.02])
def test_rk_steps_conserve_on_the_gpu(mu):
    torch, dg, d, mesh, gas, q0 = _setup((3, 3, 2), 3, mu=mu)
    q = torch.tensor(q0, device="cuda")
    before = dg.dg_integrals(mesh, q).cpu().numpy()
    dt = dg.stable_dt(mesh, gas, q, 0.5)
    dg.lsrk4_step(mesh, gas, q, dt, steps=3)
    after = dg.dg_integrals(mesh, q).cpu().numpy()
    scale = dgn.integrals(d.ref, d.geo, np.abs(q0))
    assert np.all(np.abs(after - before) <= 1e-13 * scale), (after - before) / scale


def test_partitioned_reductions_equal_the_whole_mesh():
    torch, dg, d, mesh, gas, q0 = _setup((4, 3, 2), 2, mu=0.01)
    from paper_2512_17101_gb300.partition import (HaloExchange, LocalRouter, RankState, partition_mesh,
                                                  partitioned_integrals, partitioned_stable_dt)
    nodes = equispaced_tet_nodes(2)
    ranks = []
    for p in partition_mesh(d.vertices, d.period, 2, nodes, 3):
        m = dg.Mesh(p.vertices, d.period, 2, nodes, face_bc=p.face_bc)
        qq = torch.tensor(np.ascontiguousarray(q0[:, p.local]), device="cuda")
        ranks.append(RankState(m, HaloExchange(p, m.Np, qq.device), qq, ()))
    q = torch.tensor(q0, device="cuda")
    whole = dg.dg_integrals(mesh, q).cpu().numpy()
    scale = dgn.integrals(d.ref, d.geo, np.abs(q0))
    for t in partitioned_integrals(ranks, LocalRouter()):
        assert np.all(np.abs(t.cpu().numpy() - whole) <= 1e-14 * scale)
    assert partitioned_stable_dt(ranks, gas, LocalRouter(), 0.4) == dg.stable_dt(mesh, gas, q, 0.4)
