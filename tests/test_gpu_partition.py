"""GPU parity of the partitioned form (paper_2512_17101_gb300/partition.py): partitions of one
mesh held on one device, each with its halo elements, the halos refreshed before every stage by
the library's gather / scatter kernels with the buffers handed between partitions on the host
(LocalRouter: no kernel waits on another).  Two LSRK4 steps at the owned elements against the
unpartitioned mesh on the GPU and against the oracle, Euler and Navier-Stokes, periodic and with
walls and inflow / outflow faces."""

import numpy as np
import pytest

import oracle.boundary as bd
from oracle.lsrk import lsrk4_step
from oracle.thermo import PerfectGas
from tests._gpu import rel_err, torch_cuda
from tests._oracle_case import Disc, bc_disc
from workloads import box_mesh, equispaced_tet_nodes, isentropic_vortex, uniform_perturbation

pytestmark = pytest.mark.gpu
GAS = PerfectGas(1.4, 1.0)
MU, PR = 2e-2, 0.71
Q_IN = np.array([1.1, 1.98, 0.055, -0.022, 0.75 / 0.4 + 0.5 * 1.1 * (1.8 ** 2 + 0.05 ** 2 + 0.02 ** 2)])

CASES = {
    "euler_periodic_3": (False, None, 3),
    "ns_periodic_2": (True, None, 2),
    "ns_walls_3": (True, {(1, 0): bd.NOSLIP_WALL, (1, 1): bd.SLIP_WALL}, 3),
    "euler_in_out_4": (False, {(0, 0): bd.INFLOW, (0, 1): bd.OUTFLOW, (1, 0): bd.SLIP_WALL,
                               (1, 1): bd.SLIP_WALL}, 4),
}


def _disc(sides, N):
    n = (4, 3, 2)
    if sides is None:
        v, per = box_mesh(n, 1.0)
        return Disc(v, per, N)
    return bc_disc(n, N, sides)


def _flow(d):
    q = isentropic_vortex(d.xyz, 0.0, period=np.where(np.asarray(d.period) > 0, d.period, 1.0))
    return uniform_perturbation(q, 1e-3, seed=5)


@pytest.mark.parametrize("N", [2, 3])
@pytest.mark.parametrize("name", list(CASES))
def test_partitioned_steps_match_the_whole_mesh(name, N):
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    from paper_2512_17101_gb300.partition import HaloExchange, LocalRouter, RankState, partition_mesh
    viscous, sides, nparts = CASES[name]
    d = _disc(sides, N)
    nodes = equispaced_tet_nodes(N)
    inflow = sides is not None and bd.INFLOW in sides.values()
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=MU if viscous else 0.0, Pr=PR)
    q0 = _flow(d)
    dt = 2e-3

    whole = dg.Mesh(d.vertices, d.period, N, nodes, face_bc=d.face_bc)
    if inflow:
        whole.set_inflow(Q_IN)
    qw = torch.tensor(q0, device="cuda")
    dg.lsrk4_step(whole, gas, qw, dt, steps=2)

    ranks, parts = [], partition_mesh(d.vertices, d.period, N, nodes, nparts, face_bc=d.face_bc)
    for p in parts:
        m = dg.Mesh(p.vertices, d.period, N, nodes, face_bc=p.face_bc)
        m.set_inflow(Q_IN)  # the halo's outer faces are outflow faces; inflow faces may be there too
        q = torch.tensor(np.ascontiguousarray(q0[:, p.local]), device="cuda")
        q[:, len(p.owned):] = float("nan")  # nothing may read the halo before its first refresh
        ranks.append(RankState(m, HaloExchange(p, m.Np, q.device), q, (torch.empty_like(q), torch.zeros_like(q))))
    from paper_2512_17101_gb300.partition import partitioned_lsrk4_step
    for _ in range(2):
        partitioned_lsrk4_step(ranks, gas, LocalRouter(), dt)

    got = np.empty_like(q0)
    for p, r in zip(parts, ranks):
        got[:, p.owned] = r.q.cpu().numpy()[:, :len(p.owned)]
    ref = qw.cpu().numpy()
    # the same arithmetic node by node: equal to the whole mesh's step up to rounding
    assert rel_err(got - q0, ref - q0) <= 1e-12
    f = (lambda u: bd.rhs_ns_bc(d.ref, d.geo, d.conn, u, GAS, MU, PR, q_in=Q_IN)) if viscous else \
        (lambda u: bd.rhs_euler_bc(d.ref, d.geo, d.conn, u, GAS, q_in=Q_IN))
    want = lsrk4_step(lsrk4_step(q0, dt, f), dt, f)
    assert rel_err(got - q0, want - q0) <= 1e-11
    for r in ranks:
        assert r.mesh.status() == 0


def test_gather_scatter_round_trip():
    torch = torch_cuda()
    from paper_2512_17101_gb300 import capi
    import ctypes
    V, K, Np = 9, 37, 10
    x = torch.randn(V, K, Np, dtype=torch.float64, device="cuda")
    ix = torch.tensor([36, 0, 5, 17, 18], dtype=torch.int32, device="cuda")
    buf = torch.empty(V, len(ix), Np, dtype=torch.float64, device="cuda")
    lib = capi.load()
    capi.check(lib.dg_gather_elements(ctypes.c_void_p(x.data_ptr()), V, K, Np, ctypes.c_void_p(ix.data_ptr()),
                                      len(ix), ctypes.c_void_p(buf.data_ptr()), None))
    assert torch.equal(buf, x[:, ix.long()])
    y = torch.zeros_like(x)
    capi.check(lib.dg_scatter_elements(ctypes.c_void_p(buf.data_ptr()), V, K, Np, ctypes.c_void_p(ix.data_ptr()),
                                       len(ix), ctypes.c_void_p(y.data_ptr()), None))
    torch.cuda.synchronize()
    want = torch.zeros_like(x)
    want[:, ix.long()] = x[:, ix.long()]
    assert torch.equal(y, want)
    # an index outside [0, K) is skipped by the kernels; bad sizes are refused on the host
    bad = torch.tensor([0, K, -1], dtype=torch.int32, device="cuda")
    buf3 = torch.full((V, 3, Np), 7.0, dtype=torch.float64, device="cuda")
    capi.check(lib.dg_gather_elements(ctypes.c_void_p(x.data_ptr()), V, K, Np, ctypes.c_void_p(bad.data_ptr()),
                                      3, ctypes.c_void_p(buf3.data_ptr()), None))
    torch.cuda.synchronize()
    assert torch.equal(buf3[:, 0], x[:, 0]) and bool((buf3[:, 1:] == 7.0).all())
    with pytest.raises(capi.DGError):
        capi.check(lib.dg_gather_elements(ctypes.c_void_p(x.data_ptr()), 0, K, Np, ctypes.c_void_p(ix.data_ptr()),
                                          len(ix), ctypes.c_void_p(buf.data_ptr()), None))
