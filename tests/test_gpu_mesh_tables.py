"""A mesh uploaded from the caller's own tables (element-local arrays and connectivity data,
Sec. 1 Fig. 1, Sec. 4.1.2), with its elements relabelled, gives the oracle's right-hand side and RK
stage at 1e-11 per conserved variable (after undoing the relabelling)."""

import numpy as np
import pytest

from oracle.euler import rhs_strong
from oracle.ns import rhs_ns
from oracle.thermo import PerfectGas
from tests._gpu import rel_err, torch_cuda
from tests._oracle_case import Disc
from tests.test_mesh_tables import relabelled_tables
from workloads import box_mesh, physical_nodes, taylor_green, uniform_perturbation

pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.mark.parametrize("N,viscous", [(1, False), (2, True), (3, True), (4, False)])
def test_relabelled_caller_tables_match_oracle(N, viscous):
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    v2, period, nodes, t, new_of_old = relabelled_tables(N, seed=7 + N)
    mesh = dg.Mesh(v2, period, N, nodes, tables=t)
    mu = 2e-2 if viscous else 0.0
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=mu, Pr=0.71)
    verts, _ = box_mesh((3, 2, 2), 1.0)
    d = Disc(verts, period, N)
    q0 = uniform_perturbation(taylor_green(physical_nodes(verts, nodes), mach=0.3, noise=0.01, seed=3), 1e-3, seed=5)
    g = PerfectGas(1.4, 1.0)
    want = rhs_ns(d.ref, d.geo, d.conn, q0, g, mu, 0.71) if viscous else rhs_strong(d.ref, d.geo, d.conn, q0, g)
    q = torch.tensor(np.ascontiguousarray(q0[:, np.argsort(new_of_old)]), device="cuda")  # relabelled state
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs)
    got = rhs.cpu().numpy()[:, new_of_old]                          # back to the original labels
    assert rel_err(got, want) <= TOL
    assert mesh.status() == 0
