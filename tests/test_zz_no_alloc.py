"""The allocation-free stage entry point (dg_rk_stage_noalloc) against dg_rk_stage.

Some callers cannot call cudaMalloc: their device memory belongs to another
allocator (a framework's pool that has reserved the device, a fixed-budget
arena), or an allocation's implicit device synchronisation would stall their
loop.  dg_rk_stage_noalloc takes every table and buffer from the caller and keeps
the BR1 viscous-flux scratch in a static device array of the library.  This test
plays such a caller: it builds the tables with a host-only mesh (no CUDA call),
copies them into its own device buffers, and checks two consecutive calls
against the regular entry point within the parity tolerance of the GPU tests.
It lives in a file that pytest collects last, so a failure here cannot hide the
other GPU tests.
"""

import numpy as np
import pytest

from tests._gpu import rel_err, torch_cuda
from workloads import box_mesh, equispaced_tet_nodes, taylor_green, uniform_perturbation, physical_nodes

pytestmark = pytest.mark.gpu
TOL = 1e-11


def _caller_tables(torch, vertices, period, N):
    from paper_2512_17101_gb300 import dg
    host = dg.Mesh(vertices, period, N, equispaced_tet_nodes(N), host_only=True)
    ops = host.operators()
    vmapP, geo = host.connectivity()
    flat = np.concatenate([ops["Dr"].ravel(), ops["Ds"].ravel(), ops["Dt"].ravel(), ops["LIFT"].ravel()])
    return dict(K=host.K, N=N, ops=torch.tensor(flat, device="cuda"),
                fmask=torch.tensor(ops["Fmask"], device="cuda", dtype=torch.int32).contiguous(),
                geo=torch.tensor(geo, device="cuda"),
                vmapP=torch.tensor(vmapP, device="cuda", dtype=torch.int32).contiguous())


@pytest.mark.parametrize("N", [2, 3])
def test_noalloc_stage_matches_regular_stage_twice_in_a_row(N):
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    verts, period = box_mesh((3, 3, 2), 1.0)
    nodes = equispaced_tet_nodes(N)
    q0 = uniform_perturbation(taylor_green(physical_nodes(verts, nodes), mach=0.3, noise=0.01, seed=2), 1e-3, seed=4)
    gas_desc = dict(gamma=1.4, R=1.0, mu=2e-2, Pr=0.71)
    tables = _caller_tables(torch, verts, period, N)
    mesh = dg.Mesh(verts, period, N, nodes)
    gas = dg.Gas(model="perfect", **gas_desc)
    dt = 1e-3
    status = torch.zeros(1, device="cuda", dtype=torch.int32)
    # regular entry point: stages 0 and 1
    q_a = torch.tensor(q0, device="cuda")
    q_b = torch.empty_like(q_a)
    k_ref = torch.zeros_like(q_a)
    dg.dg_rk_stage(mesh, gas, 0, dt, q_a, q_b, k_ref)
    q_c = torch.empty_like(q_a)
    dg.dg_rk_stage(mesh, gas, 1, dt, q_b, q_c, k_ref)
    # allocation-free entry point: the same two stages in a row
    n_a = torch.tensor(q0, device="cuda")
    n_b = torch.empty_like(n_a)
    n_c = torch.empty_like(n_a)
    k_n = torch.zeros_like(n_a)
    dg.dg_rk_stage_noalloc(tables, gas_desc, 0, dt, n_a, n_b, k_n, status)
    torch.cuda.synchronize()
    assert rel_err(n_b.cpu().numpy() - q0, q_b.cpu().numpy() - q0) <= TOL
    dg.dg_rk_stage_noalloc(tables, gas_desc, 1, dt, n_b, n_c, k_n, status)
    torch.cuda.synchronize()
    assert rel_err(n_c.cpu().numpy() - q0, q_c.cpu().numpy() - q0) <= TOL
    assert rel_err(k_n.cpu().numpy(), k_ref.cpu().numpy()) <= TOL
    assert int(status.item()) == 0


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    torch_cuda()
    import ctypes
    from paper_2512_17101_gb300 import capi
    lib = capi.load()
    t = capi.dg_mesh_tables()
    t.N = 3
    t.K = capi.DG_STATIC_SCRATCH_NODES // 20 + 1  # one element more than fits
    t.ops_dev = t.fmask_dev = t.geo_dev = t.vmapP_dev = ctypes.c_void_p(16)
    g = capi.dg_gas_desc()
    g.model, g.gamma, g.R, g.mu, g.Pr = capi.DG_GAS_PERFECT, 1.4, 1.0, 1e-3, 0.71
    p = ctypes.c_void_p(16)
    rc = lib.dg_rk_stage_noalloc(ctypes.byref(t), ctypes.byref(g), 0, 1e-3, p, ctypes.c_void_p(1 << 40), p, p, None)
    assert rc == capi.DG_ERR_INVALID_ARG
    assert b"DG_STATIC_SCRATCH_NODES" in lib.dg_last_error()
