"""The allocation-free stage entry point (dg_rk_stage_noalloc) against dg_rk_stage.

Some callers cannot call cudaMalloc: their device memory belongs to another
allocator (a framework's pool that has reserved the device, a fixed-budget
arena), or an allocation's implicit device synchronisation would stall their
loop.  dg_rk_stage_noalloc takes every table and buffer from the caller and keeps
the BR1 viscous-flux scratch in a static device array of the library.  These
tests play such a caller: they build the tables with a host-only mesh (no CUDA
call), copy them into their own device buffers, and check two consecutive calls
against the regular entry point within the parity tolerance of the GPU tests,
at every order, on a box with wall and outflow faces, and on a mesh close to the
static array's node limit.  The file is collected last, so a failure here cannot
hide the other GPU tests.
"""

import numpy as np
import pytest

from tests._gpu import rel_err, torch_cuda
from workloads import box_mesh, equispaced_tet_nodes, taylor_green, uniform_perturbation, physical_nodes
from workloads.mesh import box_face_bc

pytestmark = pytest.mark.gpu
TOL = 1e-11
SLIP, NOSLIP, INFLOW, OUTFLOW = 1, 2, 3, 4
GAS_DESC = dict(gamma=1.4, R=1.0, mu=2e-2, Pr=0.71)


def _caller_tables(torch, vertices, period, N, face_bc=None):
    from paper_2512_17101_gb300 import dg
    host = dg.Mesh(vertices, period, N, equispaced_tet_nodes(N), host_only=True, face_bc=face_bc)
    ops = host.operators()
    vmapP, geo = host.connectivity()
    flat = np.concatenate([ops["Dr"].ravel(), ops["Ds"].ravel(), ops["Dt"].ravel(), ops["LIFT"].ravel()])
    return dict(K=host.K, N=N, ops=torch.tensor(flat, device="cuda"),
                fmask=torch.tensor(ops["Fmask"], device="cuda", dtype=torch.int32).contiguous(),
                geo=torch.tensor(geo, device="cuda"),
                vmapP=torch.tensor(vmapP, device="cuda", dtype=torch.int32).contiguous())


def _walled_box(n, sides):
    verts, period = box_mesh(n, 1.0)
    period = np.array(period, dtype=float)
    for axis, _ in sides:
        period[axis] = 0.0
    return verts, period, box_face_bc(verts, 1.0, sides=sides)


def _two_stages_both_ways(verts, period, N, face_bc=None, mach=0.3, tol=TOL):
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    nodes = equispaced_tet_nodes(N)
    q0 = uniform_perturbation(taylor_green(physical_nodes(verts, nodes), mach=mach, noise=0.01, seed=2), 1e-3,
                              seed=4)
    tables = _caller_tables(torch, verts, period, N, face_bc)
    mesh = dg.Mesh(verts, period, N, nodes, face_bc=face_bc)
    gas = dg.Gas(model="perfect", **GAS_DESC)
    dt = 1e-3
    status = torch.zeros(1, device="cuda", dtype=torch.int32)
    # regular entry point: stages 0 and 1
    q_a = torch.tensor(q0, device="cuda")
    q_b = torch.empty_like(q_a)
    k_ref = torch.zeros_like(q_a)
    dg.dg_rk_stage(mesh, gas, 0, dt, q_a, q_b, k_ref)
    q_c = torch.empty_like(q_a)
    dg.dg_rk_stage(mesh, gas, 1, dt, q_b, q_c, k_ref)
    assert mesh.status() == 0
    # allocation-free entry point: the same two stages in a row
    n_a = torch.tensor(q0, device="cuda")
    n_b = torch.empty_like(n_a)
    n_c = torch.empty_like(n_a)
    k_n = torch.zeros_like(n_a)
    dg.dg_rk_stage_noalloc(tables, GAS_DESC, 0, dt, n_a, n_b, k_n, status)
    torch.cuda.synchronize()
    assert rel_err(n_b.cpu().numpy() - q0, q_b.cpu().numpy() - q0) <= tol
    dg.dg_rk_stage_noalloc(tables, GAS_DESC, 1, dt, n_b, n_c, k_n, status)
    torch.cuda.synchronize()
    assert rel_err(n_c.cpu().numpy() - q0, q_c.cpu().numpy() - q0) <= tol
    assert rel_err(k_n.cpu().numpy(), k_ref.cpu().numpy()) <= tol
    assert int(status.item()) == 0


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_noalloc_stage_matches_regular_stage_twice_in_a_row(N):
    verts, period = box_mesh((3, 3, 2), 1.0)
    _two_stages_both_ways(verts, period, N)


@pytest.mark.parametrize("N", [2, 3])
def test_noalloc_stage_with_wall_and_outflow_faces(N):
    """Slip and no-slip walls across y, outflow faces across x, periodic in z."""
    verts, period, face_bc = _walled_box((3, 3, 2), {(0, 0): OUTFLOW, (0, 1): OUTFLOW, (1, 0): NOSLIP,
                                                     (1, 1): SLIP})
    _two_stages_both_ways(verts, period, N, face_bc=face_bc)


def test_noalloc_stage_near_the_node_limit():
    """16^3 x 6 = 24,576 tetrahedra at N = 3: 491,520 nodes, 94 % of DG_STATIC_SCRATCH_NODES."""
    from paper_2512_17101_gb300 import capi
    verts, period = box_mesh(16, 1.0)
    assert 0.9 * capi.DG_STATIC_SCRATCH_NODES < verts.shape[0] * 20 <= capi.DG_STATIC_SCRATCH_NODES
    _two_stages_both_ways(verts, period, 3, mach=0.1)


def test_noalloc_inflow_faces_are_flagged_nonphysical():
    """The entry point carries no inflow state: an inflow face's ghost density is zero, and the stage
    reports it through the status word (no fault, no trap)."""
    torch = torch_cuda()
    from paper_2512_17101_gb300 import capi, dg
    verts, period, face_bc = _walled_box((3, 3, 2), {(0, 0): INFLOW, (0, 1): OUTFLOW})
    nodes = equispaced_tet_nodes(2)
    q0 = taylor_green(physical_nodes(verts, nodes), mach=0.3, noise=0.01, seed=2)
    tables = _caller_tables(torch, verts, period, 2, face_bc)
    status = torch.zeros(1, device="cuda", dtype=torch.int32)
    q = torch.tensor(q0, device="cuda")
    out, k = torch.empty_like(q), torch.zeros_like(q)
    dg.dg_rk_stage_noalloc(tables, GAS_DESC, 0, 1e-3, q, out, k, status)
    torch.cuda.synchronize()
    assert int(status.item()) & capi.DG_STATUS_NONPHYSICAL


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
