"""Batched form: uneven cases of orders 1..4, Euler and Navier-Stokes, advanced together by one
graph launch per RK4 step; per case identical to the single-case mixed stages, and within the
precision form's error of the FP64 oracle."""

import numpy as np
import pytest

from oracle.euler import rhs_strong
from oracle.lsrk import lsrk4_step
from oracle.ns import rhs_ns
from oracle.thermo import PerfectGas
from tests._gpu import component_err, field_err, torch_cuda
from tests._oracle_case import Disc
from workloads.configs import batched_cases

pytestmark = pytest.mark.gpu


def _small_batch():
    cases = batched_cases(ncases=12, seed=3, n_min=2, n_max=4)
    assert {c["N"] for c in cases} == {1, 2, 3, 4}
    return cases


def _handles(torch, dg, cases):
    out = []
    for c in cases:
        mesh = dg.Mesh(c["vertices"], c["period"], c["N"], c["ref_nodes"])
        g = c["gas"]
        gas = dg.Gas(model="perfect", gamma=g.gamma, R=g.R, mu=g.mu, Pr=g.Pr)
        out.append((mesh, gas, c["dt"], torch.tensor(c["q"], device="cuda")))
    return out


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_equals_single_case_stages(autotune):
    torch = torch_cuda()
    from paper_2512_17101_gb300 import capi, dg
    cases = _small_batch()
    hs = _handles(torch, dg, cases)
    batch = dg.Batch(hs, autotune=autotune)
    # reference: the same mixed stages, case by case through dg_rk_stage
    refs = []
    opts = dg._opts(precision=capi.DG_PREC_MIXED)
    for (mesh, gas, dt, q), c in zip(hs, cases):
        qr = torch.tensor(c["q"], device="cuda")
        dg.lsrk4_step(mesh, gas, qr, dt, steps=2, opts=opts)
        refs.append(qr)
    batch.step(2)
    torch.cuda.synchronize()
    assert batch.status() == 0
    for (mesh, gas, dt, q), qr in zip(hs, refs):
        # per row the batched tiles do the same arithmetic as the single-case kernels
        assert float((q - qr).abs().max()) <= 1e-12 * float(qr.abs().max())
    rt, vt, _ = batch.tiles()
    for c in cases:
        assert rt[c["N"] - 1, int(c["viscous"])] > 0
        if c["viscous"]:
            assert vt[c["N"] - 1] > 0


def test_batch_against_oracle():
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    # N >= 2: at N = 1 on 2-cell boxes every node sits where the Taylor-Green velocity vanishes
    cases = [c for c in _small_batch() if c["n"] <= 3 and c["N"] >= 2][:4]
    assert {c["viscous"] for c in cases} == {False, True}
    hs = _handles(torch, dg, cases)
    batch = dg.Batch(hs, autotune=True)
    batch.step(1)
    torch.cuda.synchronize()
    for (mesh, gas, dt, q), c in zip(hs, cases):
        d = Disc(c["vertices"], c["period"], c["N"])
        g = c["gas"]
        if c["viscous"]:
            f = lambda u: rhs_ns(d.ref, d.geo, d.conn, u, PerfectGas(g.gamma, g.R), g.mu, g.Pr)
        else:
            f = lambda u: rhs_strong(d.ref, d.geo, d.conn, u, PerfectGas(g.gamma, g.R))
        want = lsrk4_step(c["q"], dt, f)
        assert field_err(q.cpu().numpy(), want) <= 1e-6
        assert component_err(q.cpu().numpy(), want) <= 1e-4


@pytest.mark.slow
def test_full_batched_workload_equals_single_case_stages():
    """The benchmark's batch (64 cases, n ~ U{2..20}, N ~ U{1..4}, seed 0), autotuned: one graph
    launch per RK4 step equals the same mixed stages case by case."""
    torch = torch_cuda()
    from paper_2512_17101_gb300 import capi, dg
    cases = batched_cases(ncases=64, seed=0)
    hs = _handles(torch, dg, cases)
    batch = dg.Batch(hs, autotune=True)
    opts = dg._opts(precision=capi.DG_PREC_MIXED)
    refs = []
    for (mesh, gas, dt, q), c in zip(hs, cases):
        qr = torch.tensor(c["q"], device="cuda")
        dg.lsrk4_step(mesh, gas, qr, dt, steps=1, opts=opts)
        refs.append(qr)
    batch.step(1)
    torch.cuda.synchronize()
    assert batch.status() == 0
    for (mesh, gas, dt, q), qr in zip(hs, refs):
        assert float((q - qr).abs().max()) <= 1e-12 * float(qr.abs().max())


def test_batch_with_boundary_faces_equals_single_case_stages():
    """Cases with slip and no-slip walls and inflow / outflow faces (ghost node records) in one
    batch with a periodic case: each equals its single-case mixed stages."""
    torch = torch_cuda()
    from paper_2512_17101_gb300 import capi, dg
    from tests.test_gpu_boundary import Q_IN, SIDES, _smooth
    from tests._oracle_case import bc_disc
    from workloads import equispaced_tet_nodes
    specs = [((3, 3, 2), 2, "noslip_y_slip_z", 2e-2), ((3, 3, 2), 3, "in_out_x_walls_y", 0.0),
             ((3, 3, 2), 3, "slip_y", 2e-2), ((3, 3, 2), 2, None, 0.0)]
    hs, q0s = [], []
    for n, N, sides, mu in specs:
        if sides is None:
            from workloads import box_mesh
            v, per = box_mesh(n, 1.0)
            mesh = dg.Mesh(v, per, N, equispaced_tet_nodes(N))
            xyz = Disc(v, per, N).xyz
        else:
            d = bc_disc(n, N, SIDES[sides])
            mesh = dg.Mesh(d.vertices, d.period, N, equispaced_tet_nodes(N), face_bc=d.face_bc)
            if "in_out" in sides:
                mesh.set_inflow(Q_IN)
            xyz = d.xyz
        gas = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=mu, Pr=0.71)
        q0 = _smooth(xyz, seed=len(hs))
        q0s.append(q0)
        hs.append((mesh, gas, 1e-3, torch.tensor(q0, device="cuda")))
    batch = dg.Batch(hs, autotune=False)
    opts = dg._opts(precision=capi.DG_PREC_MIXED)
    refs = []
    for (mesh, gas, dt, _), q0 in zip(hs, q0s):
        qr = torch.tensor(q0, device="cuda")
        dg.lsrk4_step(mesh, gas, qr, dt, steps=2, opts=opts)
        refs.append(qr)
    batch.step(2)
    torch.cuda.synchronize()
    assert batch.status() == 0
    for (mesh, gas, dt, q), qr in zip(hs, refs):
        assert mesh.status() == 0
        assert float((q - qr).abs().max()) <= 1e-12 * float(qr.abs().max())


def test_batch_needs_the_inflow_state():
    torch = torch_cuda()
    from paper_2512_17101_gb300 import capi, dg
    from tests.test_gpu_boundary import SIDES, _smooth
    from tests._oracle_case import bc_disc
    from workloads import equispaced_tet_nodes
    d = bc_disc((3, 3, 2), 2, SIDES["in_out_x_walls_y"])
    mesh = dg.Mesh(d.vertices, d.period, 2, equispaced_tet_nodes(2), face_bc=d.face_bc)
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0)
    with pytest.raises(capi.DGError) as e:
        dg.Batch([(mesh, gas, 1e-3, torch.tensor(_smooth(d.xyz), device="cuda"))], autotune=False)
    assert e.value.code == capi.DG_ERR_INVALID_ARG
