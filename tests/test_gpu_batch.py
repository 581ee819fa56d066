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
