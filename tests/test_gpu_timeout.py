"""Bounded waits of the tensor-core kernels: a wait that runs out is reported, not hung on.

Every wait of a tcgen05 kernel for its MMA completion has an iteration bound.  dg_opts.wait_polls
shrinks that bound to a few polls of the non-blocking test, which run out before the tensor core
can finish: the kernels then set DG_STATUS_TIMEOUT, stop at their next issue point, wait once more
with the full bound for the MMA in flight, free their tensor memory and return.  The tests check
the status bit and that the device stays usable: the same call with the default bound afterwards
runs its tensor-core kernels again (they allocate tensor memory, which a leak would withhold) and
gives the right answer.  No fault, trap or endless loop is involved.
"""

import numpy as np
import pytest

from tests._gpu import field_err, torch_cuda
from workloads import box_mesh, equispaced_tet_nodes, physical_nodes, taylor_green, uniform_perturbation

pytestmark = pytest.mark.gpu


def test_mixed_stage_waits_run_out_and_return():
    torch = torch_cuda()
    from paper_2512_17101_gb300 import capi, dg
    N = 2
    verts, period = box_mesh(3, 1.0)
    nodes = equispaced_tet_nodes(N)
    q0 = uniform_perturbation(taylor_green(physical_nodes(verts, nodes), mach=0.3, noise=0.01, seed=1), 1e-3, seed=2)
    mesh = dg.Mesh(verts, period, N, nodes)
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=2e-2, Pr=0.71)  # BR1 pass and right-hand side on tcgen05
    q = torch.tensor(q0, device="cuda")
    dt = 1e-3
    out, k = torch.empty_like(q), torch.zeros_like(q)
    dg.dg_rk_stage(mesh, gas, 0, dt, q, out, k, opts=dg._opts(precision=capi.DG_PREC_MIXED, wait_polls=1))
    assert mesh.status() & capi.DG_STATUS_TIMEOUT
    # tensor memory was released and the device is usable: the default bound gives the right stage
    out2, k2 = torch.empty_like(q), torch.zeros_like(q)
    dg.dg_rk_stage(mesh, gas, 0, dt, q, out2, k2, opts=dg._opts(precision=capi.DG_PREC_MIXED))
    assert mesh.status() == 0
    ref, kr = torch.empty_like(q), torch.zeros_like(q)
    dg.dg_rk_stage(mesh, gas, 0, dt, q, ref, kr)
    assert mesh.status() == 0
    assert field_err((out2 - q).cpu().numpy(), (ref - q).cpu().numpy()) < 1e-4


def test_mlp_guess_waits_run_out_and_return():
    torch = torch_cuda()
    from oracle.thermo import Nasa7Gas
    from paper_2512_17101_gb300 import capi, dg
    from workloads.gas import seeded_nasa7_mixture
    from workloads.mlp import glorot_params, temperature_samples
    mix = seeded_nasa7_mixture(7, seed=0)
    gas = dg.Gas(model="nasa7", W=mix.W, nasa7=mix.coeffs, newton_tol=1e-10, newton_max_it=50)
    go = Nasa7Gas(W=mix.W, coeffs=mix.coeffs)
    n = 700
    T, Y = temperature_samples(n, 7, seed=3)
    q = torch.tensor(go.conserved(np.ones(n), np.zeros((3, n)), Y, T), device="cuda")
    dg.dg_mlp_set(gas, glorot_params(2), dict(e_mean=1e6, e_scale=1e6, T_mean=1650.0, T_scale=780.0,
                                              T_min=300.0, T_max=3000.0))
    Tm = torch.empty(n, device="cuda", dtype=torch.float64)
    dg.dg_temperature(gas, q, Tm, opts=dg._opts(t_seed=capi.DG_TSEED_MLP, wait_polls=1))
    assert gas.status() & capi.DG_STATUS_TIMEOUT
    dg.dg_temperature(gas, q, Tm, opts=dg._opts(t_seed=capi.DG_TSEED_MLP))
    assert gas.status() == 0
    assert np.abs(Tm.cpu().numpy() - T).max() < 1e-8


def test_negative_wait_bound_is_rejected():
    torch = torch_cuda()
    from paper_2512_17101_gb300 import capi, dg
    verts, period = box_mesh(2, 1.0)
    mesh = dg.Mesh(verts, period, 1, equispaced_tet_nodes(1))
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0)
    q = torch.ones((5, mesh.K, 4), device="cuda", dtype=torch.float64)
    q[4] = 2.5
    with pytest.raises(Exception):
        dg.dg_rhs(mesh, gas, q, torch.empty_like(q), opts=dg._opts(precision=capi.DG_PREC_MIXED, wait_polls=-1))
