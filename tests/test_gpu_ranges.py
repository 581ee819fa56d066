"""Element ranges of the FP64 stage (dg_opts.elem_begin / elem_end), the primitives pass of a range
(dg_primitives, then dg_opts.prims_given) and the viscous flux of a range (dg_viscous_flux_range):
the pieces a partition schedules around its halo exchanges.  A stage split into ranges equals the
whole stage bit for bit, and leaves the elements outside its range untouched."""

import ctypes

import numpy as np
import pytest

from tests._gpu import torch_cuda
from tests._oracle_case import Disc
from workloads import box_mesh, equispaced_tet_nodes, taylor_green, uniform_perturbation

pytestmark = pytest.mark.gpu


def _case(torch, dg, N, viscous):
    v, per = box_mesh((3, 3, 2), 1.0)
    d = Disc(v, per, N)
    mesh = dg.Mesh(v, per, N, equispaced_tet_nodes(N))
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=2e-2 if viscous else 0.0, Pr=0.71)
    q = torch.tensor(uniform_perturbation(taylor_green(d.xyz, mach=0.3, noise=0.01, seed=4), 1e-3, seed=5),
                     device="cuda")
    k0 = torch.tensor(np.random.default_rng(6).standard_normal(tuple(q.shape)) * 1e-3, device="cuda")
    return mesh, gas, q, k0


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("N", [2, 3])
def test_ranged_stages_equal_the_whole_stage(N, viscous):
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    mesh, gas, q, k0 = _case(torch, dg, N, viscous)
    K, s, dt = q.shape[1], 2, 1e-3
    out, k = torch.empty_like(q), k0.clone()
    dg.dg_rk_stage(mesh, gas, s, dt, q, out, k)
    cut = K // 3
    # ranges, the viscous flux (if any) and the primitives computed inside each call
    out2, k2 = torch.full_like(q, 7.0), k0.clone()
    dg.dg_rk_stage(mesh, gas, s, dt, q, out2, k2, opts=dg._opts(elems=(0, cut)))
    assert torch.equal(out2[:, cut:], torch.full_like(out2[:, cut:], 7.0))  # untouched outside the range
    assert torch.equal(k2[:, cut:], k0[:, cut:])
    dg.dg_rk_stage(mesh, gas, s, dt, q, out2, k2, opts=dg._opts(elems=(cut, K)))
    assert torch.equal(out2, out) and torch.equal(k2, k)
    # the partition's pieces: primitives by range, viscous flux by range, stages with both given
    from paper_2512_17101_gb300 import capi
    lib = capi.load()
    qp = ctypes.c_void_p(q.data_ptr())
    out3, k3 = torch.full_like(q, 7.0), k0.clone()
    capi.check(lib.dg_primitives(mesh.handle, gas.handle, qp, 0, cut + 1, None))
    capi.check(lib.dg_primitives(mesh.handle, gas.handle, qp, cut + 1, K, None))
    if viscous:
        capi.check(lib.dg_viscous_flux_range(mesh.handle, gas.handle, qp, cut, K, None))
        capi.check(lib.dg_viscous_flux_range(mesh.handle, gas.handle, qp, 0, cut, None))
    for r in [(cut, K), (0, cut)]:
        dg.dg_rk_stage(mesh, gas, s, dt, q, out3, k3, opts=dg._opts(elems=r, viscous_given=viscous, prims_given=True))
    assert torch.equal(out3, out) and torch.equal(k3, k)
    # an empty range does nothing, (0, 0) included
    for r in [(cut, cut), (0, 0)]:
        out4, k4 = torch.full_like(q, 7.0), k0.clone()
        dg.dg_rk_stage(mesh, gas, s, dt, q, out4, k4, opts=dg._opts(elems=r, prims_given=True))
        assert torch.equal(out4, torch.full_like(q, 7.0)) and torch.equal(k4, k0)
    assert mesh.status() == 0


def test_range_arguments():
    torch = torch_cuda()
    from paper_2512_17101_gb300 import capi, dg
    mesh, gas, q, k0 = _case(torch, dg, 2, True)
    inviscid = dg.Gas(model="perfect", gamma=1.4, R=1.0)
    K = q.shape[1]
    out = torch.empty_like(q)
    lib = capi.load()
    qp = ctypes.c_void_p(q.data_ptr())
    for r in [(-1, 3), (5, 4), (0, K + 1)]:
        with pytest.raises(capi.DGError) as e:
            dg.dg_rk_stage(mesh, gas, 0, 1e-3, q, out, k0.clone(), opts=dg._opts(elems=r))
        assert e.value.code == capi.DG_ERR_INVALID_ARG
        assert lib.dg_primitives(mesh.handle, gas.handle, qp, r[0], r[1], None) == capi.DG_ERR_INVALID_ARG
        assert lib.dg_viscous_flux_range(mesh.handle, gas.handle, qp, r[0], r[1], None) == capi.DG_ERR_INVALID_ARG
    assert lib.dg_viscous_flux_range(mesh.handle, inviscid.handle, qp, 0, K, None) == capi.DG_ERR_INVALID_ARG
    mixed = dict(precision=capi.DG_PREC_MIXED)
    for extra in [dict(elems=(0, 4)), dict(elems=(0, 0)), dict(prims_given=True)]:
        with pytest.raises(capi.DGError) as e:
            dg.dg_rk_stage(mesh, gas, 0, 1e-3, q, out, k0.clone(), opts=dg._opts(**mixed, **extra))
        assert e.value.code == capi.DG_ERR_UNSUPPORTED
