"""The node records of the mixed form's primitives pass (the float pairs that the tensor-core
kernels read): rho, momentum and energy rounded to FP32 exactly as the hardware rounds, and
rho, p and T (evaluated in FP64: p = (gamma - 1)(rho E - |rho u|^2 / (2 rho)), T = p / (rho R))
as float pairs hi + lo within 1e-12 of the FP64 values, normalised (|lo| <= ulp(hi) / 2)."""

import ctypes

import numpy as np
import pytest

from tests._gpu import torch_cuda
from tests._oracle_case import Disc
from workloads import box_mesh, equispaced_tet_nodes, taylor_green, uniform_perturbation

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mach", [0.1, 0.9])
def test_node_records_hold_the_fp64_primitives(mach):
    torch = torch_cuda()
    from paper_2512_17101_gb300 import capi, dg
    N = 3
    v, per = box_mesh((3, 3, 2), 1.0)
    d = Disc(v, per, N)
    mesh = dg.Mesh(v, per, N, equispaced_tet_nodes(N))
    gamma, R = 1.4, 287.0
    gas = dg.Gas(model="perfect", gamma=gamma, R=R, mu=1e-3, Pr=0.71)
    q0 = uniform_perturbation(taylor_green(d.xyz, mach=mach, noise=0.01, seed=3), 2e-2, seed=4)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    dg.dg_rhs(mesh, gas, q, rhs, opts=dg._opts(precision=capi.DG_PREC_MIXED))
    K, Np = q.shape[1], q.shape[2]
    KNp = K * Np
    # the mesh's scratch (10 doubles per node) copied out through the element gather, then read as floats
    base = ctypes.c_void_p()
    capi.check(capi.load().dg_mesh_viscous_buffer(mesh.handle, ctypes.byref(base)))
    raw = torch.empty(10, K, Np, dtype=torch.float64, device="cuda")
    ix = torch.arange(K, dtype=torch.int32, device="cuda")
    capi.check(capi.load().dg_gather_elements(base, 10, K, Np, ctypes.c_void_p(ix.data_ptr()), K,
                                              ctypes.c_void_p(raw.data_ptr()), None))
    flat = raw.cpu().numpy().reshape(-1).view(np.float32)
    node = flat[:8 * KNp].reshape(KNp, 8).astype(np.float64)
    temp = flat[16 * KNp:18 * KNp].reshape(KNp, 2).astype(np.float64)
    rho, mx, my, mz, E = (q0[v].reshape(-1) for v in range(5))
    p = (gamma - 1.0) * (E - 0.5 * (mx * mx + my * my + mz * mz) / rho)
    T = p / (rho * R)
    f32 = lambda x: x.astype(np.float32).astype(np.float64)
    for col, x in [(0, rho), (1, mx), (2, my), (3, mz), (4, E), (5, p)]:
        assert np.array_equal(node[:, col], f32(x)) or col == 5  # p_hi: the pair's normalised hi
    pair_err = lambda hi, lo, x: np.abs((hi + lo) - x).max() / np.abs(x).max()
    assert pair_err(node[:, 0], node[:, 7], rho) <= 2.0 ** -46
    assert pair_err(node[:, 5], node[:, 6], p) <= 1e-12
    assert pair_err(temp[:, 0], temp[:, 1], T) <= 1e-12
    for hi, lo in [(node[:, 5], node[:, 6]), (temp[:, 0], temp[:, 1]), (node[:, 0], node[:, 7])]:
        assert np.all(np.abs(lo) <= np.abs(hi) * 2.0 ** -24)
    assert np.abs(node[:, 5] - p).max() <= 2.0 ** -23 * np.abs(p).max()
    assert mesh.status() == 0
