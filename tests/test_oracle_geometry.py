"""Pins of the oracle's geometric factors and periodic connectivity."""

import numpy as np
import pytest

from oracle.geometry import connect, geometric_factors
from tests._oracle_case import Disc, box_disc, reference
from workloads import box_mesh


@pytest.mark.parametrize("n,L", [(2, 1.0), (3, (1.0, 2.0, 0.5)), ((4, 3, 1), (10.0, 7.5, 2.5))])
def test_volume_and_closed_surfaces(n, L):
    v, per = box_mesh(n, L)
    geo = geometric_factors(v)
    assert abs(np.sum(geo.J) * 4.0 / 3.0 - np.prod(per)) < 1e-12 * np.prod(per)
    # sum over faces of (area * outward normal) vanishes for a closed surface; area = 2 sJ
    for comp in (geo.nx, geo.ny, geo.nz):
        assert np.abs(np.sum(2 * geo.sJ * comp, axis=1)).max() < 1e-14 * np.prod(per)
    # unit normals pointing away from the element
    cent = v.mean(axis=1)
    fv = ((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3))
    for f, idx in enumerate(fv):
        fc = v[:, list(idx)].mean(axis=1)
        n_ = np.stack([geo.nx[:, f], geo.ny[:, f], geo.nz[:, f]], 1)
        assert np.all(np.einsum("kd,kd->k", n_, fc - cent) > 0)
        assert np.allclose(np.linalg.norm(n_, axis=1), 1.0, atol=1e-15)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_chain_rule_on_linear_fields(N):
    d = box_disc(3, N)
    drdx = d.geo.drdx()
    D = (d.ref.Dr, d.ref.Ds, d.ref.Dt)
    for e in range(3):  # field x_e (unwrapped within each element: linear)
        f = d.xyz[:, :, e]
        for dd in range(3):
            g = sum(drdx[a, dd][:, None] * np.einsum("ij,kj->ki", D[a], f) for a in range(3))
            assert np.abs(g - (1.0 if dd == e else 0.0)).max() < 1e-12


@pytest.mark.parametrize("n,N", [(2, 1), (2, 3), (3, 2), ((3, 2, 1), 2)])
def test_periodic_connectivity(n, N):
    v, per = box_mesh(n, 1.0)
    d = Disc(v, per, N)
    c = d.conn
    K, Np, Nfp = d.K, d.ref.Np, d.ref.Nfp
    # face pairing is an involution
    for f in range(4):
        k2, f2 = c.EToE[:, f], c.EToF[:, f]
        assert np.array_equal(c.EToE[k2, f2], np.arange(K))
        assert np.array_equal(c.EToF[k2, f2], np.full(K, f))
    # node pairing is an involution on face-node slots (k, f, i) -> (k2, f2, j) -> (k, f, i)
    vP = c.vmapP.reshape(K, 4, Nfp)
    slot_of = np.full((K, 4, Np), -1)
    for f in range(4):
        slot_of[:, f, d.ref.Fmask[f]] = np.arange(Nfp)[None, :]
    k2 = vP // Np
    n2 = vP % Np
    f2 = np.broadcast_to(c.EToF[:, :, None], vP.shape)
    j = slot_of[k2, f2, n2]
    assert np.all(j >= 0)
    back = vP[k2, f2, j]
    assert np.array_equal(back, c.vmapM.reshape(K, 4, Nfp))
    flatM = c.vmapM.ravel()
    flatP = c.vmapP.ravel()
    # partners coincide modulo the period
    xyz = d.xyz.reshape(-1, 3)
    dx = xyz[flatM] - xyz[flatP]
    dx -= per * np.round(dx / per)
    assert np.abs(dx).max() < 1e-12
    # normals of paired faces are opposite
    n_ = np.stack([d.geo.nx, d.geo.ny, d.geo.nz], -1)
    assert np.abs(n_ + n_[c.EToE, c.EToF]).max() < 1e-14


def test_open_mesh_is_rejected():
    v, per = box_mesh(2, 1.0)
    with pytest.raises(ValueError):
        connect(v, np.zeros(3), reference(1))
