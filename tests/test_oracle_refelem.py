"""Pins of the oracle's reference operators against mathematics, not against the oracle itself.

* exact differentiation of random degree-<=N polynomials (products of affine forms),
* mass and face-mass matrices against collapsed Gauss quadrature,
* the integration-by-parts identity M D_a + D_a^T M = sum_f n_a,f (A_f/2) E_f,
* closed-form N=1 operators (tests/golden/p1_tet_operators.json).
"""

import json
import os

import numpy as np
import pytest

from oracle.refelem import build_reference
from workloads import equispaced_tet_nodes, n_nodes, n_face_nodes
from tests._polyquad import AffineProduct, tet_rule, tri_rule

ORDERS = [1, 2, 3, 4]
_REFS = {}


def ref_of(N):
    if N not in _REFS:
        _REFS[N] = build_reference(N, equispaced_tet_nodes(N))
    return _REFS[N]


@pytest.mark.parametrize("N", ORDERS)
def test_sizes(N):
    ref = ref_of(N)
    assert ref.Np == n_nodes(N) == (N + 1) * (N + 2) * (N + 3) // 6
    assert ref.Nfp == n_face_nodes(N)
    assert ref.LIFT.shape == (ref.Np, 4 * ref.Nfp)
    # every face node set is distinct and each vertex belongs to 3 faces
    assert len({tuple(f) for f in ref.Fmask}) == 4


@pytest.mark.parametrize("N", ORDERS)
def test_exact_differentiation(N):
    ref = ref_of(N)
    rng = np.random.default_rng(10 + N)
    x = ref.nodes
    for deg in range(0, N + 1):
        for _ in range(3):
            p = AffineProduct(deg, 3, rng)
            vals, g = p(x), p.grad(x)
            scale = max(1.0, np.abs(g).max())
            for a, D in enumerate((ref.Dr, ref.Ds, ref.Dt)):
                assert np.abs(D @ vals - g[:, a]).max() <= 1e-12 * scale


@pytest.mark.parametrize("N", ORDERS)
def test_constant_in_kernel(N):
    ref = ref_of(N)
    for D in (ref.Dr, ref.Ds, ref.Dt):
        assert np.abs(D @ np.ones(ref.Np)).max() < 1e-12


@pytest.mark.parametrize("N", ORDERS)
def test_mass_matrix_against_quadrature(N):
    ref = ref_of(N)
    rng = np.random.default_rng(20 + N)
    qp, qw = tet_rule(N + 3)
    assert abs(qw.sum() - 4.0 / 3.0) < 1e-14
    assert abs(np.ones(ref.Np) @ ref.M @ np.ones(ref.Np) - 4.0 / 3.0) < 1e-13
    assert np.allclose(ref.M, ref.M.T, atol=1e-15)
    assert np.linalg.eigvalsh(ref.M).min() > 0
    for _ in range(5):
        p = AffineProduct(N, 3, rng)
        q = AffineProduct(rng.integers(0, N + 1), 3, rng)
        exact = np.sum(qw * p(qp) * q(qp))
        assert abs(p(ref.nodes) @ ref.M @ q(ref.nodes) - exact) < 1e-13 * max(1, abs(exact))


def _face_points(f, xy):
    """Reference-tetrahedron points of face f at parameter coordinates xy[Q][2]."""
    a, b = xy[:, 0], xy[:, 1]
    if f == 0:
        return np.stack([a, b, -np.ones_like(a)], 1)
    if f == 1:
        return np.stack([a, -np.ones_like(a), b], 1)
    if f == 2:
        return np.stack([-1 - a - b, a, b], 1)
    return np.stack([-np.ones_like(a), a, b], 1)


_FACE_PARAM_AXES = ((0, 1), (0, 2), (1, 2), (1, 2))


@pytest.mark.parametrize("N", ORDERS)
def test_face_mass_against_quadrature(N):
    ref = ref_of(N)
    rng = np.random.default_rng(30 + N)
    qp, qw = tri_rule(N + 3)
    assert abs(qw.sum() - 2.0) < 1e-14
    for f in range(4):
        pts = _face_points(f, qp)
        fnodes = ref.nodes[ref.Fmask[f]]
        Ef = ref.E[:, f * ref.Nfp:(f + 1) * ref.Nfp]
        for _ in range(3):
            p = AffineProduct(N, 3, rng)
            q = AffineProduct(N, 3, rng)
            exact = np.sum(qw * p(pts) * q(pts))
            got = p(ref.nodes) @ Ef @ q(fnodes)
            assert abs(got - exact) < 1e-13 * max(1, abs(exact))


@pytest.mark.parametrize("N", ORDERS)
def test_integration_by_parts(N):
    """int_T d(l_i l_j)/dr_a = sum over faces of int_f l_i l_j n_a dA (exact for polynomials)."""
    ref = ref_of(N)
    verts = np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float)
    fv = ((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3))
    for a, D in enumerate((ref.Dr, ref.Ds, ref.Dt)):
        lhs = ref.M @ D + D.T @ ref.M
        rhs = np.zeros_like(lhs)
        for f, (i0, i1, i2) in enumerate(fv):
            cr = np.cross(verts[i1] - verts[i0], verts[i2] - verts[i0])
            opp = ({0, 1, 2, 3} - {i0, i1, i2}).pop()
            if cr @ (verts[opp] - verts[i0]) > 0:
                cr = -cr
            area = np.linalg.norm(cr) / 2
            n = cr / np.linalg.norm(cr)
            full = np.zeros((ref.Np, ref.Np))
            full[:, ref.Fmask[f]] = ref.E[:, f * ref.Nfp:(f + 1) * ref.Nfp]
            rhs += n[a] * (area / 2.0) * full
        assert np.abs(lhs - rhs).max() < 1e-13


def test_lift_is_mass_inverse_of_face_mass():
    for N in ORDERS:
        ref = ref_of(N)
        assert np.abs(ref.M @ ref.LIFT - ref.E).max() < 1e-13


def test_p1_closed_forms():
    path = os.path.join(os.path.dirname(__file__), "golden", "p1_tet_operators.json")
    g = json.load(open(path))
    ref = build_reference(1, np.array(g["nodes"], float))
    assert np.array_equal(ref.Fmask, np.array(g["Fmask"]))
    assert np.abs(ref.Dr - np.array(g["Dr_rows"])).max() < 1e-15
    assert np.abs(ref.Ds - np.array(g["Ds_rows"])).max() < 1e-15
    assert np.abs(ref.Dt - np.array(g["Dt_rows"])).max() < 1e-15
    assert np.abs(ref.M - np.array(g["M_numerators_over_15"]) / 15.0).max() < 1e-15
    fm = np.array(g["face_mass_numerators_over_6"]) / 6.0
    for f in range(4):
        block = ref.E[ref.Fmask[f], f * 3:(f + 1) * 3]
        assert np.abs(block - fm).max() < 1e-15


def test_planted_mistake_is_caught():
    """A transposed derivative matrix must fail the exact-differentiation pin."""
    ref = ref_of(3)
    rng = np.random.default_rng(1)
    p = AffineProduct(3, 3, rng)
    assert np.abs(ref.Dr.T @ p(ref.nodes) - p.grad(ref.nodes)[:, 0]).max() > 1e-3
