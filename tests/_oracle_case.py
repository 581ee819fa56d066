"""Builds oracle discretisations (reference element, geometry, connectivity) for tests."""

import functools

import numpy as np

from oracle.geometry import connect, geometric_factors, affine_nodes
from oracle.refelem import build_reference
from workloads import box_mesh, equispaced_tet_nodes
from workloads.mesh import box_face_bc


@functools.lru_cache(maxsize=None)
def reference(N):
    return build_reference(N, equispaced_tet_nodes(N))


class Disc:
    def __init__(self, vertices, period, N, face_bc=None):
        self.N = N
        self.vertices = vertices
        self.period = np.asarray(period, float)
        self.face_bc = face_bc
        self.ref = reference(N)
        self.geo = geometric_factors(vertices)
        self.conn = connect(vertices, period, self.ref, face_bc=face_bc)
        self.xyz = affine_nodes(vertices, self.ref.nodes)
        self.K = vertices.shape[0]

    def integrate(self, u):
        """sum_k J_k 1^T M u_k for u[..., K, Np]."""
        return np.einsum("...kn,nm,k->...", u, self.ref.M, self.geo.J)

    def abs_integral(self, u):
        """sum_k J_k |u_k|^T |M| 1: a positive scale for cancellation checks of integrate()."""
        return np.einsum("...kn,nm,k->...", np.abs(u), np.abs(self.ref.M), self.geo.J)

    def l2(self, u):
        """L2 norm over the box, sqrt(sum_k J_k u_k^T M u_k), per leading index of u[..., K, Np]."""
        return np.sqrt(np.einsum("...kn,nm,...km,k->...", u, self.ref.M, u, self.geo.J))


@functools.lru_cache(maxsize=None)
def box_disc(n, N, L=1.0):
    v, per = box_mesh(n, L)
    return Disc(v, per, N)


def bc_disc(n, N, sides, L=1.0):
    """Box mesh with boundary conditions sides[(axis, end)] = code; the axes that carry codes are
    not periodic."""
    v, per = box_mesh(n, L)
    per = np.array(per, dtype=float)
    for axis, _ in sides:
        per[axis] = 0.0
    return Disc(v, per, N, face_bc=box_face_bc(v, L, sides=sides))
