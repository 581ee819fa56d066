"""Periodic box meshes of tetrahedra and the reference-node lattice.

A box of nx*ny*nz hexahedra is split into 6 tetrahedra per hexahedron along
its main diagonal (Kuhn / Freudenthal split): one tetrahedron per permutation
of the axes, walking from the cell's low corner to its high corner one axis at
a time.  The same split is used in every cell, so the mesh is conforming, and
it stays conforming across the periodic seams.  Vertex coordinates are stored
per element and *unwrapped* (a cell in the last layer keeps the coordinate L,
not 0); periodicity is described by the box lengths alone.

Element ordering: ((k*ny + j)*nx + i)*6 + p for cell (i, j, k) and axis
permutation p (itertools order).  Every element has positive orientation.
"""

from __future__ import annotations

import itertools

import numpy as np

_PERMS = list(itertools.permutations(range(3)))


def n_nodes(N: int) -> int:
    """Nodes of an order-N nodal tetrahedron: (N+1)(N+2)(N+3)/6."""
    return (N + 1) * (N + 2) * (N + 3) // 6


def n_face_nodes(N: int) -> int:
    """Nodes on one face of an order-N nodal tetrahedron: (N+1)(N+2)/2."""
    return (N + 1) * (N + 2) // 2


def _as3(v, cast):
    if np.isscalar(v):
        return (cast(v),) * 3
    v = tuple(cast(x) for x in v)
    if len(v) != 3:
        raise ValueError("expected a scalar or a triple")
    return v


def box_mesh(n, L=1.0, origin=(0.0, 0.0, 0.0)):
    """Periodic box [origin, origin+L] meshed by 6*nx*ny*nz tetrahedra.

    Returns (vertices, period): vertices float64 [K][4][3] (per element,
    unwrapped), period float64 [3] (the box lengths).
    """
    nx, ny, nz = _as3(n, int)
    Lx, Ly, Lz = _as3(L, float)
    if min(nx, ny, nz) < 1:
        raise ValueError("need at least one cell per direction")
    h = np.array([Lx / nx, Ly / ny, Lz / nz])
    o = np.asarray(origin, dtype=np.float64)
    # Corner offsets of each permutation tetrahedron in units of the cell size.
    tets = []
    for p in _PERMS:
        c0 = np.zeros(3)
        c1 = c0.copy()
        c1[p[0]] = 1.0
        c2 = c1.copy()
        c2[p[1]] = 1.0
        c3 = np.ones(3)
        corners = [c0, c1, c2, c3]
        e = np.array([corners[1] - corners[0], corners[2] - corners[0], corners[3] - corners[0]])
        if np.linalg.det(e.T) < 0:  # odd permutation: swap two vertices to orient positively
            corners[2], corners[3] = corners[3], corners[2]
        tets.append(np.array(corners))
    tets = np.array(tets)  # [6][4][3]
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cells = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1).astype(np.float64)  # [C][3]
    verts = (cells[:, None, None, :] + tets[None, :, :, :]) * h + o  # [C][6][4][3]
    verts = verts.reshape(-1, 4, 3)
    return np.ascontiguousarray(verts), np.array([Lx, Ly, Lz], dtype=np.float64)


# vertex triples of the four faces of a tetrahedron, in the library's face order
TET_FACES = ((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3))


def box_face_bc(vertices, L=1.0, origin=(0.0, 0.0, 0.0), sides=None):
    """Boundary-condition codes face_bc [K][4] (int32) of a box mesh: the code sides[(axis, end)]
    (end 0 = the plane x_axis = origin, 1 = origin + L) on faces lying in that plane, 0 elsewhere.
    Axes whose planes carry codes must be meshed without periodicity along them."""
    v = np.asarray(vertices, dtype=np.float64)
    Ls = np.asarray(_as3(L, float))
    o = np.asarray(origin, dtype=np.float64)
    out = np.zeros((v.shape[0], 4), dtype=np.int32)
    tol = 1e-9 * Ls.max()
    for (axis, end), code in (sides or {}).items():
        plane = o[axis] + (Ls[axis] if end else 0.0)
        for f, tri in enumerate(TET_FACES):
            on = np.all(np.abs(v[:, list(tri), axis] - plane) <= tol, axis=1)
            out[on, f] = code
    return out


def equispaced_tet_nodes(N: int) -> np.ndarray:
    """Equispaced (barycentric-lattice) nodes of the reference tetrahedron.

    Reference tetrahedron: vertices (-1,-1,-1), (1,-1,-1), (-1,1,-1), (-1,-1,1).
    Ordering: t index outermost, then s, then r:
    for k in 0..N, j in 0..N-k, i in 0..N-k-j: (r,s,t) = -1 + 2*(i,j,k)/N.
    Returns float64 [Np][3].
    """
    if N < 1:
        raise ValueError("order must be >= 1")
    pts = []
    for k in range(N + 1):
        for j in range(N + 1 - k):
            for i in range(N + 1 - k - j):
                pts.append((-1.0 + 2.0 * i / N, -1.0 + 2.0 * j / N, -1.0 + 2.0 * k / N))
    return np.array(pts, dtype=np.float64)


def physical_nodes(vertices: np.ndarray, ref_nodes: np.ndarray) -> np.ndarray:
    """Physical coordinates [K][Np][3] of the reference nodes under each element's affine map.

    The map sends reference vertex m to the element's vertex m; in barycentric
    form x = -(1+r+s+t)/2 v0 + (1+r)/2 v1 + (1+s)/2 v2 + (1+t)/2 v3.  Used only to
    sample initial states at the nodes.
    """
    r, s, t = ref_nodes[:, 0], ref_nodes[:, 1], ref_nodes[:, 2]
    lam = np.stack([-(1 + r + s + t) / 2, (1 + r) / 2, (1 + s) / 2, (1 + t) / 2], axis=1)  # [Np][4]
    return np.einsum("nm,kmd->knd", lam, vertices)
