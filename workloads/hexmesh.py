"""Inputs of the tensor-product hexahedron workloads: the 1-D node set, a periodic box of
axis-aligned hexahedra and the physical node coordinates.  Both the oracle and the GPU path
receive these as data (each builds its own operators from the node set).

Node index within an element: n = i + (N+1) (j + (N+1) k), i along x fastest.
Element index: e = ex + nx (ey + ny ez).
"""

from __future__ import annotations

import numpy as np


def gll_nodes(N: int) -> np.ndarray:
    """The N+1 Gauss-Lobatto-Legendre points on [-1, 1] in ascending order: -1, the roots of
    P_N', +1 (float64; the interior roots refined by Newton steps in extended precision)."""
    if N < 1:
        raise ValueError("N >= 1")
    dP = np.polynomial.legendre.Legendre.basis(N).deriv()
    ddP = dP.deriv()
    inner = np.sort(dP.roots().real) if N > 1 else np.array([])
    x = inner.astype(np.longdouble)
    for _ in range(4):
        x = x - np.asarray(dP(x), dtype=np.longdouble) / np.asarray(ddP(x), dtype=np.longdouble)
    out = np.concatenate([[-1.0], np.asarray(x, dtype=np.float64), [1.0]])
    return 0.5 * (out - out[::-1])  # exact symmetry about 0


def hex_box(n, L=1.0):
    """Periodic box [0, L]^3 of nx x ny x nz hexahedra.  Returns dict(n, L, h, origins[K][3])."""
    nx, ny, nz = (n, n, n) if np.isscalar(n) else tuple(int(v) for v in n)
    Lx, Ly, Lz = (L, L, L) if np.isscalar(L) else tuple(float(v) for v in L)
    h = np.array([Lx / nx, Ly / ny, Lz / nz])
    ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    origins = np.stack([ex.ravel() * h[0], ey.ravel() * h[1], ez.ravel() * h[2]], axis=1)
    return dict(n=(nx, ny, nz), L=np.array([Lx, Ly, Lz]), h=h, origins=origins)


def hex_nodes(box, x1d) -> np.ndarray:
    """Physical coordinates [K][Np][3] of the tensor-product nodes of every element."""
    x1d = np.asarray(x1d, dtype=np.float64)
    m = x1d.size
    k, j, i = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    ref = np.stack([x1d[i.ravel()], x1d[j.ravel()], x1d[k.ravel()]], axis=1)  # [Np][3]
    return box["origins"][:, None, :] + 0.5 * (ref[None, :, :] + 1.0) * box["h"][None, None, :]
