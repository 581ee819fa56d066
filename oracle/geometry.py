"""Affine geometric factors and face connectivity of tetrahedral meshes.

The paper's DG operators act on element-local arrays (§1, Fig. 1) and need
"connectivity data" to gather neighbour values at faces (§4.1.2; the indirect
gather idx[i, j] of §4.3).  It does not spell either out, so they follow their
definitions here:

* each element is the image of the reference tetrahedron under the affine map
  that sends reference vertex m to element vertex m,
  x = -(1+r+s+t)/2 v0 + (1+r)/2 v1 + (1+s)/2 v2 + (1+t)/2 v3;
  J = det(dx/dr), and (rx, ry, rz, sx, ...) are the entries of (dx/dr)^-1;
* the outward unit normal of each face comes from the cross product of two
  face edges, oriented away from the opposite vertex; sJ = face area / 2 (the
  face integrals of the reference operators use parameter triangles of area
  2), and Fscale = sJ / J;
* faces of a periodic mesh are paired by their centroids modulo the box
  lengths; the two centroids fix the periodic shift between the faces (a
  whole number of box lengths) and face nodes are paired by coordinates under
  that shift;
* a face that finds no partner is a boundary face, allowed only where the
  caller's face_bc[k][f] names a boundary condition (oracle/boundary.py); its
  face nodes point at themselves in vmapP and carry that code in ``bc``.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .refelem import FACE_VERTICES, RefElement


@dataclass
class Geometry:
    rx: np.ndarray  # [K] ... entries of the inverse Jacobian, constant per element
    ry: np.ndarray
    rz: np.ndarray
    sx: np.ndarray
    sy: np.ndarray
    sz: np.ndarray
    tx: np.ndarray
    ty: np.ndarray
    tz: np.ndarray
    J: np.ndarray  # [K]
    nx: np.ndarray  # [K][4]
    ny: np.ndarray
    nz: np.ndarray
    sJ: np.ndarray  # [K][4]
    Fscale: np.ndarray  # [K][4]

    def drdx(self):
        """[3][3][K]: entry [a][d] = d(r_a)/d(x_d), r_a in (r, s, t), x_d in (x, y, z)."""
        return np.array([[self.rx, self.ry, self.rz], [self.sx, self.sy, self.sz], [self.tx, self.ty, self.tz]])


def affine_nodes(vertices: np.ndarray, ref_nodes: np.ndarray) -> np.ndarray:
    """Physical node coordinates [K][Np][3] under each element's affine map."""
    r, s, t = ref_nodes[:, 0], ref_nodes[:, 1], ref_nodes[:, 2]
    w = np.stack([-(1 + r + s + t) / 2, (1 + r) / 2, (1 + s) / 2, (1 + t) / 2], axis=1)
    return np.einsum("nm,kmd->knd", w, vertices)


def geometric_factors(vertices: np.ndarray) -> Geometry:
    v = np.asarray(vertices, dtype=np.float64)
    if v.ndim != 3 or v.shape[1:] != (4, 3):
        raise ValueError("vertices must be [K][4][3]")
    jac = np.stack([(v[:, 1] - v[:, 0]) / 2, (v[:, 2] - v[:, 0]) / 2, (v[:, 3] - v[:, 0]) / 2], axis=2)  # [K][x][r]
    J = np.linalg.det(jac)
    if np.any(J <= 0):
        raise ValueError("element with non-positive Jacobian")
    inv = np.linalg.inv(jac)  # [K][r][x]
    K = v.shape[0]
    nrm = np.zeros((K, 4, 3))
    area = np.zeros((K, 4))
    for f, (a, b, c) in enumerate(FACE_VERTICES):
        d = ({0, 1, 2, 3} - {a, b, c}).pop()
        cr = np.cross(v[:, b] - v[:, a], v[:, c] - v[:, a])
        sgn = np.sign(np.einsum("kd,kd->k", cr, v[:, d] - v[:, a]))
        cr = -sgn[:, None] * cr
        mag = np.linalg.norm(cr, axis=1)
        area[:, f] = mag / 2
        nrm[:, f] = cr / mag[:, None]
    sJ = area / 2
    return Geometry(
        rx=inv[:, 0, 0], ry=inv[:, 0, 1], rz=inv[:, 0, 2],
        sx=inv[:, 1, 0], sy=inv[:, 1, 1], sz=inv[:, 1, 2],
        tx=inv[:, 2, 0], ty=inv[:, 2, 1], tz=inv[:, 2, 2],
        J=J, nx=nrm[:, :, 0], ny=nrm[:, :, 1], nz=nrm[:, :, 2], sJ=sJ, Fscale=sJ / J[:, None])


@dataclass
class Connectivity:
    EToE: np.ndarray  # [K][4]
    EToF: np.ndarray  # [K][4]
    vmapM: np.ndarray  # [K][4 Nfp] flat node index (k Np + n) of each own face node
    vmapP: np.ndarray  # [K][4 Nfp] flat node index of the matching neighbour node (own node on a boundary face)
    bc: np.ndarray = None  # [K][4 Nfp] boundary-condition code of each face node, 0 on interior faces


def _wrap(x, period):
    out = np.array(x, dtype=np.float64, copy=True)
    for d in range(3):
        L = period[d]
        if L > 0:
            out[..., d] = out[..., d] - L * np.floor(out[..., d] / L + 1e-7)
    return out




def connect(vertices: np.ndarray, period, ref: RefElement, tol_rel: float = 1e-8, face_bc=None) -> Connectivity:
    """Pair every face with its neighbour and every face node with its partner.

    Without face_bc, raises ValueError if some face or face node has no unique
    partner (the mesh must be closed under the periodic identification).  With
    face_bc [K][4], a face without a partner must carry a non-zero code there
    and a paired face must carry 0.
    """
    v = np.asarray(vertices, dtype=np.float64)
    period = np.asarray(period, dtype=np.float64)
    K = v.shape[0]
    Np, Nfp = ref.Np, ref.Nfp
    edges = np.linalg.norm(v[:, [1, 2, 3, 2, 3, 3]] - v[:, [0, 0, 0, 1, 1, 2]], axis=2)
    hmin = edges.min()
    q = 1e-6 * hmin
    cent = np.stack([v[:, list(fv)].mean(axis=1) for fv in FACE_VERTICES], axis=1)  # [K][4][3]
    keys = np.round(_wrap(cent, period) / q).astype(np.int64)
    table = {}
    for k in range(K):
        for f in range(4):
            table.setdefault(tuple(keys[k, f]), []).append((k, f))
    EToE = np.full((K, 4), -1, dtype=np.int64)
    EToF = np.full((K, 4), -1, dtype=np.int64)
    fbc = np.zeros((K, 4), dtype=np.int64) if face_bc is None else np.asarray(face_bc, dtype=np.int64).reshape(K, 4)
    for key, lst in table.items():
        if len(lst) == 1 and fbc[lst[0]] != 0:
            continue  # boundary face
        if len(lst) != 2:
            raise ValueError(f"face with centroid key {key} has {len(lst)} occurrences (expected 2)")
        if fbc[lst[0]] != 0 or fbc[lst[1]] != 0:
            raise ValueError(f"interior face with centroid key {key} carries a boundary condition")
        (k1, f1), (k2, f2) = lst
        EToE[k1, f1], EToF[k1, f1] = k2, f2
        EToE[k2, f2], EToF[k2, f2] = k1, f1
    xyz = affine_nodes(v, ref.nodes)  # [K][Np][3]
    vmapM = (np.arange(K)[:, None, None] * Np + ref.Fmask[None, :, :]).reshape(K, 4 * Nfp)
    vmapP = np.zeros((K, 4, Nfp), dtype=np.int64)
    bnd = EToE < 0
    EToE = np.where(bnd, np.arange(K)[:, None], EToE)  # boundary faces point at themselves
    EToF = np.where(bnd, np.arange(4)[None, :], EToF)
    for f in range(4):
        own = xyz[:, ref.Fmask[f]]  # [K][Nfp][3]
        nb = xyz[EToE[:, f][:, None], ref.Fmask[EToF[:, f]]]  # [K][Nfp][3]
        # one periodic shift per face pair (a whole number of box lengths), from the centroids
        shift = cent[:, f] - cent[EToE[:, f], EToF[:, f]]
        for a in range(3):
            shift[:, a] = period[a] * np.round(shift[:, a] / period[a]) if period[a] > 0 else 0.0
        d = own[:, :, None, :] - (nb[:, None, :, :] + shift[:, None, None, :])  # [K][i][j][3]
        dist = np.linalg.norm(d, axis=3)
        j = np.argmin(dist, axis=2)
        best = np.take_along_axis(dist, j[:, :, None], axis=2)[:, :, 0]
        if np.any(best > tol_rel * hmin * 1e2):
            raise ValueError("face node without a coincident partner")
        if np.any(np.sort(j, axis=1) != np.arange(Nfp)[None, :]):
            raise ValueError("face node matching is not one-to-one")
        vmapP[:, f] = EToE[:, f][:, None] * Np + ref.Fmask[EToF[:, f][:, None], j]
    bc = np.repeat(np.where(bnd, fbc, 0), Nfp, axis=1)  # [K][4 Nfp]
    EToE = np.where(bnd, -1, EToE)
    EToF = np.where(bnd, -1, EToF)
    return Connectivity(EToE=EToE, EToF=EToF, vmapM=vmapM, vmapP=vmapP.reshape(K, 4 * Nfp), bc=bc)
