"""Reference-tetrahedron operators of nodal DG, from their plain definitions.

The paper works in the nodal DG setting of Hesthaven & Warburton (§1, Fig. 1:
DOFs are local to an element and form an [Np][K] array) and applies "full
assembly of all DG operators" (§5.2).  It prints none of the operators, so they
are written here from their definitions:

* nodal basis l_i: the degree-N polynomials with l_i(x_j) = delta_ij, expressed
  through the monomial basis r^a s^b t^c (a+b+c <= N) and the Vandermonde
  V[i][m] = m(x_i);
* derivative matrices: (Dr)_ij = dl_j/dr (x_i), i.e. Dr = Vr V^-1;
* mass matrix: M_ij = integral over the reference tetrahedron of l_i l_j,
  i.e. M = V^-T G V^-1 with the exact Gram matrix G of the monomials;
* face mass: for face f, E_f[i][j] = integral over the face of l_i l^f_j in
  the face's parameter coordinates (each face parametrised by two of r, s, t,
  so every parameter triangle has area 2), l^f_j the 2-D nodal basis of the
  face nodes;
* LIFT = M^-1 E with E = [E_0 | E_1 | E_2 | E_3]  (Np x 4 Nfp).

The monomial Vandermonde is ill-conditioned at N = 4 (condition ~5e3), so the
inverses, products and the Gram matrices are evaluated in 40-digit arithmetic
(mpmath; the Gram entries are exact rationals) and rounded to float64 once.

Reference tetrahedron: vertices (-1,-1,-1), (1,-1,-1), (-1,1,-1), (-1,-1,1).
Faces (vertex triples; equation; parameter coordinates):
    0: (0,1,2)  t = -1          (r, s)
    1: (0,1,3)  s = -1          (r, t)
    2: (1,2,3)  r + s + t = -1  (s, t)
    3: (0,2,3)  r = -1          (s, t)
Face nodes are listed in increasing volume-node index.
"""

from __future__ import annotations

from dataclasses import dataclass
from fractions import Fraction
from math import comb, factorial

import mpmath
import numpy as np

_DPS = 40  # digits for the small dense solves; results are rounded to float64 once

FACE_VERTICES = ((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3))
FACE_PARAMS = ((0, 1), (0, 2), (1, 2), (1, 2))
REF_VERTICES = np.array([[-1.0, -1.0, -1.0], [1.0, -1.0, -1.0], [-1.0, 1.0, -1.0], [-1.0, -1.0, 1.0]])


def face_residual(f: int, rst: np.ndarray) -> np.ndarray:
    """Distance-like residual of the plane of reference face f (zero on the face)."""
    r, s, t = rst[:, 0], rst[:, 1], rst[:, 2]
    return (1 + t, 1 + s, 1 + r + s + t, 1 + r)[f]


def exponents3(N):
    return [(a, b, c) for a in range(N + 1) for b in range(N + 1 - a) for c in range(N + 1 - a - b)]


def exponents2(N):
    return [(a, b) for a in range(N + 1) for b in range(N + 1 - a)]


def _shifted_power(a):
    """(2u - 1)^a = sum_i coef_i u^i, exact."""
    return [(i, comb(a, i) * 2 ** i * (-1) ** (a - i)) for i in range(a + 1)]


def tet_monomial_integral(a, b, c) -> Fraction:
    """Exact integral of r^a s^b t^c over the reference tetrahedron.

    Substituting r = 2u-1, s = 2v-1, t = 2w-1 maps it to the unit simplex
    (Jacobian 8), where the integral of u^i v^j w^k is i! j! k! / (i+j+k+3)!.
    """
    total = Fraction(0)
    for i, ci in _shifted_power(a):
        for j, cj in _shifted_power(b):
            for k, ck in _shifted_power(c):
                total += Fraction(ci * cj * ck * factorial(i) * factorial(j) * factorial(k), factorial(i + j + k + 3))
    return 8 * total


def tri_monomial_integral(a, b) -> Fraction:
    """Exact integral of x^a y^b over the parameter triangle {x, y >= -1, x + y <= 0}.

    x = 2u-1, y = 2v-1 maps it to the unit triangle (Jacobian 4), where the
    integral of u^i v^j is i! j! / (i+j+2)!.
    """
    total = Fraction(0)
    for i, ci in _shifted_power(a):
        for j, cj in _shifted_power(b):
            total += Fraction(ci * cj * factorial(i) * factorial(j), factorial(i + j + 2))
    return 4 * total


def _monomials3(rst, N, dr=0, ds=0, dt=0):
    """Rows: nodes; columns: d^(dr,ds,dt) of r^a s^b t^c (a+b+c <= N), as mpmath values."""
    rows = []
    for (r, s, t) in rst:
        r, s, t = mpmath.mpf(float(r)), mpmath.mpf(float(s)), mpmath.mpf(float(t))
        row = []
        for (a, b, c) in exponents3(N):
            if a < dr or b < ds or c < dt:
                row.append(mpmath.mpf(0))
                continue
            fa = mpmath.mpf(factorial(a) // factorial(a - dr))
            fb = mpmath.mpf(factorial(b) // factorial(b - ds))
            fc = mpmath.mpf(factorial(c) // factorial(c - dt))
            row.append(fa * fb * fc * r ** (a - dr) * s ** (b - ds) * t ** (c - dt))
        rows.append(row)
    return mpmath.matrix(rows)


def _monomials2(xy, N):
    rows = []
    for (x, y) in xy:
        x, y = mpmath.mpf(float(x)), mpmath.mpf(float(y))
        rows.append([x ** a * y ** b for (a, b) in exponents2(N)])
    return mpmath.matrix(rows)


def vandermonde3(rst: np.ndarray, N: int):
    """Monomial Vandermonde V[i][m] = r_i^a s_i^b t_i^c and its r, s, t derivatives (float64)."""
    with mpmath.workdps(_DPS):
        mats = [_monomials3(rst, N), _monomials3(rst, N, dr=1), _monomials3(rst, N, ds=1),
                _monomials3(rst, N, dt=1)]
        return tuple(_to_np(m) for m in mats)


def _to_np(m):
    return np.array([[float(m[i, j]) for j in range(m.cols)] for i in range(m.rows)])


def _gram3(N):
    ex = exponents3(N)
    return mpmath.matrix([[mpmath.mpf(tet_monomial_integral(a1 + a2, b1 + b2, c1 + c2).numerator)
                           / tet_monomial_integral(a1 + a2, b1 + b2, c1 + c2).denominator
                           for (a2, b2, c2) in ex] for (a1, b1, c1) in ex])


def _gram2(N):
    ex = exponents2(N)
    return mpmath.matrix([[mpmath.mpf(tri_monomial_integral(a1 + a2, b1 + b2).numerator)
                           / tri_monomial_integral(a1 + a2, b1 + b2).denominator
                           for (a2, b2) in ex] for (a1, b1) in ex])


@dataclass
class RefElement:
    N: int
    Np: int
    Nfp: int
    nodes: np.ndarray  # [Np][3]
    V: np.ndarray
    Dr: np.ndarray
    Ds: np.ndarray
    Dt: np.ndarray
    M: np.ndarray
    Fmask: np.ndarray  # [4][Nfp] volume-node index of each face node
    E: np.ndarray  # [Np][4 Nfp]
    LIFT: np.ndarray  # [Np][4 Nfp]
    Minv: np.ndarray = None  # [Np][Np] the inverse mass matrix, formed in extended precision and rounded once


def build_reference(N: int, nodes: np.ndarray, tol: float = 1e-10) -> RefElement:
    """Assemble the reference operators of order N on the given nodes [Np][3]."""
    nodes = np.asarray(nodes, dtype=np.float64)
    Np = (N + 1) * (N + 2) * (N + 3) // 6
    Nfp = (N + 1) * (N + 2) // 2
    if nodes.shape != (Np, 3):
        raise ValueError(f"order {N} needs {Np} nodes, got {nodes.shape}")
    Fmask = np.zeros((4, Nfp), dtype=np.int64)
    for f in range(4):
        idx = np.nonzero(np.abs(face_residual(f, nodes)) < tol)[0]
        if idx.size != Nfp:
            raise ValueError(f"face {f}: found {idx.size} face nodes, expected {Nfp}")
        Fmask[f] = idx
    with mpmath.workdps(_DPS):
        V = _monomials3(nodes, N)
        Vinv = mpmath.inverse(V)
        Dr = _monomials3(nodes, N, dr=1) * Vinv
        Ds = _monomials3(nodes, N, ds=1) * Vinv
        Dt = _monomials3(nodes, N, dt=1) * Vinv
        M = Vinv.T * _gram3(N) * Vinv
        E = mpmath.zeros(Np, 4 * Nfp)
        G2 = _gram2(N)
        for f in range(4):
            V2inv = mpmath.inverse(_monomials2(nodes[Fmask[f]][:, FACE_PARAMS[f]], N))
            Mf = V2inv.T * G2 * V2inv
            for a, i in enumerate(Fmask[f]):
                for b in range(Nfp):
                    E[int(i), f * Nfp + b] = Mf[a, b]
        Minv = mpmath.inverse(M)
        LIFT = Minv * E
        return RefElement(N=N, Np=Np, Nfp=Nfp, nodes=nodes, V=_to_np(V), Dr=_to_np(Dr), Ds=_to_np(Ds),
                          Dt=_to_np(Dt), M=_to_np(M), Fmask=Fmask, E=_to_np(E), LIFT=_to_np(LIFT),
                          Minv=_to_np(Minv))
