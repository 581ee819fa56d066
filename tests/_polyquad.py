"""Test helpers: random polynomials with exact gradients, and collapsed Gauss quadrature.

These are independent of the oracle: they evaluate polynomials given as
products of affine forms (gradient by the product rule) and integrate over
the reference tetrahedron / parameter triangle with Gauss-Legendre rules
collapsed onto the simplex (Duffy transform).
"""

import numpy as np


class AffineProduct:
    """p(x) = c0 * prod_m (c_m + g_m . x), a polynomial of the given degree in dim variables."""

    def __init__(self, degree, dim, rng):
        self.c0 = rng.uniform(0.5, 1.5)
        self.c = rng.uniform(-1, 1, size=degree)
        self.g = rng.uniform(-1, 1, size=(degree, dim))

    def __call__(self, x):
        out = np.full(x.shape[0], self.c0)
        for cm, gm in zip(self.c, self.g):
            out = out * (cm + x @ gm)
        return out

    def grad(self, x):
        factors = [cm + x @ gm for cm, gm in zip(self.c, self.g)]
        out = np.zeros_like(x)
        for m in range(len(factors)):
            rest = np.full(x.shape[0], self.c0)
            for j, fj in enumerate(factors):
                if j != m:
                    rest = rest * fj
            out += rest[:, None] * self.g[m][None, :]
        return out


def tet_rule(n):
    """Points [Q][3] and weights [Q] exact for degree <= 2n-3 on the reference tetrahedron."""
    x, w = np.polynomial.legendre.leggauss(n)
    a, wa = (x + 1) / 2, w / 2
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                u = a[i]
                v = a[j] * (1 - a[i])
                z = a[k] * (1 - a[i]) * (1 - a[j])
                pts.append((2 * u - 1, 2 * v - 1, 2 * z - 1))
                wts.append(8 * wa[i] * wa[j] * wa[k] * (1 - a[i]) ** 2 * (1 - a[j]))
    return np.array(pts), np.array(wts)


def tri_rule(n):
    """Points [Q][2] and weights [Q] on the parameter triangle {x, y >= -1, x + y <= 0}."""
    x, w = np.polynomial.legendre.leggauss(n)
    a, wa = (x + 1) / 2, w / 2
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            u = a[i]
            v = a[j] * (1 - a[i])
            pts.append((2 * u - 1, 2 * v - 1))
            wts.append(4 * wa[i] * wa[j] * (1 - a[i]))
    return np.array(pts), np.array(wts)
