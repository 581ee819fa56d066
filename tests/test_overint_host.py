"""Host side of over-integration through the C ABI, no GPU: the library's own Stroud rule
(dg_tet_quadrature, Gauss-Jacobi roots by Newton in long double) integrates every monomial of total
degree <= 2q - 1 over the reference tetrahedron exactly (exact rational integrals) and misses one
of degree 2q; it has positive weights and interior points; out-of-range arguments are refused."""

import numpy as np
import pytest

from oracle.refelem import exponents3, tet_monomial_integral


def _lib():
    from paper_2512_17101_gb300 import capi, dg
    import os
    if not os.path.exists(capi.LIB_PATH):
        pytest.skip("libdg.so not built")
    return capi, dg


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 6, 7, 9, 12])
def test_library_rule_is_exact(q):
    capi, dg = _lib()
    pts, w = dg.dg_tet_quadrature(q)
    for (a, b, c) in exponents3(2 * q - 1):
        got = np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
        assert abs(got - float(tet_monomial_integral(a, b, c))) <= 2e-15
    assert abs(np.sum(w * pts[:, 2] ** (2 * q)) - float(tet_monomial_integral(0, 0, 2 * q))) > 1e-10
    assert np.all(w > 0) and np.all(pts > -1) and np.all(pts.sum(axis=1) < -1)


def test_library_rule_arguments():
    """q outside 1..DG_MAX_OVERINT_POINTS is refused before anything is written."""
    capi, dg = _lib()
    pts = np.zeros((1, 3))
    w = np.zeros(1)
    for q in (0, -1, capi.DG_MAX_OVERINT_POINTS + 1):
        with pytest.raises(capi.DGError):
            capi.check(capi.load().dg_tet_quadrature(int(q), pts.ctypes.data, w.ctypes.data))
    with pytest.raises(capi.DGError):
        capi.check(capi.load().dg_tet_quadrature(2, None, None))
