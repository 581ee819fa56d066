"""CPU checks of libdg: it loads, exports every entry point of include/dg.h, and its
host-side logic (reference operators, geometry, connectivity, argument checks)
agrees with the oracle.  No compute call is made (no GPU needed)."""

import ctypes
import os
import re

import numpy as np
import pytest

from tests._oracle_case import Disc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    from paper_2512_17101_gb300 import capi
    if not os.path.exists(capi.LIB_PATH):
        __graft_entry__.build()
    return capi.load()


def _declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(dg_\w+)\s*\(", text))
    return names


def test_exports_every_declared_symbol(lib):
    from paper_2512_17101_gb300 import capi
    declared = _declared_functions()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(capi.SIGNATURES), declared ^ set(capi.SIGNATURES)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_host_tables_match_oracle(lib, N):
    from paper_2512_17101_gb300 import dg
    from workloads import box_mesh, equispaced_tet_nodes
    v, per = box_mesh((3, 2, 2), (1.0, 0.7, 1.3))
    m = dg.Mesh(v, per, N, equispaced_tet_nodes(N), host_only=True)
    d = Disc(v, per, N)
    ops = m.operators()
    for key in ("Dr", "Ds", "Dt", "LIFT"):
        assert np.abs(ops[key] - getattr(d.ref, key)).max() <= 1e-14 * max(1.0, np.abs(getattr(d.ref, key)).max())
    assert np.array_equal(ops["Fmask"], d.ref.Fmask)
    vmapP, geo = m.connectivity()
    assert np.array_equal(vmapP, d.conn.vmapP)
    g = d.geo
    expect = np.concatenate([np.stack([g.rx, g.ry, g.rz, g.sx, g.sy, g.sz, g.tx, g.ty, g.tz], 1),
                             np.stack([g.nx, g.ny, g.nz, g.Fscale], 2).reshape(-1, 16), g.J[:, None]], 1)
    assert np.abs(geo - expect).max() <= 1e-13 * np.abs(expect).max()


BC_SIDES = [
    {(1, 0): 1, (1, 1): 2},
    {(0, 0): 3, (0, 1): 4, (2, 0): 1, (2, 1): 1},
    {(a, e): 2 for a in range(3) for e in (0, 1)},
]


@pytest.mark.parametrize("sides", BC_SIDES)
@pytest.mark.parametrize("N", [1, 3])
def test_boundary_connectivity_matches_oracle(lib, sides, N):
    """Faces without a partner keep -code in vmapP; the paired ones match the oracle's pairing."""
    from paper_2512_17101_gb300 import dg
    from tests._oracle_case import bc_disc
    from workloads import equispaced_tet_nodes
    d = bc_disc((3, 2, 2), N, sides)
    m = dg.Mesh(d.vertices, d.period, N, equispaced_tet_nodes(N), host_only=True, face_bc=d.face_bc)
    vmapP, _ = m.connectivity()
    want = np.where(d.conn.bc != 0, -d.conn.bc, d.conn.vmapP)
    assert np.array_equal(vmapP, want)


def test_boundary_faces_are_checked(lib):
    from paper_2512_17101_gb300 import capi, dg
    from workloads import box_mesh, equispaced_tet_nodes
    from workloads.mesh import box_face_bc
    v, per = box_mesh((2, 2, 2), 1.0)
    open_per = np.array([per[0], 0.0, per[2]])
    nodes = equispaced_tet_nodes(1)
    fb = box_face_bc(v, 1.0, sides={(1, 0): 1, (1, 1): 1})
    dg.Mesh(v, open_per, 1, nodes, host_only=True, face_bc=fb)  # closed by walls: fine
    with pytest.raises(capi.DGError):  # open faces without a code
        dg.Mesh(v, open_per, 1, nodes, host_only=True)
    with pytest.raises(capi.DGError):  # a code on faces that have partners
        dg.Mesh(v, per, 1, nodes, host_only=True, face_bc=fb)
    bad = fb.copy()
    bad[bad != 0] = 9
    with pytest.raises(capi.DGError):  # unknown code
        dg.Mesh(v, open_per, 1, nodes, host_only=True, face_bc=bad)
    m = dg.Mesh(v, open_per, 1, nodes, host_only=True, face_bc=fb)
    with pytest.raises(capi.DGError):
        m.set_inflow([0.0, 0.0, 0.0, 0.0, 1.0])  # rho <= 0
    with pytest.raises(capi.DGError):
        m.set_inflow([1.0, 0.0, 0.0])  # too few variables


def test_lsrk_coefficients_match_oracle(lib):
    from paper_2512_17101_gb300 import dg
    from oracle.lsrk import RK4A, RK4B
    a, b = dg.dg_lsrk4_coefficients()
    assert tuple(a) == RK4A and tuple(b) == RK4B


def _desc(K, N, nodes, verts, period, flags=1):
    from paper_2512_17101_gb300 import capi
    d = capi.dg_mesh_desc()
    d.K, d.N = K, N
    d.ref_nodes = nodes.ctypes.data_as(ctypes.c_void_p) if nodes is not None else None
    d.vertices = verts.ctypes.data_as(ctypes.c_void_p) if verts is not None else None
    for i in range(3):
        d.period[i] = period[i]
    d.flags = flags
    return d


def test_invalid_arguments_are_rejected(lib):
    from paper_2512_17101_gb300 import capi
    from workloads import box_mesh, equispaced_tet_nodes
    v, per = box_mesh(2, 1.0)
    nodes = equispaced_tet_nodes(2)
    h = ctypes.c_void_p()
    cases = [
        _desc(0, 2, nodes, v, per),                        # no elements
        _desc(v.shape[0], 5, nodes, v, per),               # order too high
        _desc(v.shape[0], 2, None, v, per),                # missing nodes
        _desc(v.shape[0], 2, nodes, v, (1.0, -1.0, 1.0)),  # negative period
        _desc(v.shape[0], 2, nodes, v, (0.0, 0.0, 0.0)),   # open mesh: faces without partners
        _desc(v.shape[0], 3, nodes, v, per),               # node count does not fit the order
    ]
    for d in cases:
        rc = lib.dg_mesh_upload(ctypes.byref(d), ctypes.byref(h))
        assert rc == capi.DG_ERR_INVALID_ARG
        assert lib.dg_last_error().decode()
    # an inverted element
    bad = v.copy()
    bad[0, [2, 3]] = bad[0, [3, 2]]
    rc = lib.dg_mesh_upload(ctypes.byref(_desc(v.shape[0], 2, nodes, bad, per)), ctypes.byref(h))
    assert rc == capi.DG_ERR_INVALID_ARG and b"Jacobian" in lib.dg_last_error()


def test_compute_calls_reject_host_only_mesh_and_bad_gas(lib):
    from paper_2512_17101_gb300 import capi, dg
    from workloads import box_mesh, equispaced_tet_nodes
    v, per = box_mesh(2, 1.0)
    m = dg.Mesh(v, per, 1, equispaced_tet_nodes(1), host_only=True)
    rc = lib.dg_rhs(m.handle, ctypes.c_void_p(1), ctypes.c_void_p(8), ctypes.c_void_p(16), None, None, None)
    assert rc == capi.DG_ERR_INVALID_ARG
    assert lib.dg_rhs(None, None, None, None, None, None, None) == capi.DG_ERR_INVALID_ARG
    g = capi.dg_gas_desc()
    g.model = capi.DG_GAS_PERFECT
    g.gamma = 0.9  # gamma must exceed 1
    g.R = 1.0
    h = ctypes.c_void_p()
    assert lib.dg_gas_create(ctypes.byref(g), ctypes.byref(h)) == capi.DG_ERR_INVALID_ARG
    g.model = 7
    assert lib.dg_gas_create(ctypes.byref(g), ctypes.byref(h)) == capi.DG_ERR_INVALID_ARG
    g.model = capi.DG_GAS_NASA7
    g.nspecies = 9
    assert lib.dg_gas_create(ctypes.byref(g), ctypes.byref(h)) == capi.DG_ERR_INVALID_ARG
    assert lib.dg_temperature(None, 10, None, None, None, None, None) == capi.DG_ERR_INVALID_ARG


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2512_17101_gb300 import capi
    saved = capi._lib
    capi._lib = None
    try:
        with pytest.raises(ImportError):
            capi.load(str(tmp_path / "missing.so"))
    finally:
        capi._lib = saved
