"""Caller-supplied mesh tables (dg_mesh_desc: EToV, EToE/EToF, vmapP, Dr/Ds/Dt/LIFT/Fmask, geometric
factors), the problem statement of element-local arrays plus connectivity data (Sec. 1 Fig. 1,
Sec. 4.1.2).  Host-only uploads make no CUDA call, so these run without a GPU: tables exported
from one mesh, with the elements relabelled, are taken as given and returned unchanged; a face
pairing alone reproduces the neighbour map; every malformed table is refused."""

import numpy as np
import pytest

from workloads import box_mesh, equispaced_tet_nodes


def vertex_numbers(verts, period):
    """Global vertex numbers [K][4] of an unwrapped periodic box mesh: positions equal modulo the
    period share a number."""
    h = np.min(np.linalg.norm(verts[:, 1] - verts[:, 0], axis=1))
    ids, out = {}, np.zeros(verts.shape[:2], dtype=np.int32)
    for k in range(verts.shape[0]):
        for m in range(4):
            x = verts[k, m].copy()
            for a in range(3):
                if period[a] > 0:
                    x[a] -= period[a] * np.floor(x[a] / period[a] + 1e-9)
            key = tuple(np.round(x / h * 1e6).astype(np.int64))
            out[k, m] = ids.setdefault(key, len(ids))
    return out


def relabelled_tables(N, n=(3, 2, 2), seed=0):
    """A box mesh's own tables, exported from a host-only upload, with its elements relabelled by a
    seeded permutation (element e becomes new_of_old[e])."""
    from paper_2512_17101_gb300 import dg
    verts, period = box_mesh(n, 1.0)
    nodes = equispaced_tet_nodes(N)
    ref = dg.Mesh(verts, period, N, nodes, host_only=True)
    ops = ref.operators()
    vmapP, geo = ref.connectivity()
    EToE, EToF = ref.face_pairs()
    K, Np = ref.K, ref.Np
    new_of_old = np.random.default_rng(seed).permutation(K).astype(np.int32)
    old_of_new = np.argsort(new_of_old)
    v2 = verts[old_of_new]
    vm2 = vmapP[old_of_new]
    vm2 = np.where(vm2 >= 0, new_of_old[np.maximum(vm2, 0) // Np] * Np + np.maximum(vm2, 0) % Np, vm2)
    E2 = EToE[old_of_new]
    E2 = np.where(E2 >= 0, new_of_old[np.maximum(E2, 0)], -1)
    tables = dict(EToV=vertex_numbers(v2, period), EToE=E2.astype(np.int32), EToF=EToF[old_of_new],
                  vmapP=vm2.astype(np.int32), Dr=ops["Dr"], Ds=ops["Ds"], Dt=ops["Dt"], LIFT=ops["LIFT"],
                  Fmask=ops["Fmask"], geo=geo[old_of_new])
    return v2, period, nodes, tables, new_of_old


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_caller_tables_are_taken_and_returned(N):
    from paper_2512_17101_gb300 import dg
    v2, period, nodes, t, _ = relabelled_tables(N, seed=N)
    m = dg.Mesh(v2, period, N, nodes, host_only=True, tables=t)
    ops = m.operators()
    for key in ("Dr", "Ds", "Dt", "LIFT", "Fmask"):
        assert np.array_equal(ops[key], t[key]), key
    vmapP, geo = m.connectivity()
    assert np.array_equal(vmapP, t["vmapP"])
    assert np.array_equal(geo, t["geo"])
    E, F = m.face_pairs()
    assert np.array_equal(E, t["EToE"]) and np.array_equal(F, t["EToF"])
    # a face pairing alone gives the same neighbour map, and so does the library's own build
    m2 = dg.Mesh(v2, period, N, nodes, host_only=True, tables=dict(EToE=t["EToE"], EToF=t["EToF"]))
    assert np.array_equal(m2.connectivity()[0], t["vmapP"])
    m3 = dg.Mesh(v2, period, N, nodes, host_only=True)
    assert np.array_equal(m3.connectivity()[0], t["vmapP"])
    assert np.abs(m3.connectivity()[1] - t["geo"]).max() == 0.0


def _corrupt(t, what):
    t = {k: v.copy() for k, v in t.items()}
    Nfp = t["Fmask"].shape[1]
    if what == "vmapP_range":
        t["vmapP"][0, 0] = t["vmapP"].size * 10
    elif what == "vmapP_position":      # two partner nodes of one face swapped
        t["vmapP"][0, [0, 1]] = t["vmapP"][0, [1, 0]]
    elif what == "vmapP_boundary":      # a boundary code on a periodic mesh's face node
        t["vmapP"][0, 0] = -1
    elif what == "EToE_asymmetric":
        t["EToE"][0, 0] = (t["EToE"][0, 0] + 1) % t["EToE"].shape[0]
        del t["vmapP"]
    elif what == "EToF_vs_vmapP":
        t["EToF"][0, 0] = (t["EToF"][0, 0] + 1) % 4
    elif what == "EToV":
        t["EToV"][0, 0] = t["EToV"].max() + 1
    elif what == "Fmask_face":          # face 0's node list given for face 1
        t["Fmask"][[0, 1]] = t["Fmask"][[1, 0]]
    elif what == "Fmask_range":
        t["Fmask"][2, 0] = 10 ** 6
    elif what == "Dr_constants":
        t["Dr"][0, 0] += 1.0
    elif what == "LIFT_nan":
        t["LIFT"][1, 1] = np.nan
    elif what == "geo_jacobian":
        t["geo"][3, 25] = -1.0
    elif what == "geo_normal":
        t["geo"][0, 9] *= 2.0
    elif what == "operators_partial":
        for k in ("Ds", "Dt", "LIFT", "Fmask"):
            del t[k]
    elif what == "EToE_alone":
        del t["EToF"]
        del t["vmapP"]
    return t


@pytest.mark.parametrize("what", ["vmapP_range", "vmapP_position", "vmapP_boundary", "EToE_asymmetric",
                                  "EToF_vs_vmapP", "EToV", "Fmask_face", "Fmask_range", "Dr_constants",
                                  "LIFT_nan", "geo_jacobian", "geo_normal", "operators_partial", "EToE_alone"])
def test_malformed_caller_tables_are_refused(what):
    from paper_2512_17101_gb300 import capi, dg
    v2, period, nodes, t, _ = relabelled_tables(2)
    with pytest.raises(capi.DGError) as e:
        dg.Mesh(v2, period, 2, nodes, host_only=True, tables=_corrupt(t, what))
    assert e.value.code == capi.DG_ERR_INVALID_ARG


def test_caller_tables_with_boundary_faces():
    """A box with slip walls across y and inflow/outflow across x: EToE = -1 at the boundary faces,
    whose codes come from face_bc; the given vmapP (holding -code there) or the pairing alone is
    taken as is."""
    from paper_2512_17101_gb300 import dg
    from workloads.mesh import box_face_bc
    verts, period = box_mesh((3, 3, 2), 1.0)
    period = np.array(period, dtype=float)
    period[:2] = 0.0
    bc = box_face_bc(verts, 1.0, sides={(0, 0): 3, (0, 1): 4, (1, 0): 1, (1, 1): 1})
    nodes = equispaced_tet_nodes(2)
    ref = dg.Mesh(verts, period, 2, nodes, host_only=True, face_bc=bc)
    vmapP, geo = ref.connectivity()
    E, F = ref.face_pairs()
    assert np.array_equal(E < 0, bc > 0) and np.all(F[E < 0] == -1)
    m = dg.Mesh(verts, period, 2, nodes, host_only=True, face_bc=bc, tables=dict(vmapP=vmapP, EToE=E, EToF=F))
    assert np.array_equal(m.connectivity()[0], vmapP)
    m2 = dg.Mesh(verts, period, 2, nodes, host_only=True, face_bc=bc, tables=dict(EToE=E, EToF=F))
    assert np.array_equal(m2.connectivity()[0], vmapP)
    # a boundary face whose face_bc code disagrees with the given vmapP is refused
    from paper_2512_17101_gb300 import capi
    bad = bc.copy()
    k, f = np.argwhere(bc == 1)[0]
    bad[k, f] = 2
    with pytest.raises(capi.DGError):
        dg.Mesh(verts, period, 2, nodes, host_only=True, face_bc=bad, tables=dict(vmapP=vmapP))
