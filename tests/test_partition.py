"""Host logic of the partitioned form (paper_2512_17101_gb300/partition.py), on CPU: every
element is owned once, a partition holds every face neighbour of its owned elements, send and
receive lists pair up element by element, the right-hand side of a partition (the oracle's, on
the partition's mesh with its halo filled) equals the global one at its owned elements, and the
torch.distributed transport delivers the halo between two gloo ranks and reduces across them."""

import os
import socket

import numpy as np
import pytest

from tests._oracle_case import Disc
from workloads import box_mesh, equispaced_tet_nodes, isentropic_vortex, uniform_perturbation


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    from paper_2512_17101_gb300 import capi
    if not os.path.exists(capi.LIB_PATH):
        __graft_entry__.build()
    return capi.load()


@pytest.mark.parametrize("nparts", [1, 2, 3, 5])
def test_partition_invariants(lib, nparts):
    from paper_2512_17101_gb300.partition import partition_mesh
    from paper_2512_17101_gb300 import dg
    N = 2
    v, per = box_mesh((3, 2, 2), 1.0)
    parts = partition_mesh(v, per, N, equispaced_tet_nodes(N), nparts)
    owned = np.concatenate([p.owned for p in parts])
    assert np.array_equal(np.sort(owned), np.arange(v.shape[0]))
    for p in parts:
        # the local mesh is closed (the library accepts it) and holds every neighbour of an owned element
        m = dg.Mesh(p.vertices, per, N, equispaced_tet_nodes(N), host_only=True, face_bc=p.face_bc)
        vmapP, _ = m.connectivity()
        own_faces = vmapP[:len(p.owned)]
        assert np.all(own_faces >= 0)
        for s, ix in p.send.items():
            theirs = parts[s].local[parts[s].recv[p.rank]]
            assert np.array_equal(p.local[ix], theirs)


@pytest.mark.parametrize("nparts", [1, 2, 3])
def test_owned_elements_interior_first(lib, nparts):
    """owned[:n_interior] have every face neighbour owned here; each of the others has one owned
    elsewhere (a halo element), and the groups keep ascending global order."""
    from paper_2512_17101_gb300 import dg
    from paper_2512_17101_gb300.partition import partition_mesh
    N = 2
    v, per = box_mesh((4, 3, 4), 1.0)
    glob = dg.Mesh(v, per, N, equispaced_tet_nodes(N), host_only=True)
    EToE, _ = glob.face_pairs()
    parts = partition_mesh(v, per, N, equispaced_tet_nodes(N), nparts)
    for p in parts:
        mine = set(p.owned.tolist())
        ni = p.n_interior
        inside = [all(int(n) in mine for n in EToE[e] if n >= 0) for e in p.owned]
        assert all(inside[:ni]) and not any(inside[ni:])
        assert np.all(np.diff(p.owned[:ni]) > 0) and np.all(np.diff(p.owned[ni:]) > 0)
        if nparts == 1:
            assert ni == len(p.owned) and len(p.halo) == 0
        else:
            assert 0 < ni < len(p.owned)


class _RecordingBackend:
    """Records the order of a partitioned step's operations (no arithmetic)."""

    flux_vars = 9

    def __init__(self):
        self.log = []

    def post(self, ranks, transport, arrays, V):
        self.log.append(("post", V))
        return None

    def finish(self, ranks, transport, handle, arrays, V):
        self.log.append(("finish", V))

    def primitives(self, rank, gas, q, elems):
        self.log.append(("prims", rank.i, tuple(elems)))

    def viscous_flux(self, rank, gas, q, elems):
        self.log.append(("viscous", rank.i, tuple(elems)))
        return q

    def stage(self, rank, gas, s, dt, q_in, q_out, viscous, elems):
        self.log.append(("stage", rank.i, tuple(elems)))


@pytest.mark.parametrize("viscous", [False, True])
def test_partitioned_step_overlaps_each_exchange_with_interior_work(lib, viscous):
    """Per stage: the state's exchange is posted before any compute and finished only after every
    rank's owned-node primitives and interior viscous flux; the halo primitives and border flux
    follow; the viscous flux's exchange is in flight over the interior stages; the border stages
    come last.  Every element range is covered once per pass."""
    import types
    import torch
    from paper_2512_17101_gb300.partition import LocalRouter, partition_mesh, partitioned_lsrk4_step
    N = 1
    v, per = box_mesh((3, 2, 4), 1.0)
    parts = partition_mesh(v, per, N, equispaced_tet_nodes(N), 2)
    ranks = []
    for i, p in enumerate(parts):
        q = torch.zeros(5, len(p.local), 4, dtype=torch.float64)
        ranks.append(types.SimpleNamespace(i=i, halo=types.SimpleNamespace(part=p), q=q,
                                           work=(torch.zeros_like(q), torch.zeros_like(q))))
    be = _RecordingBackend()
    partitioned_lsrk4_step(ranks, types.SimpleNamespace(model="perfect", mu=1e-2 if viscous else 0.0),
                           LocalRouter(), 1e-3, backend=be)
    groups = [((0, p.n_interior), (p.n_interior, len(p.owned)), (len(p.owned), len(p.local))) for p in parts]
    stage = [("post", 5)]
    stage += [op for i, (ig, bg, hg) in enumerate(groups)
              for op in [("prims", i, (0, bg[1]))] + ([("viscous", i, ig)] if viscous else [])]
    stage += [("finish", 5)]
    stage += [op for i, (ig, bg, hg) in enumerate(groups)
              for op in [("prims", i, hg)] + ([("viscous", i, bg)] if viscous else [])]
    stage += [("post", 9)] if viscous else []
    stage += [("stage", i, g[0]) for i, g in enumerate(groups)]
    stage += [("finish", 9)] if viscous else []
    stage += [("stage", i, g[1]) for i, g in enumerate(groups)]
    assert be.log == stage * 5


def test_partition_rhs_matches_global_at_owned_elements(lib):
    """Euler, the oracle on each partition's own mesh with the halo filled from the global state."""
    import oracle.boundary as bd
    from oracle.euler import rhs_strong
    from oracle.thermo import PerfectGas
    from paper_2512_17101_gb300.partition import partition_mesh
    N = 2
    v, per = box_mesh((4, 2, 2), 1.0)
    g = Disc(v, per, N)
    q = uniform_perturbation(isentropic_vortex(g.xyz, 0.0, period=per), 1e-3)
    gas = PerfectGas(1.4, 1.0)
    want = rhs_strong(g.ref, g.geo, g.conn, q, gas)
    for p in partition_mesh(v, per, N, equispaced_tet_nodes(N), 3):
        d = Disc(p.vertices, per, N, face_bc=p.face_bc)
        r = bd.rhs_euler_bc(d.ref, d.geo, d.conn, q[:, p.local], gas)
        no = len(p.owned)
        assert np.abs(r[:, :no] - want[:, p.owned]).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("viscous", [False, True])
def test_partition_rhs_with_boundary_faces(lib, viscous):
    """Walls and inflow / outflow faces stay with their elements: the oracle right-hand side of
    each partition (halo filled from the global state) equals the global one at owned elements.
    Navier-Stokes needs a second halo layer (the viscous flux of a halo element depends on its
    own neighbours), so there the comparison covers the owned elements whose neighbours are all
    owned."""
    import oracle.boundary as bd
    from oracle.thermo import PerfectGas
    from paper_2512_17101_gb300.partition import partition_mesh
    from tests._oracle_case import bc_disc
    N = 2
    sides = {(0, 0): bd.INFLOW, (0, 1): bd.OUTFLOW, (1, 0): bd.NOSLIP_WALL, (1, 1): bd.SLIP_WALL}
    g = bc_disc((4, 2, 2), N, sides)
    q = uniform_perturbation(isentropic_vortex(g.xyz, 0.0, period=np.where(g.period > 0, g.period, 1.0)), 1e-3)
    q_in = q[:, 0, 0].copy()
    gas = PerfectGas(1.4, 1.0)
    f = (lambda d, u: bd.rhs_ns_bc(d.ref, d.geo, d.conn, u, gas, 0.02, 0.71, q_in=q_in)) if viscous else \
        (lambda d, u: bd.rhs_euler_bc(d.ref, d.geo, d.conn, u, gas, q_in=q_in))
    want = f(g, q)
    for p in partition_mesh(g.vertices, g.period, N, equispaced_tet_nodes(N), 3, face_bc=g.face_bc):
        d = Disc(p.vertices, g.period, N, face_bc=p.face_bc)
        r = f(d, q[:, p.local])
        no = len(p.owned)
        keep = np.arange(no)
        if viscous:  # owned elements without a halo neighbour
            nb = d.conn.vmapP.reshape(d.K, -1) // d.ref.Np  # boundary nodes give negative values
            keep = np.array([e for e in range(no) if np.all(nb[e][nb[e] >= 0] < no)], dtype=int)
            assert len(keep) > 0
        assert np.abs(r[:, keep] - want[:, p.owned[keep]]).max() <= 1e-13 * np.abs(want).max()


def test_partition_arguments_and_local_reductions(lib):
    import torch
    from paper_2512_17101_gb300.partition import LocalRouter, partition_mesh
    v, per = box_mesh((2, 1, 1), 1.0)
    with pytest.raises(ValueError):
        partition_mesh(v, per, 1, equispaced_tet_nodes(1), 0)
    with pytest.raises(ValueError):
        partition_mesh(v, per, 1, equispaced_tet_nodes(1), v.shape[0] + 1)
    parts = partition_mesh(v, per, 1, equispaced_tet_nodes(1), v.shape[0])  # one element each
    assert all(len(p.owned) == 1 for p in parts)
    vals = [torch.tensor([1.0, -2.0]), torch.tensor([3.0, 5.0]), torch.tensor([-4.0, 0.5])]
    r = LocalRouter()
    assert all(t.tolist() == [0.0, 3.5] for t in r.reduce_all(vals, "sum"))
    assert all(t.tolist() == [3.0, 5.0] for t in r.reduce_all(vals, "max"))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _exchange_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ok = False
    try:
        from paper_2512_17101_gb300.partition import TorchTransport, partition_mesh
        N, Np = 1, 4
        v, per = box_mesh((4, 2, 2), 1.0)
        parts = partition_mesh(v, per, N, equispaced_tet_nodes(N), world)
        p = parts[rank]
        rng = np.random.default_rng(0)
        glob = rng.standard_normal((5, v.shape[0], Np))  # every rank knows the global field here
        local = glob[:, p.local].copy()
        local[:, len(p.owned):] = np.nan  # the halo before the exchange
        sends = {s: torch.from_numpy(local[:, ix]) for s, ix in p.send.items()}
        shapes = {s: (5, len(ix), Np) for s, ix in p.recv.items()}
        got = TorchTransport().exchange_all([sends], [shapes], torch.zeros(1, dtype=torch.float64))[0]
        for s, buf in got.items():
            local[:, p.recv[s]] = buf.numpy()
        ok = bool(np.array_equal(local, glob[:, p.local]))
        t = TorchTransport()
        v = torch.tensor([1.0 + rank, 10.0 * rank], dtype=torch.float64)
        ok = ok and t.reduce_all([v], "sum")[0].tolist() == [3.0, 10.0]
        ok = ok and t.reduce_all([v], "max")[0].tolist() == [2.0, 10.0] and v.tolist() == [1.0 + rank, 10.0 * rank]
    finally:
        out.put((rank, ok))
        dist.destroy_process_group()


def test_gloo_halo_exchange_two_ranks(lib):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_exchange_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert res == {0: True, 1: True}


class OracleBackend:
    """The compute of one partition on the CPU with the oracle (the test's stand-in for the
    library's kernels): halo rows copied by index, the BR1 viscous flux of the oracle's first pass
    (3 x 5 fields per node), the stage from the oracle's right-hand side with that flux.  The
    element ranges are honoured the way the library does: each call computes from the whole local
    state and stores the range's elements only, so a range that read a halo not yet refreshed
    (NaN before the first exchange) would carry NaN into the result."""

    flux_vars = 15

    def __init__(self, gas, mu, Pr):
        self.gas, self.mu, self.Pr = gas, mu, Pr

    def post(self, ranks, transport, arrays, V):
        import torch
        like = torch.zeros(1, dtype=torch.float64)
        sends = [{s: a[:, torch.from_numpy(ix).long()].contiguous() for s, ix in r.part.send.items()}
                 for r, a in zip(ranks, arrays)]
        shapes = [{s: (V, len(ix), a.shape[2]) for s, ix in r.part.recv.items()} for r, a in zip(ranks, arrays)]
        return transport.start(sends, shapes, like)

    def finish(self, ranks, transport, handle, arrays, V):
        import torch
        for r, a, got in zip(ranks, arrays, transport.finish(handle)):
            for s, buf in got.items():
                a[:, torch.from_numpy(r.part.recv[s]).long()] = buf

    def primitives(self, rank, gas, q, elems):
        pass  # the oracle forms its primitives itself

    def viscous_flux(self, rank, gas, q, elems):
        import torch
        import oracle.boundary as bd
        d = rank.disc
        with np.errstate(all="ignore"):
            fv = bd.viscous_flux_bc(d.ref, d.geo, d.conn, q.numpy(), self.gas, self.mu, self.Pr)
        fv = torch.from_numpy(np.ascontiguousarray(fv.reshape(15, d.K, d.ref.Np)))
        if rank.fv is None:
            rank.fv = torch.full_like(fv, float("nan"))
        rank.fv[:, elems[0]:elems[1]] = fv[:, elems[0]:elems[1]]
        return rank.fv

    def stage(self, rank, gas, s, dt, q_in, q_out, viscous, elems):
        import torch
        import oracle.boundary as bd
        from oracle.lsrk import RK4A, RK4B
        d, q = rank.disc, q_in.numpy()
        with np.errstate(all="ignore"):
            if viscous:
                rhs = bd.rhs_ns_bc(d.ref, d.geo, d.conn, q, self.gas, self.mu, self.Pr,
                                   Fv=rank.fv.numpy().reshape(3, 5, d.K, d.ref.Np))
            else:
                rhs = bd.rhs_euler_bc(d.ref, d.geo, d.conn, q, self.gas)
        e = slice(elems[0], elems[1])
        k = RK4A[s] * rank.work[1].numpy()[:, e] + dt * rhs[:, e]
        rank.work[1][:, e] = torch.from_numpy(k)
        q_out[:, e] = torch.from_numpy(q[:, e] + RK4B[s] * k)


def _two_step_case(viscous):
    from workloads import physical_nodes, taylor_green
    N = 2
    v, per = box_mesh((4, 2, 2), 1.0)
    nodes = equispaced_tet_nodes(N)
    xyz = physical_nodes(v, nodes)
    if viscous:
        q0 = uniform_perturbation(taylor_green(xyz, mach=0.3, noise=0.01, seed=1), 1e-3, seed=2)
    else:
        q0 = uniform_perturbation(isentropic_vortex(xyz, 0.0, period=per), 1e-3, seed=2)
    return N, v, per, nodes, q0, 2e-3, (2e-2 if viscous else 0.0)


def _partitioned_step_worker(rank, world, port, viscous, out):
    import types
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle.thermo import PerfectGas
        from paper_2512_17101_gb300.partition import TorchTransport, partition_mesh, partitioned_lsrk4_step
        N, v, per, nodes, q0, dt, mu = _two_step_case(viscous)
        p = partition_mesh(v, per, N, nodes, world)[rank]
        q = torch.from_numpy(np.ascontiguousarray(q0[:, p.local]))
        q[:, len(p.owned):] = float("nan")  # the halo before the first exchange
        st = types.SimpleNamespace(part=p, halo=types.SimpleNamespace(part=p),
                                   disc=Disc(p.vertices, per, N, face_bc=p.face_bc), q=q,
                                   work=(torch.full_like(q, float("nan")), torch.zeros_like(q)), fv=None)
        gas = types.SimpleNamespace(model="perfect", mu=mu)
        backend = OracleBackend(PerfectGas(1.4, 1.0), mu, 0.71)
        for _ in range(2):
            partitioned_lsrk4_step([st], gas, TorchTransport(), dt, backend=backend)
        out.put((rank, p.owned, st.q[:, :len(p.owned)].numpy().copy()))
    except Exception as e:  # reported to the parent, which fails the test
        out.put((rank, None, repr(e)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("viscous", [False, True])
def test_gloo_partitioned_lsrk4_steps_two_ranks(lib, viscous):
    """Two full LSRK4 steps of a mesh split over two gloo ranks (halo of the state, and for
    Navier-Stokes of the BR1 viscous flux, exchanged before every stage by TorchTransport), each
    rank's compute by the oracle, equal the single-mesh oracle steps at 1e-12."""
    import multiprocessing as mp
    import oracle.boundary as bd
    from oracle.lsrk import lsrk4_step
    from oracle.thermo import PerfectGas
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_partitioned_step_worker, args=(r, 2, port, viscous, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = [out.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    for _, owned, q in res:
        assert owned is not None, q
    N, v, per, nodes, q0, dt, mu = _two_step_case(viscous)
    g = Disc(v, per, N)
    gas = PerfectGas(1.4, 1.0)
    f = (lambda u: bd.rhs_ns_bc(g.ref, g.geo, g.conn, u, gas, mu, 0.71)) if viscous else \
        (lambda u: bd.rhs_euler_bc(g.ref, g.geo, g.conn, u, gas))
    want = lsrk4_step(lsrk4_step(q0, dt, f), dt, f)
    got = np.full_like(want, np.nan)
    for _, owned, q in res:
        got[:, owned] = q
    assert not np.isnan(got).any()
    scale = np.abs(want).max(axis=(1, 2))
    assert (np.abs(got - want).max(axis=(1, 2)) / scale).max() <= 1e-12
