"""Element partitions of a tetrahedral mesh for the multi-process form, and their halo exchange.

The paper runs its largest cases over many GPUs, exchanging face data between the ranks of a
domain decomposition (§5.4).  Here a rank uploads its owned elements followed by copies of their
face neighbours owned by other ranks (halo elements; their faces that lead out of the local set
carry DG_BC_OUTFLOW, so the local mesh is closed; the halo's own right-hand side is never
computed).  Before each right-hand side the halo copies are refreshed from their owners; for
Navier-Stokes the viscous flux is computed, its halo refreshed, and the stage then uses it
(`dg_opts.viscous_given`).

The owned elements come in two groups: the interior ones, none of whose face neighbours is a halo
element, then the border ones.  As in the paper's execution engine (§4.6.1: receives posted
first, every part run as soon as its inputs are there), a stage posts each exchange, computes the
interior elements' part while the data is in flight, and finishes the border elements after it.

The library moves the data (`dg_gather_elements`, `dg_scatter_elements`); the transport between
ranks is a small object: `start(sends, recv_shapes, like)` posts an exchange and returns a handle,
`finish(handle)` waits for it and returns what arrived (`exchange_all` does both), and
`reduce_all(values, op)` (op "sum" or "max") is the global reduction.  `TorchTransport` uses
torch.distributed point-to-point messages (NCCL on GPUs, gloo on CPUs) for the one partition a
process holds; `LocalRouter` hands the buffers between partitions held by one process.

Partitioning: contiguous ranges of the element index (for the box meshes of the workloads these
are slabs across the z direction); the face adjacency comes from the library's own connectivity.
"""

from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np

from . import capi
from .capi import check, load

OUTFLOW = capi.DG_BC_OUTFLOW


@dataclass
class Partition:
    rank: int
    owned: np.ndarray            # global ids of the owned elements: interior, then border (each ascending)
    halo: np.ndarray             # global ids of the halo elements (ascending)
    vertices: np.ndarray         # [len(owned) + len(halo)][4][3]
    face_bc: np.ndarray          # [len(owned) + len(halo)][4]
    send: dict = field(default_factory=dict)   # rank -> local indices of owned elements it holds as halo
    recv: dict = field(default_factory=dict)   # rank -> local indices of the halo elements it owns
    n_interior: int = 0          # owned[:n_interior] have no face neighbour in the halo

    @property
    def local(self) -> np.ndarray:
        return np.concatenate([self.owned, self.halo])


def partition_mesh(vertices, period, N, ref_nodes, nparts, face_bc=None):
    """The nparts partitions of a mesh (contiguous element ranges), each with its halo and
    exchange lists.  Send and receive lists between two ranks are in ascending global order, so
    that they pair up element by element."""
    from .dg import Mesh
    v = np.ascontiguousarray(vertices, dtype=np.float64)
    K = v.shape[0]
    if not 1 <= nparts <= K:
        raise ValueError("need 1 <= nparts <= K")
    glob = Mesh(v, period, N, ref_nodes, host_only=True, face_bc=face_bc)
    vmapP, _ = glob.connectivity()
    Np, Nfp = glob.Np, glob.Nfp
    first = vmapP[:, ::Nfp]  # [K][4]: a face node's partner, or -code on a boundary face
    partner = np.where(first >= 0, first // Np, -1)
    gbc = np.zeros((K, 4), dtype=np.int32) if face_bc is None else np.asarray(face_bc, dtype=np.int32)
    owner = (np.arange(K, dtype=np.int64) * nparts) // K
    parts = []
    for r in range(nparts):
        owned = np.flatnonzero(owner == r)
        nbs = partner[owned].ravel()
        halo = np.setdiff1d(np.unique(nbs[nbs >= 0]), owned)
        # interior elements first: none of their face partners is owned elsewhere
        border = ((partner[owned] >= 0) & (owner[np.maximum(partner[owned], 0)] != r)).any(axis=1)
        owned = np.concatenate([owned[~border], owned[border]])
        local = np.concatenate([owned, halo])
        in_local = np.zeros(K, dtype=bool)
        in_local[local] = True
        fbc = gbc[local].copy()
        hp = partner[halo]  # [H][4]
        leaves = (hp >= 0) & ~in_local[np.maximum(hp, 0)]
        fbc[len(owned):][leaves] = OUTFLOW  # halo faces leading out of the local set
        parts.append(Partition(rank=r, owned=owned, halo=halo, vertices=np.ascontiguousarray(v[local]),
                               face_bc=np.ascontiguousarray(fbc, dtype=np.int32), n_interior=int((~border).sum())))
    for p in parts:
        pos = {int(g): i for i, g in enumerate(p.local)}
        for s in range(nparts):
            if s == p.rank:
                continue
            mine_there = np.intersect1d(p.owned, parts[s].halo)   # ascending
            theirs_here = p.halo[owner[p.halo] == s]               # ascending
            if len(mine_there):
                p.send[s] = np.array([pos[int(g)] for g in mine_there], dtype=np.int32)
            if len(theirs_here):
                p.recv[s] = np.array([pos[int(g)] for g in theirs_here], dtype=np.int32)
    return parts


class TorchTransport:
    """Point-to-point exchange through torch.distributed (one message each way per neighbour),
    for the one partition this process holds.  As in the paper's execution engine (§5.4), every
    receive is posted before the sends."""

    def __init__(self, group=None):
        self.group = group

    def start(self, sends: list, recv_shapes: list, like):
        import torch
        import torch.distributed as dist
        assert len(sends) == 1, "a process holds one partition"
        out = {s: torch.empty(shape, dtype=like.dtype, device=like.device) for s, shape in recv_shapes[0].items()}
        reqs = [dist.irecv(out[s], src=s, group=self.group) for s in out]
        # the send buffers stay referenced by the handle until the exchange is finished
        bufs = {s: buf.contiguous() for s, buf in sends[0].items()}
        reqs += [dist.isend(buf, dst=s, group=self.group) for s, buf in bufs.items()]
        return out, reqs, bufs

    def finish(self, handle) -> list:
        out, reqs, _ = handle
        for r in reqs:
            r.wait()
        return [out]

    def exchange_all(self, sends: list, recv_shapes: list, like) -> list:
        return self.finish(self.start(sends, recv_shapes, like))

    def reduce_all(self, values: list, op: str) -> list:
        import torch.distributed as dist
        assert len(values) == 1, "a process holds one partition"
        t = values[0].clone()
        dist.all_reduce(t, op=dist.ReduceOp.SUM if op == "sum" else dist.ReduceOp.MAX, group=self.group)
        return [t]


class LocalRouter:
    """Exchange among partitions held by one process (each message is the sender's buffer)."""

    def start(self, sends: list, recv_shapes: list, like):
        out = [dict() for _ in sends]
        for r, sd in enumerate(sends):
            for s, buf in sd.items():
                out[s][r] = buf
        for r, shapes in enumerate(recv_shapes):
            for s, shape in shapes.items():
                assert tuple(out[r][s].shape) == tuple(shape), "send and receive lists do not pair up"
        return out

    def finish(self, handle) -> list:
        return handle

    def exchange_all(self, sends: list, recv_shapes: list, like) -> list:
        return self.finish(self.start(sends, recv_shapes, like))

    def reduce_all(self, values: list, op: str) -> list:
        import torch
        st = torch.stack(values)
        t = st.sum(dim=0) if op == "sum" else st.max(dim=0).values
        return [t.clone() for _ in values]


class HaloExchange:
    """Refreshes the halo of [V][K_local][Np] device arrays of one partition."""

    def __init__(self, part: Partition, Np: int, device):
        import torch
        self.part, self.Np = part, Np
        self.K = len(part.local)
        self.send = {s: torch.tensor(ix, device=device) for s, ix in part.send.items()}
        self.recv = {s: torch.tensor(ix, device=device) for s, ix in part.recv.items()}

    def pack(self, ptr: int, V: int, like) -> dict:
        import torch
        out = {}
        for s, ix in self.send.items():
            buf = torch.empty((V, len(ix), self.Np), dtype=torch.float64, device=like.device)
            check(load().dg_gather_elements(ctypes.c_void_p(ptr), V, self.K, self.Np, ctypes.c_void_p(ix.data_ptr()),
                                            len(ix), ctypes.c_void_p(buf.data_ptr()), None))
            out[s] = buf
        return out

    def unpack(self, ptr: int, V: int, received: dict):
        for s, buf in received.items():
            ix = self.recv[s]
            check(load().dg_scatter_elements(ctypes.c_void_p(buf.data_ptr()), V, self.K, self.Np,
                                             ctypes.c_void_p(ix.data_ptr()), len(ix), ctypes.c_void_p(ptr), None))

    def recv_shapes(self, V: int) -> dict:
        return {s: (V, len(ix), self.Np) for s, ix in self.recv.items()}


def viscous_buffer(mesh) -> int:
    p = ctypes.c_void_p()
    check(load().dg_mesh_viscous_buffer(mesh.handle, ctypes.byref(p)))
    return p.value


@dataclass
class RankState:
    """One partition on this process: its mesh, halo exchange, state and RK work buffers."""
    mesh: object
    halo: HaloExchange
    q: object
    work: tuple


def _post(ranks, transport, ptrs, V):
    like = ranks[0].q
    return transport.start([r.halo.pack(p, V, like) for r, p in zip(ranks, ptrs)],
                           [r.halo.recv_shapes(V) for r in ranks], like)


def _finish(ranks, transport, handle, ptrs, V):
    for r, p, g in zip(ranks, ptrs, transport.finish(handle)):
        r.halo.unpack(p, V, g)


def _ptr(a):
    return a if isinstance(a, int) else a.data_ptr()


class LibdgBackend:
    """The partitioned step on the library's kernels (FP64 form, perfect gas): the halo packed and
    unpacked on the device (dg_gather_elements / dg_scatter_elements), the per-node primitives of
    an element range (dg_primitives), the BR1 viscous flux of a range into the mesh's buffer
    (dg_viscous_flux_range, 9 fields per node), the stage of a range by dg_rk_stage with
    prims_given and, when the gas is viscous, viscous_given."""

    flux_vars = 9

    def post(self, ranks, transport, arrays, V):
        return _post(ranks, transport, [_ptr(a) for a in arrays], V)

    def finish(self, ranks, transport, handle, arrays, V):
        _finish(ranks, transport, handle, [_ptr(a) for a in arrays], V)

    def refresh(self, ranks, transport, arrays, V):
        self.finish(ranks, transport, self.post(ranks, transport, arrays, V), arrays, V)

    def primitives(self, rank, gas, q, elems):
        check(load().dg_primitives(rank.mesh.handle, gas.handle, ctypes.c_void_p(q.data_ptr()), int(elems[0]),
                                   int(elems[1]), None))

    def viscous_flux(self, rank, gas, q, elems):
        check(load().dg_viscous_flux_range(rank.mesh.handle, gas.handle, ctypes.c_void_p(q.data_ptr()),
                                           int(elems[0]), int(elems[1]), None))
        return viscous_buffer(rank.mesh)

    def stage(self, rank, gas, s, dt, q_in, q_out, viscous, elems):
        from .dg import _opts, dg_rk_stage
        opts = _opts(elems=elems, viscous_given=viscous, prims_given=True)
        dg_rk_stage(rank.mesh, gas, s, dt, q_in, q_out, rank.work[1], opts=opts)


def _groups(rank):
    """(interior, border, halo) element ranges of a rank's local mesh."""
    p = rank.halo.part
    no, ni = len(p.owned), p.n_interior
    return (0, ni), (ni, no), (no, len(p.local))


def partitioned_lsrk4_step(ranks: list, gas, transport, dt, backend=None):
    """One LSRK4 step of the partitions held by this process (perfect gas).  Each stage:

    * post the exchange of the state's halo;
    * the owned nodes' primitives, then (Navier-Stokes) the interior elements' viscous flux;
    * finish the exchange; the halo nodes' primitives, the border elements' viscous flux;
    * (Navier-Stokes) post the exchange of the viscous flux's halo;
    * the interior elements' stage;
    * finish that exchange; the border elements' stage.

    The interior elements' work reads no halo data, so it overlaps each exchange in flight; every
    node's primitives are computed once per stage, and the halo's right-hand side not at all.
    backend: the compute of one partition (LibdgBackend, the default, runs the library's kernels;
    any object with the same methods and flux_vars works, e.g. a CPU one in the tests)."""
    backend = backend or LibdgBackend()
    if getattr(gas, "model", "perfect") != "perfect":
        raise ValueError("the partitioned step takes a perfect gas")
    V = ranks[0].q.shape[0]
    viscous = gas.mu > 0
    groups = [_groups(r) for r in ranks]
    cur = [r.q for r in ranks]
    nxt = [r.work[0] for r in ranks]
    for s in range(5):
        h = backend.post(ranks, transport, cur, V)
        for r, c, (ig, bg, hg) in zip(ranks, cur, groups):
            backend.primitives(r, gas, c, (ig[0], bg[1]))
            if viscous:
                backend.viscous_flux(r, gas, c, ig)
        backend.finish(ranks, transport, h, cur, V)
        fv = []
        for r, c, (ig, bg, hg) in zip(ranks, cur, groups):
            backend.primitives(r, gas, c, hg)
            if viscous:
                fv.append(backend.viscous_flux(r, gas, c, bg))
        if viscous:
            h = backend.post(ranks, transport, fv, backend.flux_vars)
        for r, c, n, (ig, bg, hg) in zip(ranks, cur, nxt, groups):
            backend.stage(r, gas, s, dt, c, n, viscous, ig)
        if viscous:
            backend.finish(ranks, transport, h, fv, backend.flux_vars)
        for r, c, n, (ig, bg, hg) in zip(ranks, cur, nxt, groups):
            backend.stage(r, gas, s, dt, c, n, viscous, bg)
        cur, nxt = nxt, cur
    for r, c in zip(ranks, cur):
        if c is not r.q:
            r.q.copy_(c)


def partitioned_integrals(ranks: list, transport):
    """The integrals of the conserved variables over the whole mesh (each partition's owned
    elements, then summed across partitions); one device tensor [V] per partition held here."""
    from .dg import dg_integrals
    vals = [dg_integrals(r.mesh, r.q, K_count=len(r.halo.part.owned)) for r in ranks]
    return transport.reduce_all(vals, "sum")


def partitioned_stable_dt(ranks: list, gas, transport, cfl) -> float:
    """CFL / (largest stability rate over every partition's owned elements)."""
    from .dg import dg_max_rate
    vals = [dg_max_rate(r.mesh, gas, r.q, K_count=len(r.halo.part.owned)) for r in ranks]
    return float(cfl) / float(transport.reduce_all(vals, "max")[0].item())
