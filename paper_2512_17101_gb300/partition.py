"""Element partitions of a tetrahedral mesh for the multi-process form, and their halo exchange.

The paper runs its largest cases over many GPUs, exchanging face data between the ranks of a
domain decomposition (§5.4).  Here a rank uploads its owned elements followed by copies of their
face neighbours owned by other ranks (halo elements; their faces that lead out of the local set
carry DG_BC_OUTFLOW, so the local mesh is closed; the halo's own right-hand side is never used).
Before each right-hand side the halo copies are refreshed from their owners; for Navier-Stokes the
viscous flux is computed, its halo refreshed the same way, and the stage then uses it
(`dg_opts.viscous_given`).  The library moves the data (`dg_gather_elements`,
`dg_scatter_elements`); the transport between ranks is a small object with one method,
`exchange_all(sends, recv_shapes, like)`, and one more for the global reductions,
`reduce_all(values, op)` (op "sum" or "max"): `TorchTransport` uses torch.distributed point-to-point
messages (NCCL on GPUs, gloo on CPUs) for the one partition a process holds, `LocalRouter` hands
the buffers between partitions held by one process.

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
    owned: np.ndarray            # global element ids owned by this rank (ascending)
    halo: np.ndarray             # global ids of the halo elements (ascending)
    vertices: np.ndarray         # [len(owned) + len(halo)][4][3]
    face_bc: np.ndarray          # [len(owned) + len(halo)][4]
    send: dict = field(default_factory=dict)   # rank -> local indices of owned elements it holds as halo
    recv: dict = field(default_factory=dict)   # rank -> local indices of the halo elements it owns

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
        local = np.concatenate([owned, halo])
        in_local = np.zeros(K, dtype=bool)
        in_local[local] = True
        fbc = gbc[local].copy()
        hp = partner[halo]  # [H][4]
        leaves = (hp >= 0) & ~in_local[np.maximum(hp, 0)]
        fbc[len(owned):][leaves] = OUTFLOW  # halo faces leading out of the local set
        parts.append(Partition(rank=r, owned=owned, halo=halo, vertices=np.ascontiguousarray(v[local]),
                               face_bc=np.ascontiguousarray(fbc, dtype=np.int32)))
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

    def exchange_all(self, sends: list, recv_shapes: list, like) -> list:
        import torch
        import torch.distributed as dist
        assert len(sends) == 1, "a process holds one partition"
        out = {s: torch.empty(shape, dtype=like.dtype, device=like.device) for s, shape in recv_shapes[0].items()}
        reqs = [dist.irecv(out[s], src=s, group=self.group) for s in out]
        reqs += [dist.isend(buf.contiguous(), dst=s, group=self.group) for s, buf in sends[0].items()]
        for r in reqs:
            r.wait()
        return [out]

    def reduce_all(self, values: list, op: str) -> list:
        import torch.distributed as dist
        assert len(values) == 1, "a process holds one partition"
        t = values[0].clone()
        dist.all_reduce(t, op=dist.ReduceOp.SUM if op == "sum" else dist.ReduceOp.MAX, group=self.group)
        return [t]


class LocalRouter:
    """Exchange among partitions held by one process (each message is the sender's buffer)."""

    def exchange_all(self, sends: list, recv_shapes: list, like) -> list:
        out = [dict() for _ in sends]
        for r, sd in enumerate(sends):
            for s, buf in sd.items():
                out[s][r] = buf
        for r, shapes in enumerate(recv_shapes):
            for s, shape in shapes.items():
                assert tuple(out[r][s].shape) == tuple(shape), "send and receive lists do not pair up"
        return out

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


def _refresh(ranks, transport, ptrs, V):
    like = ranks[0].q
    got = transport.exchange_all([r.halo.pack(p, V, like) for r, p in zip(ranks, ptrs)],
                                 [r.halo.recv_shapes(V) for r in ranks], like)
    for r, p, g in zip(ranks, ptrs, got):
        r.halo.unpack(p, V, g)


class LibdgBackend:
    """The partitioned step on the library's kernels (FP64 form, perfect gas): the halo packed and
    unpacked on the device (dg_gather_elements / dg_scatter_elements), the BR1 viscous flux into
    the mesh's buffer (dg_viscous_flux, 9 fields per node), the stage by dg_rk_stage with
    viscous_given when the gas is viscous."""

    flux_vars = 9

    def refresh(self, ranks, transport, arrays, V):
        _refresh(ranks, transport, [a if isinstance(a, int) else a.data_ptr() for a in arrays], V)

    def viscous_flux(self, rank, gas, q):
        check(load().dg_viscous_flux(rank.mesh.handle, gas.handle, ctypes.c_void_p(q.data_ptr()), None))
        return viscous_buffer(rank.mesh)

    def stage(self, rank, gas, s, dt, q_in, q_out, viscous):
        from .dg import _opts, dg_rk_stage
        opts = _opts()
        opts.viscous_given = 1 if viscous else 0
        dg_rk_stage(rank.mesh, gas, s, dt, q_in, q_out, rank.work[1], opts=opts)


def partitioned_lsrk4_step(ranks: list, gas, transport, dt, backend=None):
    """One LSRK4 step of the partitions held by this process (perfect gas).  Before every stage the
    halos of the states are refreshed; with viscosity each partition's viscous flux is computed,
    its halo refreshed, and the stage uses it (the two exchanges of a BR1 right-hand side).
    backend: the compute of one partition (LibdgBackend, the default, runs the library's kernels;
    any object with the same three methods and flux_vars works, e.g. a CPU one in the tests)."""
    backend = backend or LibdgBackend()
    if getattr(gas, "model", "perfect") != "perfect":
        raise ValueError("the partitioned step takes a perfect gas")
    V = ranks[0].q.shape[0]
    viscous = gas.mu > 0
    cur = [r.q for r in ranks]
    nxt = [r.work[0] for r in ranks]
    for s in range(5):
        backend.refresh(ranks, transport, cur, V)
        if viscous:
            fv = [backend.viscous_flux(r, gas, c) for r, c in zip(ranks, cur)]
            backend.refresh(ranks, transport, fv, backend.flux_vars)
        for r, c, n in zip(ranks, cur, nxt):
            backend.stage(r, gas, s, dt, c, n, viscous)
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
