"""One operator sharded over R ranks by a hash of its z plane.

The multi-device form of the ORQA partition (Sec. II: the operator is the
disjoint sum of partial operators O^(m), Eq. eq:Om, placed by a map f,
Eq. distributor).  Here f is owner(z): a fixed 64-bit mix of the z words
reduced mod R, computed by liborqa (on the host for placement, on the
device for the exchange).

Why z: an X rotation flips x bits only, so a string and every partner it can
merge with in an X layer (P xor X_q) share z.  With strings placed by
owner(z) an X layer -- branching, merging and truncation of Algorithm 1 --
runs on every rank with no data from another.  A ZZ layer maps every string
to exactly one string whose z changes (z' = z xor L x); after it the
strings whose new owner is another rank move there in ONE all-to-all per
layer, and because the layer is a bijection the arriving strings are
distinct from everything already held, so no merge follows.  <0|O|0>
(Eq. magnetization) is one sum over ranks.

Every per-string step runs in liborqa's kernels (orqa_shard_split,
orqa_shard_append, the layer kernels); this module only places the input,
moves the records between ranks (torch.distributed: NCCL between GPUs, gloo
on CPUs) and sums the ranks' scalars.

    engine = GpuShard(Context(n, capacity))          # one per rank / GPU
    ev = ShardedEvolution(engine, TorchComm())
    ev.set_terms(observable)
    for step: ev.apply_layer(zz, delta); ev.apply_layer(xx, delta); m = ev.expect()

The truncation is the absolute one (|c| < delta after every gate), which is
per string and therefore shard-local; the relative one of Eq. (truncation1)
would need a max over ranks after every gate and is not offered here.
"""
from __future__ import annotations

import numpy as np

from . import orqa as B


def owners(z: np.ndarray, n_qubits: int, n_ranks: int) -> np.ndarray:
    """owner(z) of every row of the [N, W] z planes."""
    return B.orqa_shard_owner(n_qubits, z, n_ranks)


def moves_z(gates) -> bool:
    """True if a layer can change z planes (then an exchange follows it):
    ZZ gates can; X gates flip x bits only."""
    for g in gates:
        kind = g[0] if isinstance(g, tuple) else ("rzz" if g.kind == B.ORQA_RZZ else "rx")
        if kind == "rzz":
            return True
    return False


def record_words(n_qubits: int) -> int:
    """uint64 words per exchanged string: x words, z words, coefficient."""
    return 2 * B.words_per_plane(n_qubits) + 1


class TorchComm:
    """Collectives over torch.distributed's default group (NCCL for CUDA
    tensors, gloo for CPU tensors)."""

    def __init__(self):
        import torch.distributed as dist
        self.dist = dist
        self.rank = dist.get_rank()
        self.size = dist.get_world_size()

    def alltoallv(self, send, counts):
        """send: [sum(counts), K] int64 tensor, rows grouped by destination
        rank; returns the rows sent to this rank, grouped by source rank."""
        import torch
        dist = self.dist
        cnt = torch.tensor([int(c) for c in counts], dtype=torch.int64, device=send.device)
        recv_cnt = torch.empty_like(cnt)
        dist.all_to_all_single(recv_cnt, cnt)
        rc = [int(v) for v in recv_cnt.tolist()]
        recv = torch.empty((sum(rc), send.shape[1]), dtype=send.dtype, device=send.device)
        dist.all_to_all_single(recv, send, output_split_sizes=rc, input_split_sizes=[int(c) for c in counts])
        return recv

    def sum(self, value: float, device="cpu") -> float:
        import torch
        t = torch.tensor([float(value)], dtype=torch.float64, device=device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return float(t.item())

    def max(self, value: float, device="cpu") -> float:
        import torch
        t = torch.tensor([float(value)], dtype=torch.float64, device=device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())


class GpuShard:
    """One rank's part of the operator in a liborqa context on this rank's
    GPU, with a device send buffer for the exchange."""

    def __init__(self, ctx, send_capacity: int | None = None):
        import torch
        self.ctx = ctx
        self.n_qubits = ctx.n_qubits
        self.K = record_words(ctx.n_qubits)
        self.device = ctx.device
        cap = send_capacity if send_capacity is not None else ctx.capacity
        self.send = torch.empty((max(1, cap), self.K), dtype=torch.int64, device=self.device)
        self.comm_device = self.device

    def set_terms(self, x, z, c):
        self.ctx.set_operator(x, z, c)

    def apply_layer(self, gates, delta: float):
        return self.ctx.apply_layer(gates, delta)

    def split(self, n_ranks: int, rank: int):
        counts = B.orqa_shard_split(self.ctx.ctx, n_ranks, rank, self.send.shape[0], self.send.data_ptr())
        return self.send[: int(counts.sum())], [int(v) for v in counts]

    def append(self, recv):
        if recv.shape[0]:
            recv = recv.contiguous()
            B.orqa_shard_append(self.ctx.ctx, recv.shape[0], recv.data_ptr())

    def expect(self) -> float:
        return self.ctx.expect()

    def size(self) -> int:
        return len(self.ctx)


class ShardedEvolution:
    """The rank-local driver: every rank builds one with its own engine and
    calls the same methods in the same order (they are collective)."""

    def __init__(self, engine, comm):
        self.engine = engine
        self.comm = comm
        self.exchanged = 0   # strings this rank sent, summed over exchanges

    def set_terms(self, terms):
        """Places the observable: each rank keeps the (label, c) terms whose
        z plane it owns."""
        n = self.engine.n_qubits
        labels = [t[0] for t in terms]
        x, z = B.strings_from_labels(labels, n)
        c = np.array([t[1] for t in terms], dtype=np.float64)
        mine = owners(z, n, self.comm.size) == self.comm.rank if len(c) else np.zeros(0, bool)
        self.engine.set_terms(x[mine], z[mine], c[mine])

    def exchange(self):
        send, counts = self.engine.split(self.comm.size, self.comm.rank)
        self.exchanged += int(sum(counts))
        recv = self.comm.alltoallv(send, counts)
        self.engine.append(recv)

    def apply_layer(self, gates, delta: float):
        self.engine.apply_layer(gates, delta)
        if moves_z(gates):
            self.exchange()

    def expect(self) -> float:
        return self.comm.sum(self.engine.expect(), self.engine.comm_device)

    def size(self) -> int:
        return int(round(self.comm.sum(self.engine.size(), self.engine.comm_device)))


class LocalShards:
    """R shards driven from one process (for example R contexts on one GPU):
    the same steps as ShardedEvolution with the exchange done by device
    copies.  Used to run the sharded path where only one GPU is present."""

    def __init__(self, engines):
        self.engines = list(engines)
        self.R = len(self.engines)
        self.exchanged = 0

    def set_terms(self, terms):
        n = self.engines[0].n_qubits
        x, z = B.strings_from_labels([t[0] for t in terms], n)
        c = np.array([t[1] for t in terms], dtype=np.float64)
        own = owners(z, n, self.R) if len(c) else np.zeros(0, np.int32)
        for r, e in enumerate(self.engines):
            e.set_terms(x[own == r], z[own == r], c[own == r])

    def exchange(self):
        import torch
        sends = [e.split(self.R, r) for r, e in enumerate(self.engines)]
        starts = [np.concatenate([[0], np.cumsum(cnt)]) for _, cnt in sends]
        for r, e in enumerate(self.engines):
            parts = [buf[starts[s][r]: starts[s][r + 1]] for s, (buf, _) in enumerate(sends) if s != r]
            parts = [p.to(e.comm_device) for p in parts if p.shape[0]]
            if parts:
                e.append(torch.cat(parts))
        self.exchanged += int(sum(sum(cnt) for _, cnt in sends))

    def apply_layer(self, gates, delta: float):
        for e in self.engines:
            e.apply_layer(gates, delta)
        if moves_z(gates):
            self.exchange()

    def expect(self) -> float:
        return float(sum(e.expect() for e in self.engines))

    def size(self) -> int:
        return int(sum(e.size() for e in self.engines))

    def sizes(self):
        return [e.size() for e in self.engines]
