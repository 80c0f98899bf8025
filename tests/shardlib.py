"""A shard engine backed by the CPU oracle, for tests of the sharded driver
(paper_2506_13241_gb300.shard) on CPU ranks: the same interface as the
package's GpuShard, with every per-string step done by the oracle and the
owner map taken from liborqa's host function."""
from __future__ import annotations

import numpy as np

from paritylib import codes_to_planes, index_words_to_codes, planes_to_index_words


class OracleShard:
    def __init__(self, n: int, oracle_mod):
        from paper_2506_13241_gb300 import orqa as B
        self.B = B
        self.n = self.n_qubits = n
        self.W = B.words_per_plane(n)
        self.K = 2 * self.W + 1
        self.oracle_mod = oracle_mod
        self.op = oracle_mod.Oracle(n)
        self.comm_device = "cpu"

    def _load(self, x, z, c):
        self.op = self.oracle_mod.Oracle(self.n)
        for key, v in zip(planes_to_index_words(x, z, self.n), c):
            self.op.add(tuple(int(w) for w in key), float(v))

    def set_terms(self, x, z, c):
        self._load(x, z, c)

    def apply_layer(self, gates, delta: float):
        for g in gates:
            self.op.apply(g, delta)

    def planes(self):
        keys, c = self.op.export()
        x, z = codes_to_planes(index_words_to_codes(keys, self.n), self.W)
        return x, z, c

    def split(self, n_ranks: int, rank: int):
        import torch
        x, z, c = self.planes()
        own = self.B.orqa_shard_owner(self.n, z, n_ranks) if len(c) else np.zeros(0, np.int32)
        keep = own == rank
        self._load(x[keep], z[keep], c[keep])
        out = np.nonzero(~keep)[0]
        out = out[np.argsort(own[out], kind="stable")]
        rec = np.zeros((len(out), self.K), dtype=np.uint64)
        rec[:, :self.W] = x[out]
        rec[:, self.W:2 * self.W] = z[out]
        rec[:, 2 * self.W] = c[out].view(np.uint64)
        counts = np.bincount(own[~keep], minlength=n_ranks) if len(out) else np.zeros(n_ranks, np.int64)
        return torch.from_numpy(rec.view(np.int64)), [int(v) for v in counts]

    def append(self, recv):
        rec = recv.numpy().view(np.uint64)
        x, z = rec[:, :self.W], rec[:, self.W:2 * self.W]
        c = rec[:, 2 * self.W].copy().view(np.float64)
        for key, v in zip(planes_to_index_words(x, z, self.n), c):
            self.op.add(tuple(int(w) for w in key), float(v))

    def expect(self) -> float:
        return self.op.expect_zero()

    def size(self) -> int:
        return len(self.op)
