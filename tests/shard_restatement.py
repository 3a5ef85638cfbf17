"""A test-only restatement of one shard's steps of point-sharded seeding
(multi.seed_sharded), in NumPy FP64, for integer coordinates.

It stands in for the GPU kernels (kpp_shard_first / _pass / _pick / _phi) so
that the host protocol -- the order of the steps and the two exchanges per
pass -- can run on CPU processes over gloo.  With integer coordinates every
D^2, every total and every prefix is an exact integer, so the draws follow
Algorithm 1's probability line exactly and the result must be the oracle's
bit for bit.  The exchange buffer has the library's layout: the centre's
global index, its scale word, then the stored FP32 row as 64-bit words.
"""
from __future__ import annotations

import math

import numpy as np
import torch

import oracle


class CpuShard:
    def __init__(self, x_local: np.ndarray, row0: int, n_global: int, K: int, seed: int,
                 stream_id: int, rank: int, world: int):
        self.xf = np.ascontiguousarray(x_local, dtype=np.float32)
        self.x = self.xf.astype(np.float64)
        self.n, self.d = self.x.shape
        self.row0, self.N, self.K = row0, n_global, K
        self.seed, self.stream, self.rank, self.world = seed, stream_id, rank, world
        self.words = 2 + 2 * math.ceil(self.d * 4 / 16)
        self.exchange = torch.zeros(self.words, dtype=torch.int64)
        self.total = torch.zeros(2, dtype=torch.float32)
        self.totals = torch.zeros(2 * world, dtype=torch.float32)
        self.idx = np.full(K, -1, dtype=np.int64)
        self.d2 = np.zeros(self.n)
        self.phi = None
        self.status = oracle.OK

    def _put(self, i_local: int):
        ex = np.zeros(self.words, dtype=np.int64)
        ex[0] = self.row0 + i_local
        row = np.zeros((self.words - 2) * 2, dtype=np.float32)
        row[: self.d] = self.xf[i_local]
        ex[2:] = row.view(np.int64)
        self.exchange.copy_(torch.from_numpy(ex))

    def _rank_totals(self):
        t = self.totals.numpy().astype(np.float64).reshape(-1, 2)
        return t[:, 0] + t[:, 1]

    def first(self):
        self.exchange.zero_()
        i0 = min(int(math.floor(oracle.uniform(self.seed, self.stream, 0) * self.N)), self.N - 1)
        if self.row0 <= i0 < self.row0 + self.n:
            self._put(i0 - self.row0)

    def local_pass(self, m: int):
        if self.status != oracle.OK:
            return
        ex = self.exchange.numpy()
        self.idx[m] = int(ex[0])
        c = ex[2:].view(np.float32)[: self.d].astype(np.float64)
        delta = ((self.x - c) ** 2).sum(axis=1)
        self.d2 = delta if m == 0 else np.minimum(self.d2, delta)
        T = float(self.d2.sum())
        hi = np.float32(T)
        lo = np.float32(T - float(hi))
        self.total.copy_(torch.tensor([hi, lo], dtype=torch.float32))

    def pick(self, m: int):
        if self.status != oracle.OK:
            return
        self.exchange.zero_()
        tot = self._rank_totals()
        T = float(tot.sum())
        if T == 0.0:
            self.idx[m + 1:] = -1
            self.status = oracle.DEGENERATE
            return
        t = oracle.uniform(self.seed, self.stream, m + 1) * T
        cum = np.cumsum(tot)
        over = np.nonzero(cum > t)[0]
        owner = int(over[0]) if over.size else int(np.nonzero(tot > 0)[0][-1])
        if owner != self.rank:
            return
        base = float(cum[owner - 1]) if owner > 0 else 0.0
        P = base + np.cumsum(self.d2)
        hit = np.nonzero(P > t)[0]
        i = int(hit[0]) if hit.size else int(np.nonzero(self.d2 > 0)[0][-1])
        self._put(i)

    def finish(self):
        self.phi = float(self._rank_totals().sum())
