"""Second, independent oracle route: meet in the middle, pure Python.

TEST INFRASTRUCTURE ONLY.  Shares no code with ``mhr_oracle.c``: it has its
own edge-weight loop (same canonical fp64 operation order, Python floats are
IEEE doubles and Python never fuses a multiply-add) and finds paths the other
way round: a map of the out-edges of s, a map of the in-edges of t built by
scanning every edge, and a join over the middle edges.  Every path is
materialised and sorted, so it is only for small graphs.

Definitions followed: TransE-L1 score gamma - sum_j |h_j + r_j - t_j|
(Alg. 3, Alg. 4, Sec. 3.1); DistMult sum_j h_j r_j t_j; simple paths with the
target ending a path (Alg. 7); path score = sum of edge weights; order score
descending then (u, r1, v, r2, r3) ascending.
"""

from __future__ import annotations

import numpy as np


def _rows_as_floats(tab: np.ndarray, dtype: str):
    if dtype == "bf16":
        tab = (np.asarray(tab, dtype=np.uint16).astype(np.uint32) << np.uint32(16)).view(np.float32)
    return [[float(x) for x in row] for row in np.asarray(tab, dtype=np.float32)]


class MITM:
    def __init__(self, g, fn: str = "transe", gamma: float = 1.0):
        self.g = g
        self.fn = fn
        self.gamma = float(gamma)
        self.E = _rows_as_floats(g.vemb, g.dtype)
        self.Rr = _rows_as_floats(g.remb, g.dtype)
        self.off = [int(x) for x in g.offsets]
        self.cols = [int(x) for x in g.cols]
        self.rels = [int(x) for x in g.rels]

    def weight(self, u: int, r: int, v: int) -> float:
        h, rr, t = self.E[u], self.Rr[r], self.E[v]
        acc = 0.0
        if self.fn == "transe":
            for j in range(len(h)):
                acc = acc + abs((h[j] + rr[j]) - t[j])
            return self.gamma - acc
        for j in range(len(h)):
            acc = acc + (h[j] * rr[j]) * t[j]
        return acc

    def all_paths(self, s: int, t: int):
        """Every simple s->t three-hop path, sorted; tuples (S, u, r1, v, r2, r3)."""
        if s == t:
            raise ValueError("s == t")
        off, cols, rels = self.off, self.cols, self.rels
        out_s = {}
        for i in range(off[s], off[s + 1]):
            u = cols[i]
            if u in (s, t):
                continue
            out_s.setdefault(u, []).append((rels[i], self.weight(s, rels[i], u)))
        in_t = {}
        for v in range(self.g.n):
            if v in (s, t):
                continue
            for k in range(off[v], off[v + 1]):
                if cols[k] == t:
                    in_t.setdefault(v, []).append((rels[k], self.weight(v, rels[k], t)))
        paths = []
        for u, a_list in out_s.items():
            for j in range(off[u], off[u + 1]):
                v = cols[j]
                if v == u or v not in in_t:
                    continue
                r2 = rels[j]
                w2 = self.weight(u, r2, v)
                for r1, w1 in a_list:
                    for r3, w3 in in_t[v]:
                        paths.append(((w1 + w2) + w3, u, r1, v, r2, r3))
        paths.sort(key=lambda p: (-p[0], p[1], p[2], p[3], p[4], p[5]))
        return paths

    def topk(self, s: int, t: int, K: int):
        if K <= 0:
            raise ValueError("K <= 0")
        return self.all_paths(s, t)[:K]
