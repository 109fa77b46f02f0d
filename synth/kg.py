"""Seeded synthetic typed knowledge graphs and query sets.

The paper measures on WikiKG90Mv2 (Sec. 4.1, Table 1: 91 M entities, 1,387
relations, 601 M triples, embeddings trimmed to 8 dimensions, K = 50).  That
dataset is not available here, so every workload is synthetic; the recipes
below stand in for it with the same kinds of structure: power-law degrees,
typed vertices, several relation types per vertex pair, dense per-entity and
per-relation embedding tables (Sec. 3.1: three inputs, an edge list of
(h, r, t) triples, an entity embedding table and a relation embedding table).

Random streams: ``numpy.random.default_rng([seed, stream])`` with stream 0 for
the graph, 1 for embeddings, 2 for queries and 3 for training queries.

Canonical graph form (what every consumer receives):
  * CSR by source: ``offsets`` int64[n+1], ``cols`` uint32[E] (destinations),
    ``rels`` uint16[E] (relation ids);
  * each row sorted by (col, rel), no duplicate (u, r, v), no self loops;
  * ``vtypes`` uint8[n]; embeddings row-major [n, d] and [R, d], float32 or
    bfloat16 (stored as uint16 bit patterns).
"""

from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np


# ----------------------------------------------------------------------------
# containers
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class KG:
    n: int
    R: int
    n_types: int
    offsets: np.ndarray  # int64[n+1]
    cols: np.ndarray     # uint32[E]
    rels: np.ndarray     # uint16[E]
    vtypes: np.ndarray   # uint8[n]
    vemb: Optional[np.ndarray] = None  # float32[n,d] or uint16[n,d] (bf16 bits)
    remb: Optional[np.ndarray] = None  # float32[R,d] or uint16[R,d]
    dtype: str = "f32"   # "f32" | "bf16"

    @property
    def E(self) -> int:
        return int(self.cols.shape[0])

    @property
    def d(self) -> int:
        return int(self.vemb.shape[1]) if self.vemb is not None else 0

    def out_degree(self) -> np.ndarray:
        return np.diff(self.offsets)

    def in_degree(self) -> np.ndarray:
        return np.bincount(self.cols, minlength=self.n).astype(np.int64)

    def src_of_edges(self) -> np.ndarray:
        return np.repeat(np.arange(self.n, dtype=np.uint32), self.out_degree())

    def vemb_f32(self) -> np.ndarray:
        return self.vemb if self.dtype == "f32" else bf16_bits_to_f32(self.vemb)

    def remb_f32(self) -> np.ndarray:
        return self.remb if self.dtype == "f32" else bf16_bits_to_f32(self.remb)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


# ----------------------------------------------------------------------------
# canonical CSR
# ----------------------------------------------------------------------------
def _triple_keys(n: int, R: int, u: np.ndarray, r: np.ndarray, v: np.ndarray) -> np.ndarray:
    # key order (u, v, r) == CSR row order followed by (col, rel) inside a row
    return (u.astype(np.uint64) * np.uint64(n) + v.astype(np.uint64)) * np.uint64(R) + r.astype(np.uint64)


def _keys_to_csr(n: int, R: int, keys: np.ndarray):
    keys = np.sort(keys)
    r = (keys % np.uint64(R)).astype(np.uint16)
    uv = keys // np.uint64(R)
    v = (uv % np.uint64(n)).astype(np.uint32)
    u = (uv // np.uint64(n)).astype(np.int64)
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(u, minlength=n), out=offsets[1:])
    return offsets, v, r


def canonicalize(n: int, R: int, src, rel, dst):
    """Edge list -> canonical CSR (sorted rows, no duplicate triple, no self loop)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    rel = np.asarray(rel, dtype=np.int64)
    if src.size and (src.min() < 0 or src.max() >= n or dst.min() < 0 or dst.max() >= n):
        raise ValueError("vertex id out of range")
    if rel.size and (rel.min() < 0 or rel.max() >= R):
        raise ValueError("relation id out of range")
    keep = src != dst
    keys = np.unique(_triple_keys(n, R, src[keep], rel[keep], dst[keep]))
    return _keys_to_csr(n, R, keys)


# ----------------------------------------------------------------------------
# embeddings
# ----------------------------------------------------------------------------
def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 bit patterns, round to nearest even."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    rounding = ((b >> np.uint32(16)) & np.uint32(1)) + np.uint32(0x7FFF)
    return ((b + rounding) >> np.uint32(16)).astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.ascontiguousarray(b, dtype=np.uint16).astype(np.uint32) << np.uint32(16)).view(np.float32)


def gen_embeddings(n: int, R: int, d: int, var: float, seed: int = 0, dtype: str = "f32"):
    """Entity and relation tables with i.i.d. N(0, var) entries (var = variance)."""
    rng = _rng(seed, 1)
    std = np.float32(math.sqrt(var))
    vemb = rng.standard_normal((n, d), dtype=np.float32) * std
    remb = rng.standard_normal((R, d), dtype=np.float32) * std
    if dtype == "bf16":
        return to_bf16_bits(vemb), to_bf16_bits(remb)
    if dtype != "f32":
        raise ValueError(dtype)
    return vemb, remb


# ----------------------------------------------------------------------------
# graphs
# ----------------------------------------------------------------------------
def gen_zipf_kg(n: int, E: int, R: int, n_types: int, alpha: float = 2.1, seed: int = 0) -> KG:
    """Out-degree ~ Zipf(alpha) truncated to [1, n-1] and rescaled to sum to E
    exactly; destinations uniform over v != u, relation uniform per edge, no
    duplicate (v, r) inside a row."""
    rng = _rng(seed, 0)
    raw = rng.zipf(alpha, size=n).astype(np.float64)
    raw = np.minimum(raw, n - 1)
    f = raw * (E / raw.sum())
    deg = np.maximum(np.floor(f).astype(np.int64), 1)
    cap = min(n - 1, (n - 1) * R)
    deg = np.minimum(deg, cap)
    resid = E - int(deg.sum())
    frac_order = np.lexsort((np.arange(n), -(f - np.floor(f))))
    i = 0
    while resid > 0:
        u = frac_order[i % n]
        if deg[u] < cap:
            deg[u] += 1
            resid -= 1
        i += 1
    big_order = np.lexsort((np.arange(n), -deg))
    i = 0
    while resid < 0:
        u = big_order[i % n]
        if deg[u] > 1:
            deg[u] -= 1
            resid += 1
        i += 1
    vtypes = rng.integers(0, n_types, size=n, dtype=np.uint8)
    # draw rows, redraw the deficit of rows that lost edges to duplicates
    keys = np.zeros(0, dtype=np.uint64)
    need = deg.copy()
    while True:
        tot = int(need.sum())
        if tot == 0:
            break
        u = np.repeat(np.arange(n, dtype=np.int64), need)
        v = rng.integers(0, n - 1, size=tot, dtype=np.int64)
        v = v + (v >= u)
        r = rng.integers(0, R, size=tot, dtype=np.int64)
        keys = np.unique(np.concatenate([keys, _triple_keys(n, R, u, r, v)]))
        have = np.bincount((keys // np.uint64(R) // np.uint64(n)).astype(np.int64), minlength=n)
        extra = have - deg
        if (extra > 0).any():
            # drop surplus draws of a row from its end (deterministic)
            ku = (keys // np.uint64(R) // np.uint64(n)).astype(np.int64)
            start = np.zeros(n + 1, dtype=np.int64)
            np.cumsum(have, out=start[1:])
            pos = np.arange(keys.size, dtype=np.int64) - start[ku]
            keys = keys[pos < deg[ku]]
            have = np.minimum(have, deg)
        need = deg - have
    offsets, cols, rels = _keys_to_csr(n, R, keys)
    return KG(n=n, R=R, n_types=n_types, offsets=offsets, cols=cols, rels=rels, vtypes=vtypes)


def gen_rmat_kg(scale: int, n: int, E: int, R: int, n_types: int,
                a: float = 0.57, b: float = 0.19, c: float = 0.19, seed: int = 0) -> KG:
    """R-MAT edges at ``scale`` (quadrant probabilities a, b, c, 1-a-b-c);
    edges with an endpoint >= n are rejected, vertex ids are permuted with a
    seeded permutation, self loops dropped, and draws continue until exactly E
    unique (u, r, v) triples exist (the first E in draw order are kept)."""
    if n > (1 << scale):
        raise ValueError("n exceeds 2**scale")
    rng = _rng(seed, 0)
    perm = rng.permutation(n).astype(np.int64)
    vtypes = rng.integers(0, n_types, size=n, dtype=np.uint8)
    ab, abc = a + b, a + b + c
    uniq = np.zeros(0, dtype=np.uint64)
    first = np.zeros(0, dtype=np.int64)
    drawn = 0
    while uniq.size < E:
        m = int((E - uniq.size) * 1.25) + 1024
        u = np.zeros(m, dtype=np.int64)
        v = np.zeros(m, dtype=np.int64)
        for _ in range(scale):
            q = rng.random(m, dtype=np.float32)
            sb = q >= ab
            db = ((q >= a) & (q < ab)) | (q >= abc)
            u = (u << 1) | sb
            v = (v << 1) | db
        r = rng.integers(0, R, size=m, dtype=np.int64)
        ok = (u < n) & (v < n)
        u, v, r = perm[u[ok]], perm[v[ok]], r[ok]
        ok = u != v
        u, v, r = u[ok], v[ok], r[ok]
        k = _triple_keys(n, R, u, r, v)
        order = np.arange(k.size, dtype=np.int64) + drawn
        drawn += k.size
        allk = np.concatenate([uniq, k])
        allf = np.concatenate([first, order])
        uk, idx = np.unique(allk, return_index=True)
        uniq, first = uk, allf[idx]
    if uniq.size > E:
        keep = np.argsort(first, kind="stable")[:E]
        uniq = uniq[keep]
    offsets, cols, rels = _keys_to_csr(n, R, uniq)
    return KG(n=n, R=R, n_types=n_types, offsets=offsets, cols=cols, rels=rels, vtypes=vtypes)


# ----------------------------------------------------------------------------
# queries
# ----------------------------------------------------------------------------
def queries_hub(g: KG):
    """One query: s = largest out-degree, t = largest in-degree (lowest id on
    ties; the next best if it equals s)."""
    od = g.out_degree()
    idg = g.in_degree()
    s = int(np.lexsort((np.arange(g.n), -od))[0])
    order = np.lexsort((np.arange(g.n), -idg))
    t = int(order[0]) if int(order[0]) != s else int(order[1])
    return np.array([s], dtype=np.uint32), np.array([t], dtype=np.uint32)


def queries_edge_biased(g: KG, nq: int, seed: int = 0, stream: int = 2):
    """s = source of a uniform random edge, t = destination of another uniform
    random edge, t != s (degree-biased endpoints)."""
    rng = _rng(seed, stream)
    src = None
    S = np.zeros(nq, dtype=np.uint32)
    T = np.zeros(nq, dtype=np.uint32)
    for i in range(nq):
        e = int(rng.integers(0, g.E))
        s = int(np.searchsorted(g.offsets, e, side="right") - 1)
        while True:
            t = int(g.cols[int(rng.integers(0, g.E))])
            if t != s:
                break
        S[i], T[i] = s, t
    del src
    return S, T


def queries_log_degree(g: KG, nq: int, max_deg: float = 1e5, seed: int = 0, stream: int = 2):
    """x ~ log-uniform[1, max_deg]; s uniform among vertices whose out-degree
    lies in bucket floor(log2 x) (redraw if empty); t = destination of a random
    edge, t != s."""
    rng = _rng(seed, stream)
    od = g.out_degree()
    bucket = np.full(g.n, -1, dtype=np.int64)
    nz = od > 0
    bucket[nz] = np.floor(np.log2(od[nz])).astype(np.int64)
    members = {}
    for bk in np.unique(bucket[nz]):
        members[int(bk)] = np.flatnonzero(bucket == bk)
    S = np.zeros(nq, dtype=np.uint32)
    T = np.zeros(nq, dtype=np.uint32)
    for i in range(nq):
        while True:
            x = math.exp(rng.random() * math.log(max_deg))
            bk = int(math.floor(math.log2(x)))
            if bk in members:
                mem = members[bk]
                s = int(mem[int(rng.integers(0, mem.size))])
                break
        while True:
            t = int(g.cols[int(rng.integers(0, g.E))])
            if t != s:
                break
        S[i], T[i] = s, t
    return S, T


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------
WORKLOADS = {
    # 10k vertices / 4 types, 8 relations, 100k edges, Zipf(2.1) out-degree,
    # d=64 fp32 ~ N(0, 1/8); one hub query, K = 10
    "tiny": dict(kind="zipf", n=10_000, E=100_000, R=8, n_types=4, d=64, var=1 / 8,
                 dtype="f32", queries="hub", nq=1, K=10, score="transe"),
    # R-MAT (.57,.19,.19) scale 20 cut to 1M vertices, 20M edges, 16 relations,
    # 6 types, d=128 fp32 ~ N(0, 1/sqrt(d)); 64 edge-biased queries, K = 100
    "medium": dict(kind="rmat", scale=20, n=1_000_000, E=20_000_000, R=16, n_types=6, d=128,
                   var=None, dtype="f32", queries="edge", nq=64, K=100, score="transe"),
    # the medium graph with d=256; 256 queries, K = 100, DistMult
    "precision": dict(kind="rmat", scale=20, n=1_000_000, E=20_000_000, R=16, n_types=6, d=256,
                      var=None, dtype="f32", queries="edge", nq=256, K=100, score="distmult"),
    # learned ordering: the precision graph and queries with K = 50 (K = 500 by override)
    "learned": dict(kind="rmat", scale=20, n=1_000_000, E=20_000_000, R=16, n_types=6, d=256,
                    var=None, dtype="f32", queries="edge", nq=256, K=50, score="distmult"),
    # R-MAT scale 24 cut to 10M vertices, 200M edges, 32 relations, d=128 bf16;
    # 4096 queries with log-uniform source degree in [1, 1e5], K = 50
    "batching": dict(kind="rmat", scale=24, n=10_000_000, E=200_000_000, R=32, n_types=6, d=128,
                     var=None, dtype="bf16", queries="logdeg", nq=4096, K=50, score="transe"),
    # the batching recipe at a quarter of its size (about 2 GB on the device: the
    # case for full-metric profiler captures): R-MAT scale 22 cut to 2.5M vertices,
    # 50M edges, 1,024 log-degree queries, K = 50
    "batching_quarter": dict(kind="rmat", scale=22, n=2_500_000, E=50_000_000, R=32, n_types=6, d=128,
                             var=None, dtype="bf16", queries="logdeg", nq=1024, K=50, score="transe"),
}


def _cache_path(name, seed, spec):
    import hashlib
    import json
    import os
    d = os.environ.get("MHR_SYNTH_CACHE")
    if not d:
        return None
    key = hashlib.sha1(json.dumps([name, seed, sorted(spec.items())], default=str).encode()).hexdigest()[:16]
    os.makedirs(d, exist_ok=True)
    return os.path.join(d, f"{name}-{key}.npz")


def workload(name: str, seed: int = 0, **override):
    """Build a named workload.  Returns (KG with embeddings, S, T, K, spec).
    Set MHR_SYNTH_CACHE to a directory to reuse generated arrays."""
    spec = dict(WORKLOADS[name])
    spec.update(override)
    cp = _cache_path(name, seed, spec)
    if cp is not None:
        import os
        if os.path.exists(cp):
            z = np.load(cp)
            g = KG(n=spec["n"], R=spec["R"], n_types=spec["n_types"], offsets=z["offsets"],
                   cols=z["cols"], rels=z["rels"], vtypes=z["vtypes"], vemb=z["vemb"],
                   remb=z["remb"], dtype=spec["dtype"])
            return g, z["S"], z["T"], spec["K"], spec
    g, S, T, K, spec = _build_workload(spec, seed)
    if cp is not None:
        import os
        tmp = f"{cp}.{os.getpid()}.tmp.npz"  # one writer per file; the rename is atomic
        try:
            np.savez(tmp, offsets=g.offsets, cols=g.cols, rels=g.rels, vtypes=g.vtypes, vemb=g.vemb,
                     remb=g.remb, S=S, T=T)
            os.replace(tmp, cp)
        except OSError:  # no room for the cache: keep going without it
            try:
                os.unlink(tmp)
            except OSError:
                pass
    return g, S, T, K, spec


def _build_workload(spec, seed):
    if spec["kind"] == "zipf":
        g = gen_zipf_kg(spec["n"], spec["E"], spec["R"], spec["n_types"], seed=seed)
    else:
        g = gen_rmat_kg(spec["scale"], spec["n"], spec["E"], spec["R"], spec["n_types"], seed=seed)
    var = spec["var"] if spec["var"] is not None else 1.0 / math.sqrt(spec["d"])
    g.vemb, g.remb = gen_embeddings(g.n, g.R, spec["d"], var, seed=seed, dtype=spec["dtype"])
    g.dtype = spec["dtype"]
    if spec["queries"] == "hub":
        S, T = queries_hub(g)
    elif spec["queries"] == "edge":
        S, T = queries_edge_biased(g, spec["nq"], seed=seed)
    else:
        S, T = queries_log_degree(g, spec["nq"], seed=seed)
    return g, S, T, spec["K"], spec
