"""CPU oracle for exact three-hop top-K path search (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It never imports the CUDA package and
the CUDA package never imports it.

Two independent routes compute the same result:
  * ``mhr_oracle.c`` (brute force, fp64, canonical operation order) through
    ctypes: ``edge_weights``, ``topk_paths``, ``topk_paths_batch``,
    ``query_stats``, ``topk_paths_masked`` (relation and vertex-type
    constraints per hop, the query shape of Sec. 3.1), the tail-prediction scan of Alg. 3 / Alg. 4,
    ``tail_topk`` (every candidate vertex of one type scored against a
    (head, relation) pair, the K best kept), and the generic H-hop search with
    a per-path beam of Alg. 6 / Alg. 7, ``beam_paths``;
  * ``mitm.py``: a pure-Python meet-in-the-middle enumeration with its own
    edge-weight loop, used to cross-check the brute force on small graphs.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

TRANSE_L1 = 0
DISTMULT = 1
F32 = 0
BF16 = 1

PATH_DTYPE = np.dtype([("score", "<f8"), ("u", "<u4"), ("v", "<u4"),
                       ("r1", "<u2"), ("r2", "<u2"), ("r3", "<u2"), ("pad", "<u2")])
TAIL_DTYPE = np.dtype([("score", "<f8"), ("v", "<u4"), ("pad", "<u4")])
BEAM_MAX_H = 8
BPATH_DTYPE = np.dtype([("score", "<f8"), ("hops", "<i4"), ("v", "<u4", (BEAM_MAX_H + 1,)),
                        ("r", "<u2", (BEAM_MAX_H,))])
STATS_DTYPE = np.dtype([(k, "<i8") for k in
                        ("deg_s", "deg_t", "n_u", "n_v", "s_f", "s_b", "hits", "paths")])

FN_CODES = {"transe": TRANSE_L1, "transe_l1": TRANSE_L1, "distmult": DISTMULT}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no -ffast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, f64, u32 = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_uint32
        lib.oracle_edge_weight.restype = f64
        lib.oracle_edge_weight.argtypes = [P, P, i32, i32, i32, f64, u32, u32, u32]
        lib.oracle_edge_weights.restype = i32
        lib.oracle_edge_weights.argtypes = [P, P, i32, i32, i32, f64, P, P, P, i64, P]
        lib.oracle_topk_paths.restype = i32
        lib.oracle_topk_paths.argtypes = [P, P, P, i64, P, P, i32, i32, i32, f64, u32, u32, i64,
                                          P, P, P, P]
        lib.oracle_topk_paths_batch.restype = i32
        lib.oracle_topk_paths_batch.argtypes = [P, P, P, i64, P, P, i32, i32, i32, f64, i64, P, P,
                                                i64, P, P, P]
        lib.oracle_query_stats.restype = i32
        lib.oracle_query_stats.argtypes = [P, P, i64, u32, u32, P]
        lib.oracle_tail_topk_batch.restype = i32
        lib.oracle_tail_topk_batch.argtypes = [P, i64, i64, P, P, i32, i32, i32, f64, i64, P, P,
                                               i32, i64, P, P, P]
        lib.oracle_topk_paths_masked.restype = i32
        lib.oracle_topk_paths_masked.argtypes = [P, P, P, i64, P, P, P, i32, i32, i32, f64, u32, u32, P, P, P,
                                                 P, P, i64, P, P]
        lib.oracle_beam_paths.restype = i32
        lib.oracle_beam_paths.argtypes = [P, P, P, i64, P, P, i32, i32, i32, f64, u32, u32, i32, i64, P, P,
                                          P]
        lib.oracle_beam_paths_batch.restype = i32
        lib.oracle_beam_paths_batch.argtypes = [P, P, P, i64, P, P, i32, i32, i32, f64, i64, P, P, i32, i64, P,
                                                P, P]
        lib.oracle_num_threads.restype = i32
        lib.oracle_num_threads.argtypes = []
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class _G:
    """Contiguous views of a synth.KG the C oracle reads."""

    def __init__(self, g):
        self.n = int(g.n)
        self.offsets = np.ascontiguousarray(g.offsets, dtype=np.int64)
        self.cols = np.ascontiguousarray(g.cols, dtype=np.uint32)
        self.rels = np.ascontiguousarray(g.rels, dtype=np.uint16)
        if g.dtype == "f32":
            self.vemb = np.ascontiguousarray(g.vemb, dtype=np.float32)
            self.remb = np.ascontiguousarray(g.remb, dtype=np.float32)
            self.dtype = F32
        else:
            self.vemb = np.ascontiguousarray(g.vemb, dtype=np.uint16)
            self.remb = np.ascontiguousarray(g.remb, dtype=np.uint16)
            self.dtype = BF16
        self.d = int(self.vemb.shape[1])


def edge_weights(g, src, rel, dst, fn="transe", gamma=1.0) -> np.ndarray:
    lib = _load()
    G = _G(g)
    src = np.ascontiguousarray(src, dtype=np.uint32)
    rel = np.ascontiguousarray(rel, dtype=np.uint16)
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    out = np.zeros(src.shape[0], dtype=np.float64)
    rc = lib.oracle_edge_weights(_ptr(G.vemb), _ptr(G.remb), G.dtype, G.d, FN_CODES[fn],
                                 float(gamma), _ptr(src), _ptr(rel), _ptr(dst), src.shape[0],
                                 _ptr(out))
    if rc:
        raise RuntimeError(f"oracle_edge_weights: {rc}")
    return out


def topk_paths(g, s: int, t: int, K: int, fn="transe", gamma=1.0, with_counts=False):
    """The K best simple s->t three-hop paths (structured array, PATH_DTYPE)."""
    lib = _load()
    G = _G(g)
    out = np.zeros(max(int(K), 1), dtype=PATH_DTYPE)
    n_out = np.zeros(1, dtype=np.int64)
    hits = np.zeros(1, dtype=np.int64)
    paths = np.zeros(1, dtype=np.int64)
    rc = lib.oracle_topk_paths(_ptr(G.offsets), _ptr(G.cols), _ptr(G.rels), G.n, _ptr(G.vemb),
                               _ptr(G.remb), G.dtype, G.d, FN_CODES[fn], float(gamma), int(s),
                               int(t), int(K), _ptr(out), _ptr(n_out), _ptr(hits), _ptr(paths))
    if rc == 1:
        raise ValueError("invalid query (s, t out of range, s == t, or K <= 0)")
    if rc:
        raise RuntimeError(f"oracle_topk_paths: {rc}")
    res = out[: int(n_out[0])].copy()
    if with_counts:
        return res, int(hits[0]), int(paths[0])
    return res


def topk_paths_masked(g, s: int, t: int, K: int, rel1=None, rel2=None, rel3=None, types_u=None,
                      types_v=None, fn="transe", gamma=1.0):
    """The K best simple s->t three-hop paths whose relations lie in rel1 /
    rel2 / rel3 and whose intermediate vertex types lie in types_u / types_v
    (each an iterable of allowed ids; None allows every id)."""
    lib = _load()
    G = _G(g)

    def flags(allowed, size):
        f = np.zeros(size, dtype=np.uint8)
        if allowed is None:
            f[:] = 1
        else:
            f[np.asarray(list(allowed), dtype=np.int64)] = 1
        return f

    m1, m2, m3 = flags(rel1, g.R), flags(rel2, g.R), flags(rel3, g.R)
    tu, tv = flags(types_u, 256), flags(types_v, 256)
    vt = np.ascontiguousarray(g.vtypes, dtype=np.uint8)
    out = np.zeros(max(int(K), 1), dtype=PATH_DTYPE)
    n_out = np.zeros(1, dtype=np.int64)
    rc = lib.oracle_topk_paths_masked(_ptr(G.offsets), _ptr(G.cols), _ptr(G.rels), G.n, _ptr(vt),
                                      _ptr(G.vemb), _ptr(G.remb), G.dtype, G.d, FN_CODES[fn], float(gamma),
                                      int(s), int(t), _ptr(m1), _ptr(m2), _ptr(m3), _ptr(tu), _ptr(tv),
                                      int(K), _ptr(out), _ptr(n_out))
    if rc == 1:
        raise ValueError("invalid query (s, t out of range, s == t, or K <= 0)")
    if rc:
        raise RuntimeError(f"oracle_topk_paths_masked: {rc}")
    return out[: int(n_out[0])].copy()


def topk_paths_batch(g, S, T, K: int, fn="transe", gamma=1.0):
    """All queries, OpenMP over queries.  Returns (paths [nq, K], n_out [nq])."""
    lib = _load()
    G = _G(g)
    S = np.ascontiguousarray(S, dtype=np.uint32)
    T = np.ascontiguousarray(T, dtype=np.uint32)
    nq = S.shape[0]
    out = np.zeros((nq, int(K)), dtype=PATH_DTYPE)
    n_out = np.zeros(nq, dtype=np.int64)
    status = np.zeros(nq, dtype=np.int32)
    rc = lib.oracle_topk_paths_batch(_ptr(G.offsets), _ptr(G.cols), _ptr(G.rels), G.n,
                                     _ptr(G.vemb), _ptr(G.remb), G.dtype, G.d, FN_CODES[fn],
                                     float(gamma), nq, _ptr(S), _ptr(T), int(K), _ptr(out),
                                     _ptr(n_out), _ptr(status))
    if rc:
        raise ValueError(f"oracle batch failed on queries {np.flatnonzero(status).tolist()[:8]}")
    return out, n_out


def tail_topk(g, H, Rq, K: int, cand_type: int = -1, fn="transe", gamma=1.0):
    """Tail prediction (Alg. 3 / Alg. 4) for the queries (H[i], Rq[i]): the K
    best candidates c (vtypes[c] == cand_type, or all vertices when
    cand_type < 0) by w(H[i], Rq[i], c).  Returns (out [nq, K] of TAIL_DTYPE,
    n_out [nq])."""
    lib = _load()
    G = _G(g)
    vt = np.ascontiguousarray(g.vtypes, dtype=np.uint8)
    H = np.ascontiguousarray(H, dtype=np.uint32)
    Rq = np.ascontiguousarray(Rq, dtype=np.uint32)
    nq = H.shape[0]
    out = np.zeros((nq, max(int(K), 1)), dtype=TAIL_DTYPE)
    n_out = np.zeros(nq, dtype=np.int64)
    status = np.zeros(nq, dtype=np.int32)
    rc = lib.oracle_tail_topk_batch(_ptr(vt), G.n, int(g.R), _ptr(G.vemb), _ptr(G.remb), G.dtype, G.d,
                                    FN_CODES[fn], float(gamma), nq, _ptr(H), _ptr(Rq), int(cand_type),
                                    int(K), _ptr(out), _ptr(n_out), _ptr(status))
    if rc == 1:
        raise ValueError("invalid tail query (head or relation out of range, or K <= 0)")
    if rc:
        raise RuntimeError(f"oracle_tail_topk_batch: {rc}")
    return out, n_out


def beam_paths(g, s: int, t: int, H: int, K: int, fn="transe", gamma=1.0, with_expanded=False):
    """Generic H-hop search with a per-path beam of width K (Alg. 6 / Alg. 7):
    the K best s->t paths of at most H hops the beam reaches, best first
    (structured array of BPATH_DTYPE: score, hops, v[0..hops], r[0..hops-1])."""
    assert BPATH_DTYPE.itemsize == 64
    lib = _load()
    G = _G(g)
    out = np.zeros(max(int(K), 1), dtype=BPATH_DTYPE)
    n_out = np.zeros(1, dtype=np.int64)
    expanded = np.zeros(1, dtype=np.int64)
    rc = lib.oracle_beam_paths(_ptr(G.offsets), _ptr(G.cols), _ptr(G.rels), G.n, _ptr(G.vemb),
                               _ptr(G.remb), G.dtype, G.d, FN_CODES[fn], float(gamma), int(s), int(t),
                               int(H), int(K), _ptr(out), _ptr(n_out), _ptr(expanded))
    if rc == 1:
        raise ValueError("invalid beam query (s, t out of range, s == t, K <= 0, H outside [1, 8], "
                         "or K^(H-1) above 1e6)")
    if rc:
        raise RuntimeError(f"oracle_beam_paths: {rc}")
    res = out[: int(n_out[0])].copy()
    return (res, int(expanded[0])) if with_expanded else res


def beam_paths_batch(g, S, T, H: int, K: int, fn="transe", gamma=1.0):
    """beam_paths for many queries, OpenMP over queries.  Returns
    (paths [nq, K] of BPATH_DTYPE, n_out [nq])."""
    lib = _load()
    G = _G(g)
    S = np.ascontiguousarray(S, dtype=np.uint32)
    T = np.ascontiguousarray(T, dtype=np.uint32)
    nq = S.shape[0]
    out = np.zeros((nq, max(int(K), 1)), dtype=BPATH_DTYPE)
    n_out = np.zeros(nq, dtype=np.int64)
    status = np.zeros(nq, dtype=np.int32)
    rc = lib.oracle_beam_paths_batch(_ptr(G.offsets), _ptr(G.cols), _ptr(G.rels), G.n, _ptr(G.vemb),
                                     _ptr(G.remb), G.dtype, G.d, FN_CODES[fn], float(gamma), nq, _ptr(S),
                                     _ptr(T), int(H), int(K), _ptr(out), _ptr(n_out), _ptr(status))
    if rc:
        raise ValueError(f"oracle beam batch failed on queries {np.flatnonzero(status).tolist()[:8]}")
    return out, n_out


def query_stats(g, s: int, t: int) -> dict:
    lib = _load()
    G = _G(g)
    st = np.zeros(1, dtype=STATS_DTYPE)
    rc = lib.oracle_query_stats(_ptr(G.offsets), _ptr(G.cols), G.n, int(s), int(t), _ptr(st))
    if rc:
        raise ValueError("invalid query")
    return {k: int(st[k][0]) for k in STATS_DTYPE.names}


def num_threads() -> int:
    return int(_load().oracle_num_threads())
