"""ctypes binding of libmhr.so: argument marshalling only.

Every entry point has the C name and forwards to the C ABI (include/mhr.h);
there is no Python or CPU fallback for any computation.  Arrays may be NumPy
arrays (host memory) or torch CUDA tensors (device memory); the memory kind is
passed to the library, which does the copies it needs.
"""

from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

MHR_OK, MHR_EINVAL, MHR_ENOMEM, MHR_ECUDA, MHR_ETIMEOUT, MHR_ERANGE = range(6)
MHR_SCORE_TRANSE_L1, MHR_SCORE_DISTMULT = 0, 1
MHR_F32, MHR_BF16 = 0, 1
MHR_MEM_HOST, MHR_MEM_DEVICE = 0, 1
MHR_K_MAX = 1024

STATUS_NAMES = {0: "MHR_OK", 1: "MHR_EINVAL", 2: "MHR_ENOMEM", 3: "MHR_ECUDA", 4: "MHR_ETIMEOUT",
                5: "MHR_ERANGE"}
SCORE_FNS = {"transe": MHR_SCORE_TRANSE_L1, "transe_l1": MHR_SCORE_TRANSE_L1,
             "distmult": MHR_SCORE_DISTMULT}

PATH_DTYPE = np.dtype([("score", "<f8"), ("u", "<u4"), ("v", "<u4"),
                       ("r1", "<u2"), ("r2", "<u2"), ("r3", "<u2"), ("pad", "<u2")])
assert PATH_DTYPE.itemsize == 24
TAIL_DTYPE = np.dtype([("score", "<f8"), ("v", "<u4"), ("pad", "<u4")])
assert TAIL_DTYPE.itemsize == 16
MHR_TAIL_K_MAX = 4096
BEAM_MAX_H = 8
BEAM_DTYPE = np.dtype([("score", "<f8"), ("hops", "<i4"), ("v", "<u4", (BEAM_MAX_H + 1,)),
                       ("r", "<u2", (BEAM_MAX_H,))])
assert BEAM_DTYPE.itemsize == 64


class MhrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class GraphDesc(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("n_edges", ctypes.c_int64),
                ("n_relations", ctypes.c_int32), ("n_vtypes", ctypes.c_int32),
                ("dim", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("offsets", ctypes.c_void_p), ("cols", ctypes.c_void_p), ("rels", ctypes.c_void_p),
                ("vtypes", ctypes.c_void_p), ("vertex_emb", ctypes.c_void_p),
                ("rel_emb", ctypes.c_void_p), ("emb_dtype", ctypes.c_int), ("mem", ctypes.c_int),
                ("score_fn", ctypes.c_int), ("reserved1", ctypes.c_int32),
                ("gamma", ctypes.c_double)]


class MLP(ctypes.Structure):
    _fields_ = [("W1", ctypes.c_void_p), ("b1", ctypes.c_void_p), ("w2", ctypes.c_void_p),
                ("b2", ctypes.c_void_p)]


class Constraints(ctypes.Structure):
    _fields_ = [("rel1", ctypes.c_void_p), ("rel2", ctypes.c_void_p), ("rel3", ctypes.c_void_p),
                ("types_u", ctypes.c_void_p), ("types_v", ctypes.c_void_p)]


class QueryOpts(ctypes.Structure):
    _fields_ = [("chunk", ctypes.c_int32), ("order", ctypes.c_int32), ("prune", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("mlp", ctypes.POINTER(MLP)),
                ("tile", ctypes.c_int32), ("part_count", ctypes.c_int32),
                ("constraints", ctypes.POINTER(Constraints)), ("part_index", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("edges_scanned", ctypes.c_int64), ("hits", ctypes.c_int64),
                ("paths", ctypes.c_int64), ("candidates", ctypes.c_int64), ("rescored", ctypes.c_int64),
                ("pruned_edges", ctypes.c_int64), ("dense_queries", ctypes.c_int64),
                ("ms", ctypes.c_double), ("ms_device", ctypes.c_double),
                ("ms_join", ctypes.c_double), ("ms_expand", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GraphInfo(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("n_edges", ctypes.c_int64),
                ("n_relations", ctypes.c_int32), ("dim", ctypes.c_int32),
                ("max_out_degree", ctypes.c_int64), ("max_in_degree", ctypes.c_int64),
                ("eps32_edge", ctypes.c_double), ("eps64_edge", ctypes.c_double),
                ("err_path", ctypes.c_double), ("epstc_edge", ctypes.c_double),
                ("err_path_tc", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ("mhr_graph_load", "mhr_graph_free", "mhr_graph_get_info", "mhr_edge_scores", "mhr_topk_paths",
           "mhr_topk_paths_batched", "mhr_topk_paths_noalloc", "mhr_training_labels",
           "mhr_mlp_features", "mhr_mlp_forward", "mhr_mlp_backward", "mhr_mlp_adam",
           "mhr_mlp_to_bf16", "mhr_tail_topk", "mhr_beam_paths", "mhr_merge_paths", "mhr_last_error",
           "mhr_version")

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libmhr.so (building it with nvcc when missing); raises if neither works."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            path = _build.build()
        if not os.path.exists(path):
            raise ImportError(f"libmhr.so not found at {path}; run paper_2406_07727_gb300/build.py")
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        lib.mhr_graph_load.restype = ctypes.c_int
        lib.mhr_graph_load.argtypes = [ctypes.POINTER(GraphDesc), ctypes.POINTER(P), P]
        lib.mhr_graph_free.restype = ctypes.c_int
        lib.mhr_graph_free.argtypes = [P]
        lib.mhr_graph_get_info.restype = ctypes.c_int
        lib.mhr_graph_get_info.argtypes = [P, ctypes.POINTER(GraphInfo)]
        lib.mhr_edge_scores.restype = ctypes.c_int
        lib.mhr_edge_scores.argtypes = [P, P, P, P, i64, i32, P, ctypes.c_int, P]
        lib.mhr_topk_paths.restype = ctypes.c_int
        lib.mhr_topk_paths.argtypes = [P, ctypes.c_uint32, ctypes.c_uint32, i32, P, P,
                                       ctypes.POINTER(QueryOpts), ctypes.POINTER(Stats)]
        lib.mhr_topk_paths_batched.restype = ctypes.c_int
        lib.mhr_topk_paths_batched.argtypes = [P, i32, P, P, i32, P, P, ctypes.c_int,
                                               ctypes.POINTER(QueryOpts), ctypes.POINTER(Stats), P]
        lib.mhr_autotune.restype = ctypes.c_int
        lib.mhr_autotune.argtypes = [P, i32, P, P, i32, ctypes.c_int, ctypes.POINTER(QueryOpts), P, i32, P, i32,
                                     i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32), P, P]
        lib.mhr_training_labels.restype = ctypes.c_int
        lib.mhr_training_labels.argtypes = [P, i32, P, P, i64, P, P, P, P, ctypes.POINTER(i64), P]
        lib.mhr_mlp_features.restype = ctypes.c_int
        lib.mhr_mlp_features.argtypes = [P, P, P, i64, P, P]
        lib.mhr_mlp_forward.restype = ctypes.c_int
        lib.mhr_mlp_forward.argtypes = [ctypes.POINTER(MLP), P, i64, P, P, P]
        lib.mhr_mlp_backward.restype = ctypes.c_int
        lib.mhr_mlp_backward.argtypes = [ctypes.POINTER(MLP), P, i64, P, P, P, P, P, P, P]
        lib.mhr_mlp_adam.restype = ctypes.c_int
        lib.mhr_mlp_adam.argtypes = [P, P, P, P, i64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float, i32, P]
        lib.mhr_mlp_to_bf16.restype = ctypes.c_int
        lib.mhr_mlp_to_bf16.argtypes = [P, P, i64, P]
        lib.mhr_topk_paths_noalloc.restype = ctypes.c_int
        lib.mhr_topk_paths_noalloc.argtypes = [P, ctypes.c_uint32, ctypes.c_uint32, i32, P, P, P]
        lib.mhr_tail_topk.restype = ctypes.c_int
        lib.mhr_tail_topk.argtypes = [P, i32, P, P, i32, i32, P, P, ctypes.c_int, ctypes.POINTER(Stats), P]
        lib.mhr_beam_paths.restype = ctypes.c_int
        lib.mhr_beam_paths.argtypes = [P, i32, P, P, i32, i32, P, P, ctypes.c_int, ctypes.POINTER(Stats), P]
        lib.mhr_merge_paths.restype = ctypes.c_int
        lib.mhr_merge_paths.argtypes = [i32, i32, i32, P, P, P, P, ctypes.c_int, P]
        lib.mhr_last_error.restype = ctypes.c_char_p
        lib.mhr_last_error.argtypes = []
        lib.mhr_version.restype = ctypes.c_char_p
        lib.mhr_version.argtypes = []
        _lib = lib
        return lib


def mhr_last_error() -> str:
    return load_library().mhr_last_error().decode()


def mhr_version() -> str:
    return load_library().mhr_version().decode()


def _check(rc: int):
    if rc != MHR_OK:
        raise MhrError(rc, mhr_last_error())


# --------------------------------------------------------------------------- marshalling
def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def _mem_of(*arrays) -> int:
    kinds = {MHR_MEM_DEVICE if _is_torch_cuda(a) else MHR_MEM_HOST for a in arrays if a is not None}
    if len(kinds) > 1:
        raise ValueError("mixing host and device arrays in one call")
    return kinds.pop() if kinds else MHR_MEM_HOST


def _ptr(a):
    if a is None:
        return None
    if _is_torch_cuda(a):
        if not a.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("host arrays must be C-contiguous numpy arrays")
    return ctypes.c_void_p(a.ctypes.data)


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _opts(opts, n_relations: int = 0) -> Optional[QueryOpts]:
    if opts is None:
        return None
    if isinstance(opts, QueryOpts):
        return opts
    o = QueryOpts()
    known = {name for name, _ in QueryOpts._fields_} - {"reserved"}
    for k, v in dict(opts).items():
        if k not in known:
            raise ValueError(f"unknown query option {k!r} (known: {', '.join(sorted(known))})")
        if k == "mlp":
            o._mlp_keep = v if isinstance(v, MLP) else v.struct()
            o.mlp = ctypes.pointer(o._mlp_keep)
        elif k == "constraints":
            if v is not None:
                o._cons_keep = _constraints(v, n_relations)
                o.constraints = ctypes.pointer(o._cons_keep)
        else:
            setattr(o, k, int(v))
    return o


def _constraints(c, n_relations: int) -> Constraints:
    """{"rel1", "rel2", "rel3": allowed relation ids per hop, "types_u",
    "types_v": allowed vertex types of u and v} -> mhr_constraints; a missing
    or None entry allows every id.  Relation flags have the graph's
    n_relations entries (the library reads that many)."""
    if isinstance(c, Constraints):
        return c
    c = dict(c)
    unknown = set(c) - {"rel1", "rel2", "rel3", "types_u", "types_v"}
    if unknown:
        raise ValueError(f"unknown constraint {sorted(unknown)[0]!r} (known: rel1, rel2, rel3, types_u, types_v)")
    n_rel = int(n_relations)
    out = Constraints()
    keep = []
    for name in ("rel1", "rel2", "rel3"):
        ids = c.get(name)
        if ids is None:
            continue
        ids = np.asarray(list(ids), dtype=np.int64)
        if ids.size and (ids.min() < 0 or ids.max() >= n_rel):
            raise ValueError(f"{name}: relation id outside [0, {n_rel})")
        f = np.zeros(max(n_rel, 1), dtype=np.uint8)
        f[ids] = 1
        keep.append(f)
        setattr(out, name, f.ctypes.data)
    for name in ("types_u", "types_v"):
        ids = c.get(name)
        if ids is None:
            continue
        ids = np.asarray(list(ids), dtype=np.int64)
        if ids.size and (ids.min() < 0 or ids.max() > 255):
            raise ValueError(f"{name}: vertex type outside [0, 255]")
        f = np.zeros(256, dtype=np.uint8)
        f[ids] = 1
        keep.append(f)
        setattr(out, name, f.ctypes.data)
    out._keep = keep
    return out


# --------------------------------------------------------------------------- API
class Graph:
    """Owns one mhr_graph handle (freed by close() or garbage collection)."""

    def __init__(self, handle: int, n: int, E: int, R: int, d: int, score_fn: int):
        self._h = handle
        self.n, self.E, self.R, self.d = n, E, R, d
        self.score_fn = score_fn

    @property
    def handle(self):
        if not self._h:
            raise ValueError("graph is closed")
        return ctypes.c_void_p(self._h)

    def close(self):
        if self._h:
            load_library().mhr_graph_free(ctypes.c_void_p(self._h))
            self._h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mhr_graph_load(offsets, cols, rels, vertex_emb, rel_emb, n_relations: int, *, vtypes=None,
                   n_vtypes: int = 1, score_fn="transe", gamma: float = 1.0, emb_dtype="f32",
                   stream=None) -> Graph:
    """Upload a graph (numpy host arrays or torch CUDA tensors)."""
    lib = load_library()
    mem = _mem_of(offsets, cols, rels, vertex_emb, rel_emb, vtypes)
    if mem == MHR_MEM_HOST:
        offsets = _host(offsets, np.int64)
        cols = _host(cols, np.uint32)
        rels = _host(rels, np.uint16)
        dt = np.float32 if emb_dtype == "f32" else np.uint16
        vertex_emb = _host(vertex_emb, dt)
        rel_emb = _host(rel_emb, dt)
        if vtypes is not None:
            vtypes = _host(vtypes, np.uint8)
    n = int(offsets.shape[0]) - 1
    E = int(cols.shape[0])
    d = int(vertex_emb.shape[1])
    desc = GraphDesc()
    desc.n_vertices, desc.n_edges = n, E
    desc.n_relations, desc.n_vtypes, desc.dim = int(n_relations), int(n_vtypes), d
    desc.offsets, desc.cols, desc.rels = _ptr(offsets), _ptr(cols), _ptr(rels)
    desc.vtypes = _ptr(vtypes)
    desc.vertex_emb, desc.rel_emb = _ptr(vertex_emb), _ptr(rel_emb)
    desc.emb_dtype = MHR_F32 if emb_dtype == "f32" else MHR_BF16
    desc.mem = mem
    desc.score_fn = SCORE_FNS[score_fn] if isinstance(score_fn, str) else int(score_fn)
    desc.gamma = float(gamma)
    h = ctypes.c_void_p()
    _check(lib.mhr_graph_load(ctypes.byref(desc), ctypes.byref(h), _stream_ptr(stream)))
    return Graph(h.value, n, E, int(n_relations), d, desc.score_fn)


def mhr_graph_free(g: Graph):
    g.close()


def mhr_graph_get_info(g: Graph) -> dict:
    """Sizes and proven fp32 screening error bounds of a loaded graph."""
    info = GraphInfo()
    _check(load_library().mhr_graph_get_info(g.handle, ctypes.byref(info)))
    return info.as_dict()


def mhr_edge_scores(g: Graph, src=None, rel=None, dst=None, precision: int = 0, out=None,
                    stream=None):
    """Edge weights; precision 0 -> float32 (fp32 arithmetic), 2 -> float64
    (canonical fp64 order).  src is None: all edges in CSR order."""
    lib = load_library()
    mem = _mem_of(src, rel, dst, out)
    n = g.E if src is None else int(src.shape[0])
    if mem == MHR_MEM_HOST:
        if src is not None:
            src, rel, dst = _host(src, np.uint32), _host(rel, np.uint16), _host(dst, np.uint32)
        if out is None:
            out = np.empty(n, dtype=np.float32 if precision == 0 else np.float64)
    elif out is None:
        import torch
        out = torch.empty(n, dtype=torch.float32 if precision == 0 else torch.float64,
                          device=src.device)
    _check(lib.mhr_edge_scores(g.handle, _ptr(src), _ptr(rel), _ptr(dst), n, int(precision),
                               _ptr(out), mem, _stream_ptr(stream)))
    return out


def mhr_topk_paths(g: Graph, s: int, t: int, K: int, opts=None, with_stats: bool = False):
    """One query, synchronous; returns a structured array of PATH_DTYPE."""
    lib = load_library()
    out = np.zeros(max(int(K), 1), dtype=PATH_DTYPE)
    n_out = ctypes.c_int32(0)
    st = Stats()
    o = _opts(opts, g.R)
    rc = lib.mhr_topk_paths(g.handle, ctypes.c_uint32(int(s) & 0xFFFFFFFF),
                            ctypes.c_uint32(int(t) & 0xFFFFFFFF), int(K), _ptr(out),
                            ctypes.byref(n_out), ctypes.byref(o) if o is not None else None,
                            ctypes.byref(st))
    _check(rc)
    res = out[: n_out.value].copy()
    return (res, st.as_dict()) if with_stats else res


def mhr_topk_paths_batched(g: Graph, S, T, K: int, out=None, n_out=None, opts=None, stream=None,
                           with_stats: bool = False):
    """nq queries.  Host arrays in -> host arrays out (synchronous); device
    tensors in -> device tensors out (asynchronous on `stream`).  Returns
    (paths [nq, K] of PATH_DTYPE or a uint8 tensor [nq, K*24], n_out [nq])."""
    lib = load_library()
    mem = _mem_of(S, T, out, n_out)
    nq = int(S.shape[0])
    if mem == MHR_MEM_HOST:
        S, T = _host(S, np.uint32), _host(T, np.uint32)
        if out is None:
            out = np.zeros((nq, int(K)), dtype=PATH_DTYPE)
        if n_out is None:
            n_out = np.zeros(nq, dtype=np.int32)
    else:
        import torch
        if out is None:
            out = torch.empty((nq, int(K) * PATH_DTYPE.itemsize), dtype=torch.uint8, device=S.device)
        if n_out is None:
            n_out = torch.empty(nq, dtype=torch.int32, device=S.device)
    st = Stats()
    o = _opts(opts, g.R)
    rc = lib.mhr_topk_paths_batched(g.handle, nq, _ptr(S), _ptr(T), int(K), _ptr(out), _ptr(n_out),
                                    mem, ctypes.byref(o) if o is not None else None,
                                    ctypes.byref(st) if with_stats else None, _stream_ptr(stream))
    _check(rc)
    if with_stats:
        return out, n_out, st.as_dict()
    return out, n_out


def mhr_merge_paths(parts, n_parts_out, K: int, out=None, n_out=None, stream=None):
    """Tree merge (Alg. 2) of the partial top-K lists of disjoint path sets:
    parts [n_parts, nq, K] of PATH_DTYPE (or a uint8 device tensor
    [n_parts, nq, K*24]) with counts n_parts_out [n_parts, nq]; returns the
    first K of every query's merged order and the counts.  Host arrays in ->
    host arrays out (synchronous); device tensors in -> device tensors out."""
    lib = load_library()
    mem = _mem_of(parts, n_parts_out, out, n_out)
    n_parts, nq = int(n_parts_out.shape[0]), int(n_parts_out.shape[1])
    if mem == MHR_MEM_HOST:
        parts = np.ascontiguousarray(parts, dtype=PATH_DTYPE)
        n_parts_out = _host(n_parts_out, np.int32)
        if out is None:
            out = np.zeros((nq, int(K)), dtype=PATH_DTYPE)
        if n_out is None:
            n_out = np.zeros(nq, dtype=np.int32)
    else:
        import torch
        if out is None:
            out = torch.empty((nq, int(K) * PATH_DTYPE.itemsize), dtype=torch.uint8, device=parts.device)
        if n_out is None:
            n_out = torch.empty(nq, dtype=torch.int32, device=parts.device)
    _check(lib.mhr_merge_paths(nq, int(K), n_parts, _ptr(parts), _ptr(n_parts_out), _ptr(out), _ptr(n_out), mem,
                               _stream_ptr(stream)))
    return out, n_out


def mhr_autotune(g: Graph, S, T, K: int, opts=None, chunks=(8192, 16384, 32768), tiles=(4, 8),
                 reps: int = 3, stream=None):
    """Time the batched search on (S, T) for every (screen, work-item size,
    scan tile) combination (both screens when opts["precision"] < 0); returns
    (best chunk, best tile, best precision, {(precision, chunk, tile): ms})."""
    lib = load_library()
    mem = _mem_of(S, T)
    if mem == MHR_MEM_HOST:
        S, T = _host(S, np.uint32), _host(T, np.uint32)
    ch = np.ascontiguousarray(chunks, dtype=np.int32)
    tl = np.ascontiguousarray(tiles, dtype=np.int32)
    ms = np.zeros(2 * len(ch) * len(tl), dtype=np.float32)
    bc, bt, bp = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    o = _opts(opts, g.R)
    _check(lib.mhr_autotune(g.handle, int(S.shape[0]), _ptr(S), _ptr(T), int(K), mem,
                            ctypes.byref(o) if o is not None else None, _ptr(ch), len(ch), _ptr(tl), len(tl),
                            int(reps), ctypes.byref(bc), ctypes.byref(bt), ctypes.byref(bp), _ptr(ms),
                            _stream_ptr(stream)))
    req = o.precision if o is not None else 0
    precs = ([0, 1] if (g.score_fn == MHR_SCORE_DISTMULT and g.R <= 16) else [0]) if req < 0 else [req]
    table = {}
    for p_i, pr in enumerate(precs):
        for i, c in enumerate(ch):
            for j, t in enumerate(tl):
                table[(pr, int(c), int(t))] = float(ms[(p_i * len(ch) + i) * len(tl) + j])
    return int(bc.value), int(bt.value), int(bp.value), table


def mhr_topk_paths_noalloc(g: Graph, s: int, t: int, K: int, out, n_out, stream=None):
    """One query into caller-owned device buffers (out: uint8 tensor of K*24
    bytes, n_out: int32 tensor of 1), allocating nothing; asynchronous."""
    lib = load_library()
    if not (_is_torch_cuda(out) and _is_torch_cuda(n_out)):
        raise ValueError("out and n_out must be device tensors")
    _check(lib.mhr_topk_paths_noalloc(g.handle, ctypes.c_uint32(int(s)), ctypes.c_uint32(int(t)), int(K),
                                      _ptr(out), _ptr(n_out), _stream_ptr(stream)))


def mhr_tail_topk(g: Graph, H, Rq, K: int, cand_type: int = -1, out=None, n_out=None, stream=None,
                  with_stats: bool = False):
    """Tail prediction (Alg. 3 / Alg. 4): for each query (H[i], Rq[i]) the K
    best candidate vertices (vtypes == cand_type, or all when cand_type is -1)
    by the edge weight w(H[i], Rq[i], c).  Host arrays in -> host arrays out
    (out [nq, K] of TAIL_DTYPE); device tensors in -> device tensors out (a
    uint8 tensor [nq, K*16]).  Synchronous."""
    lib = load_library()
    mem = _mem_of(H, Rq, out, n_out)
    nq = int(H.shape[0])
    if mem == MHR_MEM_HOST:
        H, Rq = _host(H, np.uint32), _host(Rq, np.uint16)
        if out is None:
            out = np.zeros((nq, max(int(K), 1)), dtype=TAIL_DTYPE)
        if n_out is None:
            n_out = np.zeros(nq, dtype=np.int32)
    else:
        import torch
        if out is None:
            out = torch.empty((nq, max(int(K), 1) * TAIL_DTYPE.itemsize), dtype=torch.uint8, device=H.device)
        if n_out is None:
            n_out = torch.empty(nq, dtype=torch.int32, device=H.device)
    st = Stats()
    _check(lib.mhr_tail_topk(g.handle, nq, _ptr(H), _ptr(Rq), int(cand_type), int(K), _ptr(out), _ptr(n_out),
                             mem, ctypes.byref(st) if with_stats else None, _stream_ptr(stream)))
    if with_stats:
        return out, n_out, st.as_dict()
    return out, n_out


def mhr_beam_paths(g: Graph, S, T, H: int, K: int, out=None, n_out=None, stream=None, with_stats: bool = False):
    """Generic H-hop search with a per-path beam of width K (Alg. 6 / Alg. 7):
    the K best s->t paths of at most H hops the beam reaches, per query.  Host
    arrays in -> host arrays out (out [nq, K] of BEAM_DTYPE, n_out [nq]);
    device tensors in -> device tensors out (a uint8 tensor [nq, K*64] and an
    int32 tensor [nq]).  Synchronous."""
    lib = load_library()
    mem = _mem_of(S, T, out, n_out)
    nq = int(S.shape[0])
    if mem == MHR_MEM_HOST:
        S, T = _host(S, np.uint32), _host(T, np.uint32)
        if out is None:
            out = np.zeros((nq, max(int(K), 1)), dtype=BEAM_DTYPE)
        if n_out is None:
            n_out = np.zeros(nq, dtype=np.int32)
    else:
        import torch
        if out is None:
            out = torch.empty((nq, max(int(K), 1) * BEAM_DTYPE.itemsize), dtype=torch.uint8, device=S.device)
        if n_out is None:
            n_out = torch.empty(nq, dtype=torch.int32, device=S.device)
    st = Stats()
    _check(lib.mhr_beam_paths(g.handle, nq, _ptr(S), _ptr(T), int(H), int(K), _ptr(out), _ptr(n_out),
                              mem, ctypes.byref(st) if with_stats else None, _stream_ptr(stream)))
    return (out, n_out, st.as_dict()) if with_stats else (out, n_out)


def beams_from_device(buf, K: int) -> np.ndarray:
    """uint8 device/host buffer [nq, K*64] -> structured numpy array [nq, K]."""
    if hasattr(buf, "cpu"):
        buf = buf.cpu().numpy()
    buf = np.ascontiguousarray(buf)
    return buf.view(BEAM_DTYPE).reshape(buf.shape[0], K)


def tails_from_device(buf, K: int) -> np.ndarray:
    """uint8 device/host buffer [nq, K*16] -> structured numpy array [nq, K]."""
    if hasattr(buf, "cpu"):
        buf = buf.cpu().numpy()
    buf = np.ascontiguousarray(buf)
    return buf.view(TAIL_DTYPE).reshape(buf.shape[0], K)


# --------------------------------------------------------------------------- learned ordering
def mhr_training_labels(g: Graph, S, T, cap: int, stream=None):
    """Plain search on (S, T) (host arrays); returns device tensors
    (near_v, end_v, own, best) of the rows written."""
    import torch
    lib = load_library()
    S, T = _host(S, np.uint32), _host(T, np.uint32)
    dev = torch.device("cuda")
    near_v = torch.empty(cap, dtype=torch.int32, device=dev)
    end_v = torch.empty(cap, dtype=torch.int32, device=dev)
    own = torch.empty(cap, dtype=torch.float32, device=dev)
    best = torch.empty(cap, dtype=torch.float32, device=dev)
    n = ctypes.c_int64(0)
    _check(lib.mhr_training_labels(g.handle, len(S), _ptr(S), _ptr(T), int(cap), _ptr(near_v), _ptr(end_v),
                                   _ptr(own), _ptr(best), ctypes.byref(n), _stream_ptr(stream)))
    k = n.value
    return near_v[:k], end_v[:k], own[:k], best[:k]


def mhr_mlp_features(g: Graph, va, vb, X=None, stream=None):
    import torch
    n = int(va.shape[0])
    if X is None:
        X = torch.empty((n, 256), dtype=torch.int16, device=va.device)
    _check(load_library().mhr_mlp_features(g.handle, _ptr(va), _ptr(vb), n, _ptr(X), _stream_ptr(stream)))
    return X


def mhr_mlp_forward(m, X, y=None, z1=None, stream=None):
    import torch
    n = int(X.shape[0])
    if y is None:
        y = torch.empty(n, dtype=torch.float32, device=X.device)
    st = m if isinstance(m, MLP) else m.struct()
    _check(load_library().mhr_mlp_forward(ctypes.byref(st), _ptr(X), n, _ptr(y), _ptr(z1), _stream_ptr(stream)))
    return y


def mhr_mlp_backward(m, X, target, y, z1, work, grads, loss=None, stream=None):
    st = m if isinstance(m, MLP) else m.struct()
    _check(load_library().mhr_mlp_backward(ctypes.byref(st), _ptr(X), int(X.shape[0]), _ptr(target), _ptr(y),
                                           _ptr(z1), _ptr(work), _ptr(grads), _ptr(loss), _stream_ptr(stream)))


def mhr_mlp_adam(params, grads, m1, m2, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(load_library().mhr_mlp_adam(_ptr(params), _ptr(grads), _ptr(m1), _ptr(m2), int(params.numel()),
                                       float(lr), float(beta1), float(beta2), float(eps), int(step),
                                       _stream_ptr(stream)))


def mhr_mlp_to_bf16(src, dst, stream=None):
    _check(load_library().mhr_mlp_to_bf16(_ptr(src), _ptr(dst), int(src.numel()), _stream_ptr(stream)))


def paths_from_device(buf, K: int) -> np.ndarray:
    """uint8 device/host buffer [nq, K*24] -> structured numpy array [nq, K]."""
    if hasattr(buf, "cpu"):
        buf = buf.cpu().numpy()
    buf = np.ascontiguousarray(buf)
    return buf.view(PATH_DTYPE).reshape(buf.shape[0], K)


def load_kg(kg, score_fn="transe", gamma=1.0, device: bool = False, stream=None) -> Graph:
    """Convenience: upload a synth.KG-like object (fields offsets, cols, rels,
    vtypes, vemb, remb, dtype, R, n_types)."""
    arrays = [kg.offsets, kg.cols, kg.rels, kg.vemb, kg.remb, kg.vtypes]
    if device:
        import torch
        arrays = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]
    off, cols, rels, vemb, remb, vt = arrays
    return mhr_graph_load(off, cols, rels, vemb, remb, kg.R, vtypes=vt, n_vtypes=kg.n_types,
                          score_fn=score_fn, gamma=gamma, emb_dtype=kg.dtype, stream=stream)
