"""mhr_topk_paths_noalloc: the entry point for callers that cannot allocate
device memory (fixed memory footprint, a host allocator that owns the device
memory, or no room for the synchronisation of cudaMalloc/cudaFree).  Its
output must equal the batched entry point's, call after call, since every
call reuses the same fixed scratch array.  This file sorts last so that a run
stopping at the first failure has run every other test first."""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5


def _noalloc(mhr, G, s, t, K, out, n, stream):
    """One call through the C ABI into caller-owned device buffers."""
    import torch
    lib = mhr.load_library()
    out.fill_(0xAB)
    n.fill_(-7)
    rc = lib.mhr_topk_paths_noalloc(G.handle, ctypes.c_uint32(int(s)), ctypes.c_uint32(int(t)), K,
                                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(n.data_ptr()),
                                    ctypes.c_void_p(stream.cuda_stream))
    assert rc == mhr.MHR_OK, mhr.mhr_last_error()
    torch.cuda.synchronize()
    got_n = int(n.item())
    return out.cpu().numpy().view(mhr.PATH_DTYPE)[:got_n].copy()


def _same(got, exp, ctx):
    """Path count, ids, order and fp64 scores bit-identical."""
    assert len(got) == len(exp), (ctx, len(got), len(exp))
    for f in ("u", "r1", "v", "r2", "r3"):
        assert np.array_equal(got[f], exp[f]), (ctx, f)
    assert got["score"].tobytes() == exp["score"].tobytes(), (ctx, "score")


def _graph():
    import synth
    g = synth.gen_rmat_kg(12, 3000, 40_000, 6, 3, seed=21)
    g.vemb, g.remb = synth.gen_embeddings(g.n, g.R, 64, 1 / 8, seed=21)
    S, T = synth.queries_edge_biased(g, 6, seed=21)
    return g, S, T


def test_noalloc_matches_batched_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    import paper_2406_07727_gb300 as mhr
    lib = mhr.load_library()
    g, S, T = _graph()
    K = 40
    for fn in ("transe", "distmult"):
        G = mhr.load_kg(g, score_fn=fn)
        want, n_want = mhr.mhr_topk_paths_batched(G, S, T, K)
        out = torch.empty(K * 24, dtype=torch.uint8, device="cuda")
        n = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream()
        for q in range(len(S)):
            for call in range(2):  # two calls in a row share the scratch array
                out.fill_(0xAB)
                rc = lib.mhr_topk_paths_noalloc(G.handle, ctypes.c_uint32(int(S[q])), ctypes.c_uint32(int(T[q])),
                                                K, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(n.data_ptr()),
                                                ctypes.c_void_p(stream.cuda_stream))
                assert rc == mhr.MHR_OK, mhr.mhr_last_error()
                torch.cuda.synchronize()
                got_n = int(n.item())
                got = out.cpu().numpy().view(mhr.PATH_DTYPE)[:got_n]
                exp = want[q][: n_want[q]]
                assert got_n == int(n_want[q]), (fn, q, call)
                for f in ("u", "r1", "v", "r2", "r3"):
                    assert np.array_equal(got[f], exp[f]), (fn, q, call, f)
                assert np.all(np.abs(got["score"] - exp["score"]) <= REL_TOL * np.maximum(1.0, np.abs(exp["score"])))
        G.close()


def test_noalloc_matches_oracle_bit_exact():
    """Against the CPU oracle directly: ids, order and fp64 scores identical,
    for K = 1, 40 and 1024, both score forms."""
    torch = pytest.importorskip("torch")
    import oracle
    import paper_2406_07727_gb300 as mhr
    g, S, T = _graph()
    stream = torch.cuda.current_stream()
    out = torch.empty(1024 * 24, dtype=torch.uint8, device="cuda")
    n = torch.empty(1, dtype=torch.int32, device="cuda")
    for fn in ("transe", "distmult"):
        G = mhr.load_kg(g, score_fn=fn)
        for K in (1, 40, 1024):
            want, n_want = oracle.topk_paths_batch(g, S, T, K, fn=fn)
            for q in range(len(S)):
                got = _noalloc(mhr, G, S[q], T[q], K, out, n, stream)
                _same(got, want[q][: n_want[q]], (fn, K, q))
        G.close()


@pytest.mark.parametrize("kind", ["zero", "dyadic"])
def test_noalloc_tie_heavy(kind):
    """Scores that tie in bulk (zero embeddings: every path scores gamma*3 or 0;
    dyadic values: many exact ties): the order among equal scores is decided
    only by the (u, r1, v, r2, r3) ids in the staging flushes.  K up to
    MHR_K_MAX; oracle and batched entry point agree with it byte for byte."""
    torch = pytest.importorskip("torch")
    import oracle
    import paper_2406_07727_gb300 as mhr
    from tests._graphs import random_kg
    rng = np.random.default_rng(77 if kind == "zero" else 78)
    g = random_kg(rng, 80, 5000, 4, 8, zero=(kind == "zero"), dyadic=(kind == "dyadic"))
    S = np.array([3, 10, 41], dtype=np.uint32)
    T = np.array([7, 55, 2], dtype=np.uint32)
    stream = torch.cuda.current_stream()
    out = torch.empty(1024 * 24, dtype=torch.uint8, device="cuda")
    n = torch.empty(1, dtype=torch.int32, device="cuda")
    for s, t in zip(S.tolist(), T.tolist()):
        # more paths than MHR_K_MAX: the staging buffer fills and flushes several times
        assert oracle.topk_paths(g, s, t, 1, with_counts=True)[2] > 1500
    for fn in ("transe", "distmult"):
        G = mhr.load_kg(g, score_fn=fn)
        for K in (100, 1024):
            want, n_want = oracle.topk_paths_batch(g, S, T, K, fn=fn)
            bat, n_bat = mhr.mhr_topk_paths_batched(G, S, T, K)
            for q in range(len(S)):
                assert n_want[q] == K
                got = _noalloc(mhr, G, S[q], T[q], K, out, n, stream)
                _same(got, want[q][: n_want[q]], (kind, fn, K, q))
                assert got.tobytes() == bat[q][: n_bat[q]].tobytes()
        G.close()


def test_noalloc_accepts_frontier_at_its_limit():
    """An out-degree of s of exactly 65,536 fills the hop-1 scratch and is
    accepted; the result equals the oracle's."""
    torch = pytest.importorskip("torch")
    import oracle
    import paper_2406_07727_gb300 as mhr
    import synth
    M = 65536
    n = M + 40
    rng = np.random.default_rng(5)
    # s = 0 -> vertices 2 .. M+1; every 64th of them -> one of 30 middle vertices -> t = 1
    src = [np.zeros(M, dtype=np.int64)]
    dst = [np.arange(2, M + 2, dtype=np.int64)]
    hop1 = np.arange(2, M + 2, 64, dtype=np.int64)
    mids = rng.integers(M + 2, n, size=hop1.size)
    src.append(hop1)
    dst.append(mids)
    src.append(np.arange(M + 2, n, dtype=np.int64))
    dst.append(np.ones(n - M - 2, dtype=np.int64))
    src, dst = np.concatenate(src), np.concatenate(dst)
    rel = rng.integers(0, 3, size=src.size)
    off, cols, rels = synth.canonicalize(n, 3, src, rel, dst)
    assert off[1] - off[0] == M
    vemb = (rng.standard_normal((n, 16)) * 0.3).astype(np.float32)
    remb = (rng.standard_normal((3, 16)) * 0.3).astype(np.float32)
    g = synth.KG(n=n, R=3, n_types=1, offsets=off, cols=cols, rels=rels, vtypes=np.zeros(n, np.uint8),
                 vemb=vemb, remb=remb)
    G = mhr.load_kg(g)
    stream = torch.cuda.current_stream()
    out = torch.empty(64 * 24, dtype=torch.uint8, device="cuda")
    nn = torch.empty(1, dtype=torch.int32, device="cuda")
    want = oracle.topk_paths(g, 0, 1, 64)
    for call in range(2):
        got = _noalloc(mhr, G, 0, 1, 64, out, nn, stream)
        _same(got, want, ("limit", call))
    G.close()


def test_noalloc_rejects_frontiers_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    import paper_2406_07727_gb300 as mhr
    import synth
    n = 70_002
    src = np.zeros(n - 2, dtype=np.int64)
    dst = np.arange(2, n, dtype=np.int64)          # vertex 0 -> 70,000 vertices
    src = np.concatenate([src, dst[:5]])
    dst = np.concatenate([dst, np.ones(5, dtype=np.int64)])
    off, cols, rels = synth.canonicalize(n, 1, src, np.zeros_like(src), dst)
    vemb = np.zeros((n, 4), dtype=np.float32)
    remb = np.zeros((1, 4), dtype=np.float32)
    G = mhr.mhr_graph_load(off, cols, rels, vemb, remb, 1)
    out = torch.empty(10 * 24, dtype=torch.uint8, device="cuda")
    nn = torch.empty(1, dtype=torch.int32, device="cuda")
    with pytest.raises(mhr.MhrError) as e:
        mhr.mhr_topk_paths_noalloc(G, 0, 1, 10, out, nn)
    assert e.value.status == mhr.MHR_ERANGE and "65536" in str(e.value)
    G.close()
