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
