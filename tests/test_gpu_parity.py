"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Bar: path ids and order bit-exact; scores bit-exact (the fp64 rescoring
repeats the oracle's operation order), and in any case within 1e-5 relative.
Edge scores: fp64 precision bit-exact; fp32 precision within the proven bound.
"""

import math

import numpy as np
import pytest

import oracle
import synth
from tests._graphs import kg_from_golden, load_golden, path_tuples, random_kg

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5


@pytest.fixture(scope="module")
def mhr():
    import paper_2406_07727_gb300 as m
    return m


def compare_query(got, n_got, want, ctx=""):
    assert n_got == len(want), (ctx, n_got, len(want))
    g = path_tuples(got[:n_got])
    w = path_tuples(want)
    ids_g = [p[1:] for p in g]
    ids_w = [p[1:] for p in w]
    assert ids_g == ids_w, (ctx, next(i for i in range(len(ids_g)) if ids_g[i] != ids_w[i]))
    for a, b in zip(g, w):
        assert abs(a[0] - b[0]) <= REL_TOL * max(1.0, abs(b[0])), (ctx, a, b)
    assert [p[0] for p in g] == [p[0] for p in w], (ctx, "scores not bit-identical")


def run_and_compare(m, g, S, T, K, fn, opts=None, check=True):
    G = m.load_kg(g, score_fn=fn)
    try:
        out, n_out = m.mhr_topk_paths_batched(G, S, T, K, opts=opts)
        valid = (S != T) & (S < g.n) & (T < g.n)
        assert (n_out[~valid] == -1).all()
        if not check:
            return out, n_out
        vi = np.flatnonzero(valid)
        want, n_want = oracle.topk_paths_batch(g, S[vi], T[vi], K, fn=fn)
        for i, q in enumerate(vi):
            compare_query(out[q], int(n_out[q]), want[i, : n_want[i]], ctx=(int(q), int(S[q]), int(T[q])))
        return out, n_out
    finally:
        G.close()


# --------------------------------------------------------------------------- edge scores
@pytest.mark.parametrize("fn", ["transe", "distmult"])
def test_edge_scores_golden(mhr, fn):
    gj = load_golden()
    g = kg_from_golden(gj)
    G = mhr.load_kg(g, score_fn=fn)
    rows = gj[f"edge_weights_{fn}"]["rows"]
    src = np.array([r[0] for r in rows], dtype=np.uint32)
    rel = np.array([r[1] for r in rows], dtype=np.uint16)
    dst = np.array([r[2] for r in rows], dtype=np.uint32)
    want = [r[3] for r in rows]
    assert mhr.mhr_edge_scores(G, src, rel, dst, precision=2).tolist() == want
    assert mhr.mhr_edge_scores(G, src, rel, dst, precision=0).astype(np.float64).tolist() == want
    G.close()


@pytest.mark.parametrize("fn", ["transe", "distmult"])
@pytest.mark.parametrize("dtype,d", [("f32", 5), ("f32", 128), ("bf16", 64), ("bf16", 7), ("f32", 256)])
def test_edge_scores_random(mhr, fn, dtype, d):
    rng = np.random.default_rng(d)
    g = random_kg(rng, 500, 20000, 7, d, dtype=dtype, scale=0.3)
    G = mhr.load_kg(g, score_fn=fn)
    w64 = mhr.mhr_edge_scores(G, precision=2)            # all CSR edges
    w32 = mhr.mhr_edge_scores(G, precision=0)
    src = g.src_of_edges()
    want = oracle.edge_weights(g, src, g.rels, g.cols, fn=fn)
    assert np.array_equal(w64, want)                     # bit-exact
    # fp32 within the proven per-edge bound (global norms)
    ve = g.vemb_f32().astype(np.float64)
    re_ = g.remb_f32().astype(np.float64)
    if fn == "transe":
        N = 2 * np.abs(ve).sum(1).max() + np.abs(re_).sum(1).max()
        bound = (d + 4) * 2.0 ** -24 / (1 - (d + 4) * 2.0 ** -24) * (N + 2)
    else:
        M = np.abs(re_).max() * (ve ** 2).sum(1).max()
        bound = (d + 3) * 2.0 ** -24 / (1 - (d + 3) * 2.0 ** -24) * M
    assert np.abs(w32.astype(np.float64) - want).max() <= bound
    # explicit edge list, including a subset
    idx = rng.choice(g.E, 777, replace=False)
    sub = mhr.mhr_edge_scores(G, src[idx], g.rels[idx], g.cols[idx], precision=2)
    assert np.array_equal(sub, want[idx])
    G.close()


# --------------------------------------------------------------------------- golden paths
@pytest.mark.parametrize("fn", ["transe", "distmult"])
def test_topk_golden(mhr, fn):
    gj = load_golden()
    g = kg_from_golden(gj)
    G = mhr.load_kg(g, score_fn=fn)
    want = [tuple(p) for p in gj[f"expected_{fn}"]["paths_score_u_r1_v_r2_r3"]]
    for K in (1, 3, 5, 11, 20, 1024):
        got = mhr.mhr_topk_paths(G, 0, 9, K)
        assert path_tuples(got) == [(float(p[0]),) + tuple(p[1:]) for p in want[:K]]
    if fn == "transe":
        want2 = [tuple(p) for p in gj["expected2_transe"]["paths_score_u_r1_v_r2_r3"]]
        got = mhr.mhr_topk_paths(G, 3, 9, 10)
        assert path_tuples(got) == [(float(p[0]),) + tuple(p[1:]) for p in want2]
    G.close()


def test_topk_golden_batched_and_edge_cases(mhr):
    gj = load_golden()
    g = kg_from_golden(gj)
    S = np.array([0, 3, 0, 5, 7, 0, 8], dtype=np.uint32)
    T = np.array([9, 9, 0, 9, 0, 8, 9], dtype=np.uint32)  # (0,0) invalid; (0,8): no paths
    run_and_compare(mhr, g, S, T, 4, "transe")
    G = mhr.load_kg(g)
    with pytest.raises(mhr.MhrError) as e:
        mhr.mhr_topk_paths(G, 2, 2, 5)
    assert e.value.status == mhr.MHR_EINVAL
    with pytest.raises(mhr.MhrError) as e:
        mhr.mhr_topk_paths(G, 0, 10, 5)
    assert e.value.status == mhr.MHR_EINVAL
    with pytest.raises(mhr.MhrError) as e:
        mhr.mhr_topk_paths(G, 0, 9, mhr.MHR_K_MAX + 1)
    assert e.value.status == mhr.MHR_ERANGE
    with pytest.raises(mhr.MhrError) as e:
        mhr.mhr_topk_paths(G, 0, 9, 0)
    assert e.value.status == mhr.MHR_EINVAL
    assert len(mhr.mhr_topk_paths(G, 0, 8, 5)) == 0
    G.close()


# --------------------------------------------------------------------------- random graphs
@pytest.mark.parametrize("prune,order", [(0, 0), (1, 0), (1, 1), (0, 1)])
@pytest.mark.parametrize("fn", ["transe", "distmult"])
def test_topk_random_small_graphs(mhr, fn, prune, order):
    rng = np.random.default_rng(101 if fn == "transe" else 202)
    for trial in range(30):
        n = int(rng.integers(8, 300))
        m = int(rng.integers(20, 30 * n))
        R = int(rng.integers(1, 6))
        d = int(rng.choice([1, 3, 4, 8, 16, 64]))
        dtype = "bf16" if trial % 3 == 0 else "f32"
        g = random_kg(rng, n, m, R, d, dtype=dtype, dyadic=(trial % 5 == 0))
        nq = 24
        S = rng.integers(0, n, nq).astype(np.uint32)
        T = rng.integers(0, n, nq).astype(np.uint32)
        K = int(rng.choice([1, 2, 7, 50, 300]))
        run_and_compare(mhr, g, S, T, K, fn, opts={"prune": prune, "order": order})


@pytest.mark.parametrize("prune,order", [(0, 0), (1, 1)])
def test_topk_all_ties_zero_embeddings(mhr, prune, order):
    """Every score equal: the order is the id order and the fp32 screen cannot
    separate anything (exercises the tie-heavy exact path)."""
    rng = np.random.default_rng(7)
    for trial in range(6):
        g = random_kg(rng, 200, 8000, 3, 8, zero=True)
        S = rng.integers(0, 200, 10).astype(np.uint32)
        T = rng.integers(0, 200, 10).astype(np.uint32)
        for fn in ("transe", "distmult"):
            run_and_compare(mhr, g, S, T, int(rng.choice([5, 64, 500])), fn, opts={"prune": prune, "order": order})


def test_topk_dyadic_many_ties_large_K(mhr):
    rng = np.random.default_rng(8)
    g = random_kg(rng, 400, 30000, 2, 2, dyadic=True)
    S = rng.integers(0, 400, 16).astype(np.uint32)
    T = rng.integers(0, 400, 16).astype(np.uint32)
    run_and_compare(mhr, g, S, T, 1024, "transe")
    run_and_compare(mhr, g, S, T, 100, "distmult")


@pytest.mark.parametrize("opts", [{"prune": 1, "order": 1}, {"prune": 1, "order": 1, "chunk": 256}])
def test_topk_dyadic_ties_largest_K_pruned(mhr, opts):
    """K = 1024 (the largest K) with bound pruning, on dyadic embeddings where
    many paths tie: the kept band and the tie order at the K-th score are
    decided with pruning on, in small and large work items."""
    rng = np.random.default_rng(18)
    g = random_kg(rng, 400, 30000, 2, 2, dyadic=True)
    S = rng.integers(0, 400, 16).astype(np.uint32)
    T = rng.integers(0, 400, 16).astype(np.uint32)
    run_and_compare(mhr, g, S, T, mhr.MHR_K_MAX, "transe", opts=opts)


def test_duplicate_queries_in_one_batch(mhr):
    """The same hub query 40 times in one batch (and its reverse 40 times), in
    64-edge work items: CTAs take and steal items of many copies at once, each
    copy keeps its own threshold and candidates, and every copy returns the
    oracle's list."""
    rng = np.random.default_rng(19)
    g = random_kg(rng, 300, 12000, 4, 16)
    deg_out, deg_in = np.diff(g.offsets), np.bincount(g.cols, minlength=g.n)
    s = int(np.argmax(deg_out))
    t = int(np.argmax(np.where(np.arange(g.n) == s, -1, deg_in)))
    S = np.array([s] * 40 + [t] * 40, dtype=np.uint32)
    T = np.array([t] * 40 + [s] * 40, dtype=np.uint32)
    out, n_out = run_and_compare(mhr, g, S, T, 60, "transe", opts={"prune": 1, "order": 1, "chunk": 64})
    for q in range(1, 40):
        assert out[q][: n_out[q]].tobytes() == out[0][: n_out[0]].tobytes()
        assert out[40 + q][: n_out[40 + q]].tobytes() == out[40][: n_out[40]].tobytes()


@pytest.mark.parametrize("opts", [None, {"prune": 1, "order": 1}])
def test_more_queries_than_a_block(mhr, opts):
    """5,000 queries in one batch: more queries than one 1,024-thread block of
    the planning kernels covers per pass, so their block-wide scans carry
    across passes; every query is compared with the oracle."""
    rng = np.random.default_rng(20)
    g = random_kg(rng, 2000, 40000, 3, 8)
    S = rng.integers(0, 2000, 5000).astype(np.uint32)
    T = rng.integers(0, 2000, 5000).astype(np.uint32)
    run_and_compare(mhr, g, S, T, 10, "transe", opts=opts)


@pytest.mark.parametrize("prune,order", [(0, 0), (1, 0), (1, 1)])
@pytest.mark.parametrize("chunk", [32, 64, 1024, 16384, 32768])
def test_topk_chunk_sizes(mhr, chunk, prune, order):
    """Work items of any size give the same answer (several items per query,
    ragged tails, hub rows split across items)."""
    g = synth.gen_rmat_kg(13, 6000, 120_000, 5, 3, seed=4)
    g.vemb, g.remb = synth.gen_embeddings(g.n, g.R, 16, 0.25, seed=4)
    S, T = synth.queries_edge_biased(g, 20, seed=4)
    run_and_compare(mhr, g, S, T, 60, "transe", opts={"chunk": chunk, "prune": prune, "order": order})


def test_tiny_workload(mhr):
    """10k vertices / 100k edges Zipf(2.1), d=64 fp32, hub query, K=10 (+ K=100)."""
    g, S, T, K, spec = synth.workload("tiny")
    for prune, order in ((0, 0), (1, 0), (1, 1)):
        o = {"prune": prune, "order": order}
        run_and_compare(mhr, g, S, T, K, "transe", opts=o)
        run_and_compare(mhr, g, S, T, 100, "transe", opts=o)
        run_and_compare(mhr, g, S, T, K, "distmult", opts=o)
        S2, T2 = synth.queries_edge_biased(g, 64, seed=1)
        run_and_compare(mhr, g, S2, T2, K, "transe", opts=o)


def test_both_directions_and_repeat_determinism(mhr):
    g = synth.gen_rmat_kg(14, 12000, 200_000, 8, 3, seed=5)
    g.vemb, g.remb = synth.gen_embeddings(g.n, g.R, 32, 1 / math.sqrt(32), seed=5)
    od, idg = g.out_degree(), g.in_degree()
    rng = np.random.default_rng(5)
    # hub source with low in-degree target and the reverse, so both scan sides run
    hubs = np.argsort(-od)[:8].astype(np.uint32)
    lows = np.flatnonzero((idg > 0) & (idg < 3))[:8].astype(np.uint32)
    S = np.concatenate([hubs, lows, rng.integers(0, g.n, 16).astype(np.uint32)])
    T = np.concatenate([lows, hubs, rng.integers(0, g.n, 16).astype(np.uint32)])
    out1, n1 = run_and_compare(mhr, g, S, T, 100, "transe")
    G = mhr.load_kg(g)
    out2, n2 = mhr.mhr_topk_paths_batched(G, S, T, 100)
    G.close()
    assert np.array_equal(n1, n2)
    for q in range(len(S)):
        assert out1[q][: n1[q]].tobytes() == out2[q][: n2[q]].tobytes()


def test_large_vertex_count_coarse_bitmap(mhr):
    """n > 2^20: the shared-memory membership bitmap becomes coarse (several
    vertices per bit); a positive is found in the run of its bit in the sorted
    far list, located by the bit's rank.  Small work items exercise items and
    seed parts that start inside a run."""
    g = synth.gen_rmat_kg(22, 3_000_000, 2_000_000, 4, 2, seed=6)
    g.vemb, g.remb = synth.gen_embeddings(g.n, g.R, 8, 0.3, seed=6)
    S, T = synth.queries_edge_biased(g, 24, seed=6)
    run_and_compare(mhr, g, S, T, 50, "transe")
    run_and_compare(mhr, g, S, T, 50, "transe", opts={"prune": 1})
    run_and_compare(mhr, g, S, T, 50, "transe", opts={"prune": 1, "order": 1})
    run_and_compare(mhr, g, S, T, 50, "transe", opts={"prune": 1, "order": 1, "chunk": 256})


@pytest.mark.parametrize("opts", [None, {"prune": 1, "order": 1}])
def test_many_small_and_empty_queries(mhr, opts):
    """A batch of 600 queries whose sources have out-degree 0, 1 or 2 and whose
    targets have in-degree 0, 1 or 2: a warp's 32 expansion slots span dozens
    of query starts (several with no slot at all), so the warp's query search
    takes both its shuffle path and the per-lane fallback; results still
    match the oracle query by query."""
    rng = np.random.default_rng(31)
    n, R = 1500, 3
    src, dst = [], []
    for s in range(0, 500):                       # low-degree sources 0..499
        for _ in range(int(rng.integers(0, 3))):
            src.append(s); dst.append(int(rng.integers(500, 1000)))
    for _ in range(80000):                        # middle edges among 500..999
        src.append(int(rng.integers(500, 1000))); dst.append(int(rng.integers(500, 1000)))
    for t in range(1000, 1500):                   # low in-degree targets 1000..1499
        for _ in range(int(rng.integers(0, 3))):
            src.append(int(rng.integers(500, 1000))); dst.append(t)
    rel = rng.integers(0, R, len(src))
    offsets, cols, rels = synth.canonicalize(n, R, np.array(src), rel, np.array(dst))
    vemb = (rng.standard_normal((n, 8)) * 0.4).astype(np.float32)
    remb = (rng.standard_normal((R, 8)) * 0.4).astype(np.float32)
    g = synth.KG(n=n, R=R, n_types=1, offsets=offsets, cols=cols, rels=rels,
                 vtypes=np.zeros(n, dtype=np.uint8), vemb=vemb, remb=remb, dtype="f32")
    S = rng.integers(0, 500, 600).astype(np.uint32)
    T = rng.integers(1000, 1500, 600).astype(np.uint32)
    deg = np.diff(g.offsets)
    assert (deg[S] == 0).sum() > 100 and (deg[S] == 2).sum() > 100
    run_and_compare(mhr, g, S, T, 20, "transe", opts=opts)


def test_coarse_bitmap_dense_runs(mhr):
    """A coarse bitmap whose set bits cover runs of several far vertices: a
    hub target whose in-neighbours are consecutive vertex ids."""
    rng = np.random.default_rng(12)
    n, R = 2_200_000, 3
    hub_t, hub_s = 1_000_003, 17
    u = [hub_s] * 400
    v = list(range(2_000, 2_400))                        # hop-1: consecutive u
    r = list(rng.integers(0, R, 400))
    mids = rng.integers(2_000, 2_400, 6_000)
    for a, b in zip(mids, rng.integers(500_000, 500_600, 6_000)):
        u.append(int(a)); v.append(int(b)); r.append(int(rng.integers(0, R)))   # middle edges
    for b in range(500_000, 500_600):
        u.append(b); v.append(hub_t); r.append(int(rng.integers(0, R)))          # hop-3: consecutive v
    offsets, cols, rels = synth.canonicalize(n, R, np.array(u), np.array(r), np.array(v))
    vemb = (rng.standard_normal((n, 8)) * 0.3).astype(np.float32)
    remb = (rng.standard_normal((R, 8)) * 0.3).astype(np.float32)
    g = synth.KG(n=n, R=R, n_types=1, offsets=offsets, cols=cols, rels=rels,
                 vtypes=np.zeros(n, dtype=np.uint8), vemb=vemb, remb=remb, dtype="f32")
    S = np.array([hub_s, hub_s], dtype=np.uint32)
    T = np.array([hub_t, 500_010], dtype=np.uint32)
    for o in (None, {"prune": 1, "order": 1}, {"prune": 1, "order": 1, "chunk": 64}):
        run_and_compare(mhr, g, S, T, 40, "transe", opts=o)


def test_device_memory_batched(mhr):
    torch = pytest.importorskip("torch")
    g, S, T, K, spec = synth.workload("tiny")
    S2, T2 = synth.queries_edge_biased(g, 32, seed=2)
    G = mhr.load_kg(g, device=True)
    dS, dT = torch.from_numpy(S2.astype(np.int32)).cuda(), torch.from_numpy(T2.astype(np.int32)).cuda()
    out, n_out = mhr.mhr_topk_paths_batched(G, dS, dT, 20, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    paths = mhr.paths_from_device(out, 20)
    n_out = n_out.cpu().numpy()
    want, n_want = oracle.topk_paths_batch(g, S2, T2, 20)
    for q in range(len(S2)):
        compare_query(paths[q], int(n_out[q]), want[q, : n_want[q]], ctx=q)
    G.close()


def test_invalid_graphs_rejected(mhr):
    gj = load_golden()
    g = kg_from_golden(gj)
    bad = dict(offsets=g.offsets, cols=g.cols, rels=g.rels, vertex_emb=g.vemb, rel_emb=g.remb)

    def load(**kw):
        a = dict(bad)
        a.update(kw)
        return mhr.mhr_graph_load(a["offsets"], a["cols"], a["rels"], a["vertex_emb"], a["rel_emb"], g.R)

    cols = g.cols.copy()
    cols[0] = 99
    with pytest.raises(mhr.MhrError, match="destination"):
        load(cols=cols)
    rels = g.rels.copy()
    rels[0] = 7
    with pytest.raises(mhr.MhrError, match="relation"):
        load(rels=rels)
    cols = g.cols.copy()
    cols[1] = cols[0]
    rels = g.rels.copy()
    rels[1] = rels[0]
    with pytest.raises(mhr.MhrError, match="sorted"):
        load(cols=cols, rels=rels)
    cols = g.cols.copy()
    cols[0] = 0  # row 0 edge to itself
    with pytest.raises(mhr.MhrError):
        load(cols=cols)
    ve = g.vemb.copy()
    ve[3, 1] = np.nan
    with pytest.raises(mhr.MhrError, match="NaN"):
        load(vertex_emb=ve)
    off = g.offsets.copy()
    off[3], off[4] = off[4], off[3]
    with pytest.raises(mhr.MhrError, match="offsets"):
        load(offsets=off)


@pytest.mark.slow
def test_medium_workload_sampled(mhr):
    """The benchmark workload (R-MAT 1M vertices, 20M edges, d=128 fp32,
    64 edge-biased queries, K=100) in the benchmark's launch configuration;
    the oracle recomputes every query."""
    g, S, T, K, spec = synth.workload("medium")
    G = mhr.load_kg(g)
    out, n_out = mhr.mhr_topk_paths_batched(G, S, T, K)
    outp, n_outp, st = mhr.mhr_topk_paths_batched(G, S, T, K, opts={"prune": 1, "order": 1}, with_stats=True)
    G.close()
    assert st["pruned_edges"] > 0
    # the pruned form returns byte-identical results for every query
    assert np.array_equal(n_out, n_outp)
    for q in range(len(S)):
        assert out[q][: n_out[q]].tobytes() == outp[q][: n_outp[q]].tobytes()
    want, n_want = oracle.topk_paths_batch(g, S, T, K)
    for q in range(len(S)):
        compare_query(out[q], int(n_out[q]), want[q, : n_want[q]], ctx=int(q))


def test_work_counters_match_oracle(mhr):
    """edges_scanned = sum min(S_f, S_b); hits = middle edges joining the two
    frontiers; paths = all simple three-hop paths (counted by the oracle)."""
    g = synth.gen_rmat_kg(13, 6000, 120_000, 5, 3, seed=14)
    g.vemb, g.remb = synth.gen_embeddings(g.n, g.R, 16, 0.25, seed=14)
    S, T = synth.queries_edge_biased(g, 24, seed=14)
    G = mhr.load_kg(g)
    for chunk in (64, 16384, 32768):
        out, n_out, st = mhr.mhr_topk_paths_batched(G, S, T, 50, opts={"chunk": chunk}, with_stats=True)
        scanned = hits = paths = 0
        for s, t in zip(S.tolist(), T.tolist()):
            qs = oracle.query_stats(g, s, t)
            _, h, p = oracle.topk_paths(g, s, t, 1, with_counts=True)
            scanned += min(qs["s_f"], qs["s_b"])
            hits += h
            paths += p
        assert st["edges_scanned"] == scanned
        assert st["hits"] == hits
        assert st["paths"] == paths
        assert st["ms_join"] > 0 and st["ms_device"] >= st["ms_join"]
    G.close()


@pytest.mark.parametrize("prune", [0, 1])
def test_tensor_core_screen_distmult(mhr, prune):
    """precision 1: middle edges screened by the bf16 hi/lo tensor-core
    contraction; results identical to the oracle (and to precision 0)."""
    rng = np.random.default_rng(41 + prune)
    for trial in range(10):
        n = int(rng.integers(20, 400))
        d = int(rng.choice([3, 8, 16, 37, 64, 256]))
        R = int(rng.integers(1, 17))
        dtype = "bf16" if trial % 3 == 0 else "f32"
        g = random_kg(rng, n, int(rng.integers(50, 25 * n)), R, d, dtype=dtype, dyadic=(trial % 4 == 0))
        S = rng.integers(0, n, 16).astype(np.uint32)
        T = rng.integers(0, n, 16).astype(np.uint32)
        run_and_compare(mhr, g, S, T, int(rng.choice([1, 10, 100])), "distmult",
                        opts={"precision": 1, "prune": prune, "order": prune})
    g = synth.gen_rmat_kg(13, 6000, 120_000, 16, 3, seed=42)
    g.vemb, g.remb = synth.gen_embeddings(g.n, g.R, 256, 1 / 16, seed=42)
    S, T = synth.queries_edge_biased(g, 24, seed=42)
    run_and_compare(mhr, g, S, T, 100, "distmult", opts={"precision": 1, "prune": prune, "order": prune})


def test_tensor_core_screen_rejects_unsupported(mhr):
    gj = load_golden()
    g = kg_from_golden(gj)
    G = mhr.load_kg(g, score_fn="transe")
    with pytest.raises(mhr.MhrError) as e:
        mhr.mhr_topk_paths(G, 0, 9, 5, opts={"precision": 1})
    assert e.value.status == mhr.MHR_EINVAL
    G.close()
    rng = np.random.default_rng(5)
    g = random_kg(rng, 50, 400, 20, 8)
    G = mhr.load_kg(g, score_fn="distmult")
    with pytest.raises(mhr.MhrError):
        mhr.mhr_topk_paths(G, 0, 1, 5, opts={"precision": 1})
    G.close()


def test_autotune_picks_a_candidate_and_keeps_results(mhr):
    """The launch-shape autotuner times every (work-item size, scan tile) pair
    on the batch and returns the fastest; results with the chosen shape equal
    the default's and the oracle's."""
    g = synth.gen_rmat_kg(14, 12000, 200_000, 6, 3, seed=41)
    g.vemb, g.remb = synth.gen_embeddings(g.n, g.R, 32, 1 / 8, seed=41)
    S, T = synth.queries_edge_biased(g, 24, seed=41)
    G = mhr.load_kg(g)
    opts = {"prune": 1, "order": 1}
    chunks, tiles = (64, 512, 2048), (4, 8)
    bc, bt, bp, ms = mhr.mhr_autotune(G, S, T, 30, opts=opts, chunks=chunks, tiles=tiles, reps=2)
    assert bc in chunks and bt in tiles and bp == 0 and set(ms) == {(0, c, t) for c in chunks for t in tiles}
    assert all(v > 0 for v in ms.values()) and ms[(0, bc, bt)] == min(ms.values())
    out_b, n_b = mhr.mhr_topk_paths_batched(G, S, T, 30, opts={**opts, "chunk": bc, "tile": bt})
    out_d, n_d = mhr.mhr_topk_paths_batched(G, S, T, 30)
    assert np.array_equal(n_b, n_d)
    for q in range(len(S)):
        assert out_b[q][: n_b[q]].tobytes() == out_d[q][: n_d[q]].tobytes()
    want, n_want = oracle.topk_paths_batch(g, S, T, 30)
    for q in range(len(S)):
        compare_query(out_b[q], n_b[q], want[q][: n_want[q]], ctx=q)
    with pytest.raises(mhr.MhrError):
        mhr.mhr_autotune(G, S, T, 30, chunks=(100,))
    with pytest.raises(mhr.MhrError):
        mhr.mhr_autotune(G, S, T, 30, tiles=(5,))
    with pytest.raises(mhr.MhrError):
        mhr.mhr_topk_paths_batched(G, S, T, 30, opts={"tile": 6})
    G.close()


def test_autotune_chooses_the_screen_for_distmult(mhr):
    """With precision -1 the autotuner also times the bf16 tensor-core screen
    against the fp32 one (DistMult, <= 16 relations) and returns the faster;
    both give the oracle's lists."""
    g = synth.gen_rmat_kg(13, 6000, 80_000, 8, 3, seed=43)
    g.vemb, g.remb = synth.gen_embeddings(g.n, g.R, 32, 1 / 8, seed=43)
    S, T = synth.queries_edge_biased(g, 16, seed=43)
    G = mhr.load_kg(g, score_fn="distmult")
    bc, bt, bp, ms = mhr.mhr_autotune(G, S, T, 20, opts={"prune": 1, "order": 1, "precision": -1},
                                      chunks=(1024,), tiles=(4,), reps=1)
    assert set(ms) == {(0, 1024, 4), (1, 1024, 4)} and bp in (0, 1) and ms[(bp, bc, bt)] == min(ms.values())
    want, n_want = oracle.topk_paths_batch(g, S, T, 20, fn="distmult")
    for prec in (0, 1):
        out, n = mhr.mhr_topk_paths_batched(G, S, T, 20, opts={"prune": 1, "order": 1, "precision": prec})
        for q in range(len(S)):
            compare_query(out[q], n[q], want[q][: n_want[q]], ctx=(prec, q))
    G.close()


@pytest.mark.parametrize("fn", ["transe", "distmult"])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_subnormal_and_signed_zero_embeddings(mhr, fn, dtype):
    """Embedding tables holding subnormals, +0 and -0 next to ordinary values:
    the fp64 rescoring widens every stored value exactly, so scores stay
    bit-identical to the oracle's."""
    rng = np.random.default_rng(77)
    g = random_kg(rng, 150, 2500, 4, 16)
    vemb = g.vemb.copy()
    remb = g.remb.copy()
    for tab in (vemb, remb):
        mask = rng.random(tab.shape)
        tab[mask < 0.15] = np.float32(1e-40) * rng.choice([-1.0, 1.0], size=int((mask < 0.15).sum())).astype(np.float32)
        tab[(mask >= 0.15) & (mask < 0.2)] = np.float32(-0.0)
        tab[(mask >= 0.2) & (mask < 0.25)] = np.float32(0.0)
        tab[(mask >= 0.25) & (mask < 0.3)] = np.float32(2.0 ** -126)
    assert np.any(np.abs(vemb[vemb != 0]) < np.float32(1.1754944e-38))
    if dtype == "bf16":
        g.vemb, g.remb, g.dtype = synth.to_bf16_bits(vemb), synth.to_bf16_bits(remb), "bf16"
    else:
        g.vemb, g.remb = vemb, remb
    S = rng.integers(0, g.n, 12).astype(np.uint32)
    T = rng.integers(0, g.n, 12).astype(np.uint32)
    run_and_compare(mhr, g, S, T, 25, fn)
