"""The CPU oracle pinned to things other than itself (CPU only).

Pins: hand-derived worked examples (tests/golden), closed forms for zero
embeddings, the exact rational edge weight within the fp64 rounding bound, a
second independent route (pure-Python meet in the middle), and the
brute-force invariants: every returned path exists with its relations, scores
recompute, K = all equals the full sorted enumeration, prefix consistency in K.
"""

from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle.mitm import MITM
from tests._graphs import kg_from_golden, load_golden, path_tuples, random_kg

U64 = 2.0 ** -53


def gamma_n(n, u=U64):
    return n * u / (1 - n * u)


# --------------------------------------------------------------------------- golden
@pytest.mark.parametrize("fn", ["transe", "distmult"])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_golden_edge_weights(fn, dtype):
    gj = load_golden()
    g = kg_from_golden(gj, dtype)
    rows = gj[f"edge_weights_{fn}"]["rows"]
    src = np.array([r[0] for r in rows], dtype=np.uint32)
    rel = np.array([r[1] for r in rows], dtype=np.uint16)
    dst = np.array([r[2] for r in rows], dtype=np.uint32)
    want = np.array([r[3] for r in rows], dtype=np.float64)
    got = oracle.edge_weights(g, src, rel, dst, fn=fn)
    assert got.tolist() == want.tolist()
    m = MITM(g, fn)
    assert [m.weight(int(a), int(b), int(c)) for a, b, c in zip(src, rel, dst)] == want.tolist()


@pytest.mark.parametrize("fn", ["transe", "distmult"])
def test_golden_paths(fn):
    gj = load_golden()
    g = kg_from_golden(gj)
    want = [tuple(p) for p in gj[f"expected_{fn}"]["paths_score_u_r1_v_r2_r3"]]
    s, t = gj["query"]["s"], gj["query"]["t"]
    got, hits, npaths = oracle.topk_paths(g, s, t, 100, fn=fn, with_counts=True)
    assert path_tuples(got) == [tuple(float(x) if i == 0 else x for i, x in enumerate(p)) for p in want]
    assert npaths == len(want) == 11
    # hits: middle edges reaching V_t: (1,r0,4) (1,r1,5) (2,r1,4) (3,r0,1) (3,r2,4)
    assert hits == 5
    for K in (1, 3, 6, 11):
        assert path_tuples(oracle.topk_paths(g, s, t, K, fn=fn)) == path_tuples(got)[:K]
    assert MITM(g, fn).topk(s, t, 100) == path_tuples(got)


def test_golden_second_query():
    gj = load_golden()
    g = kg_from_golden(gj)
    want = [tuple(p) for p in gj["expected2_transe"]["paths_score_u_r1_v_r2_r3"]]
    s, t = gj["query2"]["s"], gj["query2"]["t"]
    assert path_tuples(oracle.topk_paths(g, s, t, 50)) == [
        (float(p[0]),) + tuple(p[1:]) for p in want]


def test_golden_stats():
    gj = load_golden()
    g = kg_from_golden(gj)
    st = oracle.query_stats(g, 0, 9)
    # N_out(0) = {1, 1, 2, 3, 9}: distinct u not in {s,t} = {1, 2, 3}
    assert st["deg_s"] == 5 and st["n_u"] == 3
    # S_f = deg_out(1) + deg_out(2) + deg_out(3) = 4 + 2 + 2
    assert st["s_f"] == 8
    # N_in(9) = {0, 1, 4, 4, 5, 7, 8}: distinct v not in {s,t} = {1, 4, 5, 7, 8}
    assert st["deg_t"] == 7 and st["n_v"] == 5
    # in-degrees: 1 <- {0,0,3} = 3; 4 <- {1,2,3,9} = 4; 5 <- {1} = 1; 7 <- {6} = 1; 8 <- {} = 0
    assert st["s_b"] == 9


# --------------------------------------------------------------------------- closed forms
def test_zero_vertex_embeddings_closed_form():
    """e = 0: TransE w = gamma - ||w_r||_1 and DistMult w = 0 for every edge."""
    rng = np.random.default_rng(5)
    g = random_kg(rng, 30, 200, 4, 8, dyadic=True)
    g.vemb = np.zeros_like(g.vemb)
    src = np.repeat(np.arange(g.n, dtype=np.uint32), np.diff(g.offsets))
    for gamma in (1.0, 0.25, -3.0):
        w = oracle.edge_weights(g, src, g.rels, g.cols, fn="transe", gamma=gamma)
        want = gamma - np.abs(g.remb.astype(np.float64)).sum(axis=1)[g.rels]
        assert w.tolist() == want.tolist()
    assert not oracle.edge_weights(g, src, g.rels, g.cols, fn="distmult").any()


def test_all_zero_distmult_orders_by_ids():
    """All scores 0: the order reduces to the lexicographic sort of ids."""
    rng = np.random.default_rng(6)
    for trial in range(20):
        g = random_kg(rng, 25, 250, 3, 4, zero=True)
        s, t = (int(x) for x in rng.choice(g.n, size=2, replace=False))
        allp = MITM(g, "distmult").all_paths(s, t)
        ids = sorted(p[1:] for p in allp)
        got = oracle.topk_paths(g, s, t, 10_000, fn="distmult")
        assert [p[1:] for p in path_tuples(got)] == ids
        assert all(p[0] == 0.0 for p in path_tuples(got))


def test_exact_rational_within_fp64_bound():
    """|w_fp64 - w_exact| <= gamma_{d+2} * (sum |a|+|b|+|c| + |gamma|) (TransE) and
    <= gamma_{d+1} * sum |a b c| (DistMult); a dropped term, wrong sign or
    swapped operand would be off by far more."""
    rng = np.random.default_rng(7)
    for d in (1, 7, 64, 200):
        g = random_kg(rng, 12, 60, 3, d, scale=1.0)
        src = np.repeat(np.arange(g.n, dtype=np.uint32), np.diff(g.offsets))
        wt = oracle.edge_weights(g, src, g.rels, g.cols, fn="transe", gamma=1.0)
        wd = oracle.edge_weights(g, src, g.rels, g.cols, fn="distmult")
        for i in range(len(src)):
            a = [Fraction(float(x)) for x in g.vemb[src[i]]]
            b = [Fraction(float(x)) for x in g.remb[g.rels[i]]]
            c = [Fraction(float(x)) for x in g.vemb[g.cols[i]]]
            ex_t = 1 - sum(abs(x + y - z) for x, y, z in zip(a, b, c))
            norm = sum(abs(x) + abs(y) + abs(z) for x, y, z in zip(a, b, c)) + 1
            assert abs(Fraction(wt[i]) - ex_t) <= Fraction(gamma_n(d + 2)) * norm
            ex_d = sum(x * y * z for x, y, z in zip(a, b, c))
            mag = sum(abs(x * y * z) for x, y, z in zip(a, b, c))
            assert abs(Fraction(wd[i]) - ex_d) <= Fraction(gamma_n(d + 1)) * mag


# --------------------------------------------------------------------------- two routes
@pytest.mark.parametrize("fn", ["transe", "distmult"])
def test_brute_force_equals_mitm_random(fn):
    rng = np.random.default_rng(11 if fn == "transe" else 12)
    checked = 0
    for trial in range(600):
        n = int(rng.integers(4, 40))
        m = int(rng.integers(5, 8 * n))
        R = int(rng.integers(1, 5))
        d = int(rng.integers(1, 6))
        dtype = "bf16" if trial % 5 == 0 else "f32"
        g = random_kg(rng, n, m, R, d, dtype=dtype, dyadic=(trial % 7 == 0))
        s, t = (int(x) for x in rng.choice(n, size=2, replace=False))
        want = MITM(g, fn).all_paths(s, t)
        got = path_tuples(oracle.topk_paths(g, s, t, max(len(want), 1) + 3, fn=fn))
        assert got == want, (trial, n, m, R, d)
        K = int(rng.integers(1, 6))
        assert path_tuples(oracle.topk_paths(g, s, t, K, fn=fn)) == want[:K]
        checked += len(want)
    assert checked > 1000


# --------------------------------------------------------------------------- invariants
def test_invariants_zipf_graph():
    import synth
    g = synth.gen_zipf_kg(400, 6000, 5, 3, seed=3)
    rng = np.random.default_rng(3)
    g.vemb = (rng.standard_normal((g.n, 6)) * 0.4).astype(np.float32)
    g.remb = (rng.standard_normal((g.R, 6)) * 0.4).astype(np.float32)
    od = g.out_degree()
    s = int(np.argmax(od))
    t = int(np.argmax(g.in_degree()))
    if t == s:
        t = (s + 1) % g.n
    mitm = MITM(g, "transe")
    full = mitm.all_paths(s, t)
    assert len(full) > 100
    everything = path_tuples(oracle.topk_paths(g, s, t, len(full) + 10))
    assert everything == full                                  # K = all
    for K in (1, 2, 17, 50, len(full) - 1):
        assert path_tuples(oracle.topk_paths(g, s, t, K)) == full[:K]   # prefix consistency
    edges = set(zip(np.repeat(np.arange(g.n), od).tolist(), g.rels.tolist(), g.cols.tolist()))
    for S, u, r1, v, r2, r3 in everything[:200]:
        assert (s, r1, u) in edges and (u, r2, v) in edges and (v, r3, t) in edges
        assert len({s, u, v, t}) == 4
        assert (mitm.weight(s, r1, u) + mitm.weight(u, r2, v)) + mitm.weight(v, r3, t) == S


def test_invalid_queries():
    gj = load_golden()
    g = kg_from_golden(gj)
    with pytest.raises(ValueError):
        oracle.topk_paths(g, 3, 3, 5)
    with pytest.raises(ValueError):
        oracle.topk_paths(g, 0, 10, 5)
    with pytest.raises(ValueError):
        oracle.topk_paths(g, 0, 9, 0)


def test_no_paths():
    gj = load_golden()
    g = kg_from_golden(gj)
    # vertex 8 has no in-edges: nothing ends there
    assert len(oracle.topk_paths(g, 0, 8, 10)) == 0
    # vertex 7 only reaches 9
    assert len(oracle.topk_paths(g, 7, 0, 10)) == 0


def test_batch_matches_single():
    import synth
    g = synth.gen_zipf_kg(300, 3000, 4, 3, seed=9)
    rng = np.random.default_rng(9)
    g.vemb = rng.standard_normal((g.n, 5)).astype(np.float32)
    g.remb = rng.standard_normal((g.R, 5)).astype(np.float32)
    S, T = synth.queries_edge_biased(g, 12, seed=9)
    out, n_out = oracle.topk_paths_batch(g, S, T, 7)
    for q in range(len(S)):
        single = oracle.topk_paths(g, int(S[q]), int(T[q]), 7)
        assert n_out[q] == len(single)
        assert path_tuples(out[q, : n_out[q]]) == path_tuples(single)


def test_top_k_merges_associatively():
    """Alg. 2 merges thread-private K-heaps with a tree; under the total order
    (score desc, then ids) the K best of a union are the K best of the union of
    each part's K best, however the paths are split and in whatever order the
    parts are merged."""
    rng = np.random.default_rng(41)
    g = random_kg(rng, 30, 600, 3, 4, dyadic=True)   # dyadic: many exact score ties
    full = None
    for _ in range(20):
        s, t = [int(x) for x in rng.choice(g.n, size=2, replace=False)]
        full = path_tuples(oracle.topk_paths(g, s, t, 10 ** 6))
        if len(full) > 40:
            break
    assert full and len(full) > 40
    key = lambda p: (-p[0],) + tuple(p[1:])
    for K in (1, 7, 25):
        want = sorted(full, key=key)[:K]
        assert path_tuples(oracle.topk_paths(g, s, t, K)) == want   # the oracle's bounded heap
        for workers in (2, 3, 8):
            perm = rng.permutation(len(full))
            parts = [[full[i] for i in perm[w::workers]] for w in range(workers)]
            heaps = [sorted(p, key=key)[:K] for p in parts]
            while len(heaps) > 1:                       # pairwise tree reduction
                order = rng.permutation(len(heaps))
                heaps = [sorted(heaps[order[i]] + (heaps[order[i + 1]] if i + 1 < len(heaps) else []),
                                key=key)[:K] for i in range(0, len(heaps), 2)]
            assert heaps[0] == want
