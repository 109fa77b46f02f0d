"""Constrained three-hop queries (Sec. 3.1 query shape) on the GPU against the
oracle, element by element, through the C ABI.

The paper's query follows one relation per hop (award-winner, works-in,
affiliated-with) and keeps persons as the intermediate entities; the
library takes an allowed-relation set per hop and an allowed-type set for u
and for v.  Bar: path count, ids, order and fp64 scores bit-identical to
oracle.topk_paths_masked.
"""

import numpy as np
import pytest

import oracle
import synth
from tests._graphs import kg_from_golden, load_golden, random_kg
from tests.test_gpu_parity import compare_query

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mhr():
    import paper_2406_07727_gb300 as m
    return m


def random_constraints(rng, R, n_types):
    def pick(n):
        if rng.random() < 0.25:
            return None
        k = int(rng.integers(1, n + 1))
        return sorted(int(x) for x in rng.choice(n, size=k, replace=False))
    return {"rel1": pick(R), "rel2": pick(R), "rel3": pick(R),
            "types_u": pick(n_types), "types_v": pick(n_types)}


def masked_oracle(g, S, T, K, c, fn):
    out = []
    for s, t in zip(S.tolist(), T.tolist()):
        if s == t:
            out.append(None)
            continue
        out.append(oracle.topk_paths_masked(g, s, t, K, rel1=c.get("rel1"), rel2=c.get("rel2"), rel3=c.get("rel3"),
                                            types_u=c.get("types_u"), types_v=c.get("types_v"), fn=fn))
    return out


def run_masked(m, g, S, T, K, c, fn, opts=None):
    G = m.load_kg(g, score_fn=fn)
    try:
        o = dict(opts or {})
        o["constraints"] = c
        out, n_out = m.mhr_topk_paths_batched(G, S, T, K, opts=o)
    finally:
        G.close()
    want = masked_oracle(g, S, T, K, c, fn)
    for q, w in enumerate(want):
        if w is None:
            assert n_out[q] == -1
            continue
        compare_query(out[q], int(n_out[q]), w, ctx=(q, int(S[q]), int(T[q]), c))
    return out, n_out


@pytest.mark.parametrize("fn", ["transe", "distmult"])
@pytest.mark.parametrize("opts", [{"prune": 0, "order": 0}, {"prune": 1, "order": 1},
                                  {"prune": 1, "order": 1, "chunk": 64}])
def test_random_graphs_random_constraints(mhr, fn, opts):
    rng = np.random.default_rng(101 + len(opts) + (fn == "distmult"))
    for trial in range(10):
        n = int(rng.integers(12, 300))
        R = int(rng.integers(1, 9))
        d = int(rng.choice([4, 16, 64]))
        g = random_kg(rng, n, int(rng.integers(40, 20 * n)), R, d, dtype="bf16" if trial % 3 == 0 else "f32",
                      dyadic=(trial % 4 == 1))
        S = rng.integers(0, n, 12).astype(np.uint32)
        T = rng.integers(0, n, 12).astype(np.uint32)
        c = random_constraints(rng, R, 3)
        run_masked(mhr, g, S, T, int(rng.choice([1, 7, 50, 400])), c, fn, opts)


def test_all_allowed_equals_unconstrained(mhr):
    """Constraints that allow every relation and type return the unconstrained
    search's bytes."""
    rng = np.random.default_rng(7)
    g = random_kg(rng, 400, 9000, 6, 32)
    S = rng.integers(0, g.n, 20).astype(np.uint32)
    T = rng.integers(0, g.n, 20).astype(np.uint32)
    G = mhr.load_kg(g)
    base, nb = mhr.mhr_topk_paths_batched(G, S, T, 30)
    every = {"rel1": range(6), "rel2": range(6), "rel3": range(6), "types_u": range(256), "types_v": range(256)}
    for c in ({}, every):
        out, n = mhr.mhr_topk_paths_batched(G, S, T, 30, opts={"constraints": c})
        assert np.array_equal(n, nb)
        for q in range(len(S)):
            assert out[q][: n[q]].tobytes() == base[q][: nb[q]].tobytes()
    G.close()


def test_golden_graph_turing_shape(mhr):
    """The hand graph with one relation per hop and typed intermediates: the
    shape of the Turing query (award-winner, works-in, affiliated-with; u
    and v persons)."""
    gj = load_golden()
    g = kg_from_golden(gj)
    for c in ({"rel1": [0], "rel2": [1], "rel3": [0]}, {"types_u": [1], "types_v": [0, 2]},
              {"rel1": [1], "rel2": [0, 1], "rel3": [1], "types_u": [0, 1, 2], "types_v": [1]},
              {"rel2": []}):
        for fn in ("transe", "distmult"):
            S = np.array([0, 0, 3], dtype=np.uint32)
            T = np.array([9, 5, 9], dtype=np.uint32)
            run_masked(mhr, g, S, T, 20, c, fn)


def test_tie_heavy_constrained(mhr):
    """Zero embeddings: every score ties, the order is the id order; enough
    paths that the exact fallback resolves some queries."""
    rng = np.random.default_rng(19)
    g = random_kg(rng, 60, 2500, 4, 8, zero=True)
    S = rng.integers(0, g.n, 8).astype(np.uint32)
    T = rng.integers(0, g.n, 8).astype(np.uint32)
    c = {"rel1": [0, 1, 3], "rel2": [1, 2, 3], "rel3": [0, 2], "types_u": [0, 2], "types_v": None}
    for K in (5, 100, 1024):
        run_masked(mhr, g, S, T, K, c, "distmult", {"prune": 1, "order": 1})


def test_tensor_core_screen_constrained(mhr):
    rng = np.random.default_rng(23)
    g = random_kg(rng, 300, 8000, 12, 64)
    S = rng.integers(0, g.n, 16).astype(np.uint32)
    T = rng.integers(0, g.n, 16).astype(np.uint32)
    c = random_constraints(rng, 12, 3)
    run_masked(mhr, g, S, T, 40, c, "distmult", {"precision": 1, "prune": 1, "order": 1})


def test_constraint_errors(mhr):
    rng = np.random.default_rng(3)
    g = random_kg(rng, 50, 400, 4, 8)
    G = mhr.load_kg(g)
    with pytest.raises(ValueError):
        mhr.mhr_topk_paths_batched(G, np.array([1], np.uint32), np.array([2], np.uint32), 5,
                                   opts={"constraints": {"rel1": [4]}})
    with pytest.raises(ValueError):
        mhr.mhr_topk_paths_batched(G, np.array([1], np.uint32), np.array([2], np.uint32), 5,
                                   opts={"constraints": {"types_u": [256]}})
    G.close()


@pytest.mark.slow
def test_medium_workload_constrained(mhr):
    """The medium R-MAT graph (1M vertices, 20M edges, 16 relations, 6 types)
    with a Turing-shaped constraint: half of the relations per hop, u and v of
    two of the six types; all 64 queries in one call, pruned and plain forms
    identical, 12 queries against the oracle."""
    g, S, T, K, spec = synth.workload("medium")
    c = {"rel1": range(0, 8), "rel2": range(4, 12), "rel3": range(8, 16), "types_u": [0, 1], "types_v": [2, 3]}
    G = mhr.load_kg(g)
    try:
        base, nb = mhr.mhr_topk_paths_batched(G, S, T, K, opts={"constraints": c})
        out, n, st = mhr.mhr_topk_paths_batched(G, S, T, K, opts={"constraints": c, "prune": 1, "order": 1},
                                                with_stats=True)
    finally:
        G.close()
    assert np.array_equal(n, nb)
    for q in range(len(S)):
        assert out[q][: n[q]].tobytes() == base[q][: nb[q]].tobytes()
    assert st["pruned_edges"] > 0
    sample = np.arange(0, len(S), 6)[:12]
    want = masked_oracle(g, S[sample], T[sample], K, {k: (list(v) if v is not None else None) for k, v in c.items()},
                         "transe")
    for i, q in enumerate(sample):
        compare_query(base[q], int(nb[q]), want[i], ctx=int(q))
