"""The tail-prediction oracle (Alg. 3 / Alg. 4) pinned to things other than itself.

Pins: a hand-derived example with dyadic embeddings (every value below is
worked out by hand in the comments), a closed form for zero vertex
embeddings, the selection checked against a full NumPy lexicographic sort of
the independently pinned edge weights (including many exact ties from
bfloat16 inputs on a small grid), prefix consistency in K, and the
candidate-type filter.
"""

import numpy as np
import pytest

import oracle
import synth
from tests._graphs import random_kg


def _hand_kg(dtype="f32"):
    # 6 vertices, d = 2, one relation; every value is a small dyadic rational,
    # so all arithmetic below is exact in fp32, bf16 and fp64.
    vemb = np.array([[0.5, 0.0],     # v0 (type 0, the head)
                     [1.0, -0.5],    # v1 (type 1)
                     [0.0, 0.0],     # v2 (type 1)
                     [1.0, 0.5],     # v3 (type 1)
                     [1.0, -1.0],    # v4 (type 0)
                     [0.5, -0.5]],   # v5 (type 1)
                    dtype=np.float32)
    remb = np.array([[0.5, -0.5]], dtype=np.float32)
    vtypes = np.array([0, 1, 1, 1, 0, 1], dtype=np.uint8)
    offsets, cols, rels = synth.canonicalize(6, 1, np.array([0]), np.array([0]), np.array([1]))
    if dtype == "bf16":
        vemb, remb = synth.to_bf16_bits(vemb), synth.to_bf16_bits(remb)
    return synth.KG(n=6, R=1, n_types=2, offsets=offsets, cols=cols, rels=rels, vtypes=vtypes,
                    vemb=vemb, remb=remb, dtype=dtype)


def _pairs(out, n):
    return [(float(x["score"]), int(x["v"])) for x in out[:n]]


# TransE, head 0, relation 0: q = e0 + w0 = (1, -0.5); w = 1 - |q - e_c|_1
#   v0: |0.5| + |-0.5| = 1   -> 0       v1: 0 + 0 = 0        -> 1
#   v2: 1 + 0.5 = 1.5        -> -0.5    v3: 0 + 1 = 1        -> 0
#   v4: 0 + 0.5 = 0.5        -> 0.5     v5: 0.5 + 0 = 0.5    -> 0.5
HAND_TRANSE_ALL = [(1.0, 1), (0.5, 4), (0.5, 5), (0.0, 0), (0.0, 3), (-0.5, 2)]
HAND_TRANSE_TYPE1 = [(1.0, 1), (0.5, 5), (0.0, 3), (-0.5, 2)]
# DistMult: q = e0 * w0 = (0.25, 0); w = 0.25 * e_c[0]
#   v0: 0.125  v1: 0.25  v2: 0  v3: 0.25  v4: 0.25  v5: 0.125
HAND_DISTMULT_ALL = [(0.25, 1), (0.25, 3), (0.25, 4), (0.125, 0), (0.125, 5), (0.0, 2)]


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_hand_example(dtype):
    g = _hand_kg(dtype)
    out, n = oracle.tail_topk(g, [0], [0], 10)
    assert _pairs(out[0], n[0]) == HAND_TRANSE_ALL
    out, n = oracle.tail_topk(g, [0], [0], 10, cand_type=1)
    assert _pairs(out[0], n[0]) == HAND_TRANSE_TYPE1
    out, n = oracle.tail_topk(g, [0], [0], 3, cand_type=1)
    assert _pairs(out[0], n[0]) == HAND_TRANSE_TYPE1[:3]
    out, n = oracle.tail_topk(g, [0], [0], 10, fn="distmult")
    assert _pairs(out[0], n[0]) == HAND_DISTMULT_ALL
    # a type with no vertex: nothing to return
    out, n = oracle.tail_topk(g, [0], [0], 5, cand_type=7)
    assert n.tolist() == [0]


def test_gamma_shifts_every_score():
    g = _hand_kg()
    out, n = oracle.tail_topk(g, [0], [0], 10, gamma=2.5)
    assert _pairs(out[0], n[0]) == [(s + 1.5, v) for s, v in HAND_TRANSE_ALL]


def test_zero_vertex_embeddings_closed_form():
    # every vertex embedding zero: w(h, r, c) = gamma - |w_r|_1 for every c, so
    # the K best are the K smallest ids of the type, all with that score
    rng = np.random.default_rng(3)
    g = random_kg(rng, 40, 100, 3, 4, dyadic=True)
    g.vemb[:] = 0
    for r in range(3):
        want = 1.0 - float(np.abs(g.remb[r].astype(np.float64)).sum())
        ids = np.flatnonzero(g.vtypes == 2)
        out, n = oracle.tail_topk(g, [5], [r], 7, cand_type=2)
        assert _pairs(out[0], n[0]) == [(want, int(v)) for v in ids[:7]]
        out, n = oracle.tail_topk(g, [5], [r], 7, fn="distmult")
        assert _pairs(out[0], n[0]) == [(0.0, v) for v in range(7)]


@pytest.mark.parametrize("dtype,fn", [("f32", "transe"), ("bf16", "transe"), ("f32", "distmult"),
                                      ("bf16", "distmult")])
def test_selection_equals_full_sort(dtype, fn):
    # the edge weights come from oracle.edge_weights (pinned by hand examples
    # and by the exact rational value); the selection and the tie order come
    # from a NumPy lexicographic sort, independent of the oracle's heap.  The
    # bf16 grid (values in {-1, -3/4, ..., 1}) makes many scores tie exactly.
    rng = np.random.default_rng(11)
    g = random_kg(rng, 300, 900, 5, 6, dtype=dtype, dyadic=True)
    H = rng.integers(0, g.n, size=12).astype(np.uint32)
    Rq = rng.integers(0, g.R, size=12).astype(np.uint32)
    for cand_type in (-1, 0, 2):
        ids = np.arange(g.n) if cand_type < 0 else np.flatnonzero(g.vtypes == cand_type)
        out, n = oracle.tail_topk(g, H, Rq, 50, cand_type=cand_type, fn=fn)
        ties = 0
        for q in range(len(H)):
            w = oracle.edge_weights(g, np.full(ids.size, H[q]), np.full(ids.size, Rq[q]), ids, fn=fn)
            order = np.lexsort((ids, -w))
            want = [(float(w[i]), int(ids[i])) for i in order[:50]]
            assert _pairs(out[q], n[q]) == want
            ties += int(np.sum(np.diff(w[order[:50]]) == 0))
        assert ties > 0


def test_prefix_consistency_and_short_results():
    rng = np.random.default_rng(5)
    g = random_kg(rng, 120, 400, 4, 8)
    full, nf = oracle.tail_topk(g, [9, 17], [1, 3], 200, cand_type=1)
    n1 = int(np.sum(g.vtypes == 1))
    assert nf.tolist() == [n1, n1]
    for K in (1, 2, 7, 33, n1):
        part, npart = oracle.tail_topk(g, [9, 17], [1, 3], K, cand_type=1)
        for q in range(2):
            assert _pairs(part[q], npart[q]) == _pairs(full[q], nf[q])[:K]


def test_invalid_queries():
    g = _hand_kg()
    with pytest.raises(ValueError):
        oracle.tail_topk(g, [6], [0], 3)
    with pytest.raises(ValueError):
        oracle.tail_topk(g, [0], [1], 3)
    with pytest.raises(ValueError):
        oracle.tail_topk(g, [0], [0], 0)
