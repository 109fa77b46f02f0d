"""The generic H-hop beam-search oracle (Alg. 6 / Alg. 7) pinned to things
other than itself.

Pins: hand-derived examples in which the per-path beam does and does not cut
off the best path (values worked out in the comments), direct edges (H = 1) as
a closed form, an independent pure-Python depth-first enumeration of every
simple path when the beam is wide enough to keep everything, agreement of the
three-hop part with the pinned three-hop oracle, and path invariants (edges
exist, simple, the target only at the end, scores recompute) when the beam
does cut.
"""

import numpy as np
import pytest

import oracle
import synth
from tests._graphs import random_kg


def _kg(n, edges, vemb, remb):
    e = np.array(edges, dtype=np.int64)
    offsets, cols, rels = synth.canonicalize(n, len(remb), e[:, 0], e[:, 1], e[:, 2])
    return synth.KG(n=n, R=len(remb), n_types=1, offsets=offsets, cols=cols, rels=rels,
                    vtypes=np.zeros(n, dtype=np.uint8), vemb=np.array(vemb, dtype=np.float32),
                    remb=np.array(remb, dtype=np.float32), dtype="f32")


def _tuples(res):
    return [(float(p["score"]), int(p["hops"]), [int(x) for x in p["v"][: p["hops"] + 1]],
             [int(x) for x in p["r"][: p["hops"]]]) for p in res]


# DistMult with d = 1: w(u, r, v) = e_u * w_r * e_v, exact for these values.
# s = 0, a = 1, b = 2, t = 3; e = (1, 1, 0.5, 2); w_r = (1, 0, 2).
#   s -r0-> a: 1*1*1 = 1      s -r0-> b: 1*1*0.5 = 0.5
#   a -r1-> t: 1*0*2 = 0      b -r2-> t: 0.5*2*2 = 2
# Best path s-b-t scores 0.5 + 2 = 2.5; s-a-t scores 1 + 0 = 1.
# K = 1: level 0 keeps only a (1 > 0.5), so the beam finds s-a-t alone.
# K = 2: both survive level 0; results 2.5 (b) then 1.0 (a).
HAND_EDGES = [(0, 0, 1), (0, 0, 2), (1, 1, 3), (2, 2, 3)]
HAND_VEMB = [[1.0], [1.0], [0.5], [2.0]]
HAND_REMB = [[1.0], [0.0], [2.0]]


def test_hand_beam_cuts_the_best_path():
    g = _kg(4, HAND_EDGES, HAND_VEMB, HAND_REMB)
    assert _tuples(oracle.beam_paths(g, 0, 3, 3, 1, fn="distmult")) == [(1.0, 2, [0, 1, 3], [0, 1])]
    assert _tuples(oracle.beam_paths(g, 0, 3, 3, 2, fn="distmult")) == [
        (2.5, 2, [0, 2, 3], [0, 2]), (1.0, 2, [0, 1, 3], [0, 1])]
    # one hop: no direct edge s -> t, nothing found
    assert _tuples(oracle.beam_paths(g, 0, 3, 1, 5, fn="distmult")) == []


# A longer hand example, DistMult d = 1, one relation w_r = 1:
# s = 0, a = 1, b = 2, c = 3, t = 4; e = (1, 1, 0.5, 2, -1).
#   s-a 1    s-b 0.5    a-t -1    a-c 2    b-c 1    c-t -2
# K = 1: level 0 keeps a; level 1 from s-a: t gives 0 (result), c gives 3
#   (kept); level 2 from s-a-c: t gives 3 - 2 = 1 (result).  Best result: 1.
# K = 2: level 0 keeps a, b; level 1: s-a-t 0 (result), s-a-c 3, s-b-c 1.5;
#   level 2: s-a-c-t 1, s-b-c-t -0.5.  Results: 1 (a,c), 0 (a), -0.5 (b,c).
LONG_EDGES = [(0, 0, 1), (0, 0, 2), (1, 0, 4), (1, 0, 3), (2, 0, 3), (3, 0, 4)]
LONG_VEMB = [[1.0], [1.0], [0.5], [2.0], [-1.0]]


def test_hand_levels_and_mixed_hop_counts():
    g = _kg(5, LONG_EDGES, LONG_VEMB, [[1.0]])
    assert _tuples(oracle.beam_paths(g, 0, 4, 3, 1, fn="distmult")) == [(1.0, 3, [0, 1, 3, 4], [0, 0, 0])]
    assert _tuples(oracle.beam_paths(g, 0, 4, 3, 2, fn="distmult")) == [
        (1.0, 3, [0, 1, 3, 4], [0, 0, 0]), (0.0, 2, [0, 1, 4], [0, 0])]
    assert _tuples(oracle.beam_paths(g, 0, 4, 3, 10, fn="distmult")) == [
        (1.0, 3, [0, 1, 3, 4], [0, 0, 0]), (0.0, 2, [0, 1, 4], [0, 0]), (-0.5, 3, [0, 2, 3, 4], [0, 0, 0])]
    # two hops only: s-a-t
    assert _tuples(oracle.beam_paths(g, 0, 4, 2, 10, fn="distmult")) == [(0.0, 2, [0, 1, 4], [0, 0])]


def test_direct_edges_closed_form():
    # H = 1: the results are the direct edges s -> t, by weight, then relation
    rng = np.random.default_rng(4)
    g = random_kg(rng, 20, 300, 6, 4, dyadic=True)
    s = 3
    row = slice(g.offsets[s], g.offsets[s + 1])
    cols, rels = g.cols[row], g.rels[row]
    t = int(cols[0])
    mask = cols == t
    w = oracle.edge_weights(g, np.full(mask.sum(), s), rels[mask], cols[mask])
    want = sorted(((float(x), int(r)) for x, r in zip(w, rels[mask])), key=lambda p: (-p[0], p[1]))
    got = [(float(p["score"]), int(p["r"][0])) for p in oracle.beam_paths(g, s, t, 1, 50)]
    assert got == want


def _dfs_all_paths(g, s, t, H, fn):
    """Every simple s->t path of at most H hops whose inner vertices are not t,
    with the left-to-right sum of the (pinned) edge weights."""
    out = []

    def rec(path_v, path_r, score):
        x = path_v[-1]
        for e in range(int(g.offsets[x]), int(g.offsets[x + 1])):
            y, r = int(g.cols[e]), int(g.rels[e])
            if y in path_v:
                continue
            w = float(oracle.edge_weights(g, [x], [r], [y], fn=fn)[0])
            sc = score + w
            if y == t:
                out.append((sc, len(path_v), path_v + [y], path_r + [r]))
            elif len(path_v) < H:
                rec(path_v + [y], path_r + [r], sc)

    rec([s], [], 0.0)
    return out


def _result_key(p):
    score, hops, v, r = p
    seq = []
    for i in range(1, hops):
        seq += [v[i], r[i - 1]]
    seq.append(r[hops - 1])
    return (-score, hops, seq)


@pytest.mark.parametrize("fn,dtype", [("transe", "f32"), ("distmult", "f32"), ("transe", "bf16")])
def test_wide_beam_equals_full_enumeration(fn, dtype):
    rng = np.random.default_rng(7)
    for trial in range(12):
        g = random_kg(rng, 14, 60, 3, 4, dtype=dtype, dyadic=(trial % 2 == 0))
        s, t = [int(x) for x in rng.choice(g.n, size=2, replace=False)]
        H = 3 if trial % 3 else 4
        K = max(int(np.diff(g.offsets).max()), 1) + 1
        allp = sorted(_dfs_all_paths(g, s, t, H, fn), key=_result_key)
        # the per-path heaps keep every extension when K exceeds every out-degree
        got = _tuples(oracle.beam_paths(g, s, t, H, max(K, len(allp) + 1), fn=fn))
        assert got == allp, (trial, s, t)


def test_three_hop_part_matches_three_hop_oracle():
    rng = np.random.default_rng(9)
    for trial in range(8):
        g = random_kg(rng, 16, 90, 3, 4, dyadic=True)
        s, t = [int(x) for x in rng.choice(g.n, size=2, replace=False)]
        K = int(np.diff(g.offsets).max()) + 200
        res = _tuples(oracle.beam_paths(g, s, t, 3, K))
        three = [(sc, v[1], r[0], v[2], r[1], r[2]) for sc, h, v, r in res if h == 3]
        want = [(float(p["score"]), int(p["u"]), int(p["r1"]), int(p["v"]), int(p["r2"]), int(p["r3"]))
                for p in oracle.topk_paths(g, s, t, K)]
        assert three == want, trial


def test_narrow_beam_invariants():
    rng = np.random.default_rng(12)
    for trial in range(10):
        g = random_kg(rng, 40, 400, 4, 8, scale=0.4)
        s, t = [int(x) for x in rng.choice(g.n, size=2, replace=False)]
        for H, K in ((2, 3), (3, 4), (4, 3)):
            res = _tuples(oracle.beam_paths(g, s, t, H, K))
            assert len(res) <= K
            allp = {(tuple(v), tuple(r)): sc for sc, h, v, r in _dfs_all_paths(g, s, t, H, "transe")}
            for sc, h, v, r in res:
                assert 1 <= h <= H and v[0] == s and v[-1] == t
                assert len(set(v)) == len(v) and t not in v[:-1]
                assert allp[(tuple(v), tuple(r))] == sc      # exists, simple, same score
            assert res == sorted(res, key=_result_key)


def test_batch_matches_single():
    rng = np.random.default_rng(13)
    g = random_kg(rng, 60, 700, 4, 8, scale=0.4)
    S = rng.integers(0, g.n, size=9).astype(np.uint32)
    T = ((S + 1 + rng.integers(0, g.n - 1, size=9)) % g.n).astype(np.uint32)
    out, n_out = oracle.beam_paths_batch(g, S, T, 3, 5)
    for q in range(len(S)):
        assert _tuples(out[q][: n_out[q]]) == _tuples(oracle.beam_paths(g, int(S[q]), int(T[q]), 3, 5))


def test_invalid_arguments():
    g = _kg(4, HAND_EDGES, HAND_VEMB, HAND_REMB)
    for args in ((0, 0, 3, 2), (0, 9, 3, 2), (0, 3, 0, 2), (0, 3, 9, 2), (0, 3, 3, 0)):
        with pytest.raises(ValueError):
            oracle.beam_paths(g, *args)
    with pytest.raises(ValueError):   # K^(H-1) above the oracle's memory bound
        oracle.beam_paths(g, 0, 3, 8, 10)
