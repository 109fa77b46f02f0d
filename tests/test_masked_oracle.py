"""The constrained three-hop oracle (relation per hop, vertex type of u and v;
the query shape of Sec. 3.1) pinned to things other than itself.

Pins: with every relation and type allowed it equals the (pinned)
unconstrained oracle bit for bit; with random constraints it equals the
unconstrained full enumeration (K = every path) filtered in NumPy and cut at
K; a hand-checked case on the golden 10-vertex graph.
"""

import numpy as np
import pytest

import oracle
from tests._graphs import kg_from_golden, load_golden, path_tuples, random_kg


def _filter(g, paths, rel1, rel2, rel3, types_u, types_v, K):
    keep = []
    for p in paths:
        if rel1 is not None and int(p["r1"]) not in rel1:
            continue
        if rel2 is not None and int(p["r2"]) not in rel2:
            continue
        if rel3 is not None and int(p["r3"]) not in rel3:
            continue
        if types_u is not None and int(g.vtypes[p["u"]]) not in types_u:
            continue
        if types_v is not None and int(g.vtypes[p["v"]]) not in types_v:
            continue
        keep.append(p)
    return path_tuples(keep)[:K]


@pytest.mark.parametrize("fn", ["transe", "distmult"])
def test_no_constraint_equals_unconstrained(fn):
    rng = np.random.default_rng(21)
    g = random_kg(rng, 60, 900, 5, 8, scale=0.4)
    for s, t in rng.integers(0, g.n, size=(10, 2)):
        if s == t:
            continue
        a = oracle.topk_paths(g, int(s), int(t), 40, fn=fn)
        b = oracle.topk_paths_masked(g, int(s), int(t), 40, fn=fn)
        assert path_tuples(a) == path_tuples(b)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_random_constraints_equal_filtered_enumeration(dtype):
    rng = np.random.default_rng(22)
    g = random_kg(rng, 50, 1200, 6, 6, dtype=dtype, dyadic=True)
    checked = 0
    for trial in range(40):
        s, t = [int(x) for x in rng.choice(g.n, size=2, replace=False)]
        full = oracle.topk_paths(g, s, t, 100000)
        sets = [None if rng.random() < 0.3 else set(rng.choice(g.R, size=3, replace=False).tolist())
                for _ in range(3)]
        types = [None if rng.random() < 0.3 else {int(rng.integers(0, 3))} for _ in range(2)]
        K = int(rng.integers(1, 30))
        want = _filter(g, full, *sets, *types, K)
        got = path_tuples(oracle.topk_paths_masked(g, s, t, K, rel1=sets[0], rel2=sets[1], rel3=sets[2],
                                                   types_u=types[0], types_v=types[1]))
        assert got == want, trial
        checked += len(want)
    assert checked > 50


def test_golden_graph_relation_constraint():
    gj = load_golden()
    g = kg_from_golden(gj)
    s, t = gj["query"]["s"], gj["query"]["t"]
    full = oracle.topk_paths(g, s, t, 100)
    # only the middle relation 0: the paths of the full list with r2 == 0, in order
    got = path_tuples(oracle.topk_paths_masked(g, s, t, 100, rel2=[0]))
    assert got == [p for p in path_tuples(full) if p[4] == 0]
    assert 0 < len(got) < len(full)
    # an empty relation set admits nothing
    assert len(oracle.topk_paths_masked(g, s, t, 100, rel1=[])) == 0
