"""Host-side marshalling of query options and constraints into the C structs
(no library call, no GPU)."""

import ctypes

import numpy as np
import pytest

from paper_2406_07727_gb300 import _mhr


def flags(ptr, n):
    return np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctypes.c_uint8)), shape=(n,)).copy()


def test_options_fill_the_struct():
    assert _mhr._opts(None) is None
    o = _mhr._opts({"chunk": 8192, "tile": 8, "prune": 1, "order": 2, "precision": -1, "part_count": 3,
                    "part_index": 2})
    assert (o.chunk, o.tile, o.prune, o.order, o.precision, o.part_count, o.part_index) == (8192, 8, 1, 2, -1, 3, 2)
    assert not o.mlp and not o.constraints and o.reserved == 0
    assert _mhr._opts(o) is o
    assert ctypes.sizeof(_mhr.QueryOpts) == 48


@pytest.mark.parametrize("bad", [{"prun": 1}, {"chunk_size": 4096}, {"reserved": 1}])
def test_unknown_option_is_rejected(bad):
    with pytest.raises(ValueError, match="unknown query option"):
        _mhr._opts(bad)


def test_constraints_become_flag_arrays():
    o = _mhr._opts({"constraints": {"rel1": [0, 2], "rel3": [], "types_u": [1, 255]}}, n_relations=3)
    c = o.constraints.contents
    assert flags(c.rel1, 3).tolist() == [1, 0, 1]
    assert c.rel2 is None                                  # missing entry: every relation allowed
    assert flags(c.rel3, 3).tolist() == [0, 0, 0]          # empty set: no relation allowed
    tu = flags(c.types_u, 256)
    assert tu[1] == 1 and tu[255] == 1 and tu.sum() == 2
    assert c.types_v is None
    assert ctypes.sizeof(_mhr.Constraints) == 40


@pytest.mark.parametrize("bad,msg", [({"rel1": [3]}, "relation id outside"), ({"rel2": [-1]}, "relation id outside"),
                                     ({"types_v": [256]}, "vertex type outside"),
                                     ({"rel4": [0]}, "unknown constraint")])
def test_bad_constraints_are_rejected(bad, msg):
    with pytest.raises(ValueError, match=msg):
        _mhr._constraints(bad, 3)
