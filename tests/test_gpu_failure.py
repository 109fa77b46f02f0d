"""Failure handling without a GPU fault: an allocation failure made on the
host side.  A graph-memory cap (MHR_GRAPH_MEMORY_CAP_BYTES) below what a load
needs makes mhr_graph_load fail with MHR_ENOMEM part-way through its
allocations; the failed load must release everything it allocated (no leak
over repeated failures) and leave the library usable."""

import os

import numpy as np
import pytest

from tests._graphs import random_kg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mhr():
    import paper_2406_07727_gb300 as m
    return m


def test_memory_cap_fails_cleanly_and_leaks_nothing(mhr):
    import torch
    rng = np.random.default_rng(9)
    g = random_kg(rng, 20000, 400_000, 6, 64)
    # about 6 MB of CSR, 5 MB of embeddings: caps that stop the load at
    # different allocations
    torch.cuda.synchronize()
    G = mhr.load_kg(g)  # a first load warms the context and the allocator
    want, n_want = mhr.mhr_topk_paths_batched(G, np.array([1, 2], np.uint32), np.array([3, 4], np.uint32), 20)
    G.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    try:
        for cap in (1, 100_000, 2_000_000, 6_000_000, 9_000_000) * 3:
            os.environ["MHR_GRAPH_MEMORY_CAP_BYTES"] = str(cap)
            with pytest.raises(mhr.MhrError) as e:
                mhr.load_kg(g)
            assert e.value.status == mhr.MHR_ENOMEM
            assert "MHR_GRAPH_MEMORY_CAP_BYTES" in str(e.value)
    finally:
        os.environ.pop("MHR_GRAPH_MEMORY_CAP_BYTES", None)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < 4 * 1024 * 1024, (free0, free1)
    # a cap above the need does not get in the way; results are unchanged
    os.environ["MHR_GRAPH_MEMORY_CAP_BYTES"] = str(1 << 34)
    try:
        G = mhr.load_kg(g)
    finally:
        os.environ.pop("MHR_GRAPH_MEMORY_CAP_BYTES", None)
    got, n_got = mhr.mhr_topk_paths_batched(G, np.array([1, 2], np.uint32), np.array([3, 4], np.uint32), 20)
    G.close()
    assert np.array_equal(n_got, n_want)
    for q in range(2):
        assert got[q][: n_got[q]].tobytes() == want[q][: n_want[q]].tobytes()
