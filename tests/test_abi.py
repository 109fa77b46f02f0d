"""The C ABI library builds, loads and exports every symbol the header
declares (CPU only: no call here reaches the GPU)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mhr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mhr_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("mhr_graph_load", "mhr_graph_free", "mhr_edge_scores", "mhr_topk_paths",
                 "mhr_topk_paths_batched", "mhr_tail_topk", "mhr_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2406_07727_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_abi():
    import paper_2406_07727_gb300 as m
    for n in declared_functions():
        assert hasattr(m, n), n


def test_struct_layouts():
    import paper_2406_07727_gb300 as m
    from paper_2406_07727_gb300 import _mhr
    assert m.PATH_DTYPE.itemsize == 24
    assert m.TAIL_DTYPE.itemsize == 16
    assert ctypes.sizeof(_mhr.GraphDesc) == 104
    assert ctypes.sizeof(_mhr.QueryOpts) == 48
    assert ctypes.sizeof(_mhr.Constraints) == 40
    assert ctypes.sizeof(_mhr.GraphInfo) == 80
    assert ctypes.sizeof(_mhr.Stats) == 88


def test_host_side_argument_checks():
    """Checks that return before any CUDA call."""
    import paper_2406_07727_gb300 as m
    from paper_2406_07727_gb300 import _mhr
    lib = m.load_library()
    h = ctypes.c_void_p()
    assert lib.mhr_graph_load(None, ctypes.byref(h), None) == m.MHR_EINVAL
    assert "NULL" in m.mhr_last_error()
    d = _mhr.GraphDesc()
    d.n_vertices = 0
    assert lib.mhr_graph_load(ctypes.byref(d), ctypes.byref(h), None) == m.MHR_EINVAL
    d.n_vertices, d.n_edges, d.n_relations, d.dim = 10, 5, 0, 4
    assert lib.mhr_graph_load(ctypes.byref(d), ctypes.byref(h), None) == m.MHR_EINVAL
    assert "n_relations" in m.mhr_last_error()
    assert h.value is None
    assert lib.mhr_tail_topk(None, 1, None, None, -1, 5, None, None, 0, None, None) == m.MHR_EINVAL
    assert "NULL" in m.mhr_last_error()
    assert m.mhr_version().startswith("mhr-gb300")
