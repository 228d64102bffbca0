"""C-ABI checks that need no GPU: the library loads, exports every function
include/deco.h declares, and rejects malformed input before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

import graphgen as gg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def deco():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_18612_gb300 as d
    return d


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(deco_\w+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(deco):
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(deco.lib, name), name
    assert declared == set(deco.EXPORTED)
    assert deco.deco_abi_version() == 2
    assert ctypes.sizeof(deco.deco_params) == 12 * 4   # the struct of include/deco.h


def _csr(n, rows):
    rp = [0]
    ci = []
    for r in rows:
        ci += r
        rp.append(len(ci))
    return n, np.array(rp, np.int32), np.array(ci, np.int32)


@pytest.mark.parametrize("case,status", [
    ("rowptr0", -2), ("decreasing", -2), ("range", -2), ("selfloop", -2), ("unsorted", -2),
    ("duplicate", -2), ("asym", -2), ("asymw", -2), ("fracw", -7), ("zerow", -7), ("nnz", -2),
])
def test_validation_errors(deco, case, status):
    n, rp, ci = _csr(3, [[1, 2], [0], [0]])
    w = None
    if case == "rowptr0":
        rp = rp.copy(); rp[0] = 1
    elif case == "decreasing":
        rp = np.array([0, 2, 1, 3], np.int32); ci = np.array([1, 2, 0], np.int32)
    elif case == "range":
        ci = ci.copy(); ci[1] = 7
    elif case == "selfloop":
        n, rp, ci = _csr(3, [[0, 1], [0], []])
    elif case == "unsorted":
        n, rp, ci = _csr(3, [[2, 1], [0], [0]])
    elif case == "duplicate":
        n, rp, ci = _csr(3, [[1, 1], [0], []])
    elif case == "asym":
        n, rp, ci = _csr(3, [[1, 2], [0], []])
    elif case == "asymw":
        w = np.array([1, 2, 1, 1], np.float32)
    elif case == "fracw":
        w = np.array([0.5, 1, 0.5, 1], np.float32)
    elif case == "zerow":
        w = np.array([0, 1, 0, 1], np.float32)
    elif case == "nnz":
        ci = np.concatenate([ci, ci])
    with pytest.raises(deco.DecoError) as ei:
        deco.deco_create_graph(n, rp, ci, w)
    assert ei.value.status == status, deco.last_error()
    assert deco.last_error()


def test_null_and_size_arguments(deco):
    import ctypes
    h = ctypes.c_void_p()
    assert deco.lib.deco_create_graph(0, 0, None, None, None, 0, ctypes.byref(h)) == deco.DECO_ERR_ARG
    assert deco.lib.deco_create_graph(3, 4, None, None, None, 0, ctypes.byref(h)) == deco.DECO_ERR_ARG
    assert deco.lib.deco_create_graph(3, 4, None, None, None, 0, None) == deco.DECO_ERR_ARG
    res = deco.deco_result()
    assert deco.lib.deco_solve(None, 4, None, 1, None, 0, None, None, None, None, None,
                               ctypes.byref(res)) == deco.DECO_ERR_ARG
    args = deco.step_args()
    assert deco.lib.deco_step(None, 8, 8, None, None, None, ctypes.byref(args), None, None) == deco.DECO_ERR_ARG
    assert deco.lib.deco_eval_cut(None, None, None) == deco.DECO_ERR_ARG
    n = ctypes.c_int32()
    assert deco.lib.deco_graph_info(None, ctypes.byref(n), None, None) == deco.DECO_ERR_ARG


def test_valid_graph_without_gpu_reports_cuda_error(deco):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    g = gg.er_graph(30, 0.2, 0)
    with pytest.raises(deco.DecoError) as ei:
        deco.graph_from(g)
    assert ei.value.status in (deco.DECO_ERR_CUDA, deco.DECO_ERR_OOM)


def test_fault_injection_hook_arguments(deco):
    with pytest.raises(deco.DecoError) as ei:
        deco.deco_debug_fail_scratch_alloc(-1)
    assert ei.value.status == deco.DECO_ERR_ARG
    deco.deco_debug_fail_scratch_alloc(0)


def test_threaded_validation_reports_the_lowest_offending_row(deco):
    # a graph large enough that the host checks run on several threads
    # (2 M entries): two planted errors in different threads' row ranges; the
    # message must name the lower row, as a single pass would
    g = gg.er_graph_avg_degree(200_000, 10, 21)
    rp, ci = g.row_ptr.astype(np.int32), g.col_idx.astype(np.int32).copy()
    lo_row, hi_row = 30_001, 170_003
    for v in (lo_row, hi_row):
        assert rp[v + 1] > rp[v]
    ci[rp[hi_row]] = hi_row                     # self loop in a late row
    ci[rp[lo_row + 1] - 1] = g.n + 5            # out-of-range index in an earlier row
    with pytest.raises(deco.DecoError) as ei:
        deco.deco_create_graph(g.n, rp, ci, None)
    assert ei.value.status == deco.DECO_ERR_GRAPH
    assert f"(row {lo_row})" in deco.last_error(), deco.last_error()
    # weighted symmetry (checked on the host): asymmetric weights planted in two rows
    ci = g.col_idx.astype(np.int32)
    w = np.ones(ci.size, np.float32)
    for v in (hi_row, lo_row):
        e = rp[v]
        u = int(ci[e])
        w[e] = 2.0                                 # (v, u) weighs 2, its mirror (u, v) 1
        w[rp[u]:rp[u + 1]][ci[rp[u]:rp[u + 1]] == v] = 1.0
    first = min(min(hi_row, int(ci[rp[hi_row]])), min(lo_row, int(ci[rp[lo_row]])))
    with pytest.raises(deco.DecoError) as ei:
        deco.deco_create_graph(g.n, rp, ci, w)
    assert ei.value.status == deco.DECO_ERR_GRAPH
    assert f"asymmetric weights on edge ({first}," in deco.last_error(), deco.last_error()


def test_smem_probe_rejects_bad_arguments(deco):
    import ctypes
    gbs = ctypes.c_float()
    for width, iters in ((4, 64), (16, 0), (16, 12), (8, (1 << 24) + 8)):
        assert deco.lib.deco_probe_smem_rate(width, iters, ctypes.byref(gbs), None) == deco.DECO_ERR_ARG
    assert deco.lib.deco_probe_smem_rate(16, 64, None, None) == deco.DECO_ERR_ARG
