"""deco_run_phase_noalloc: the phase runner for callers that cannot let the
library allocate device memory (their own pool holds the device, or the
latency of an allocation is not acceptable).  Its scratch block lives in a
fixed array inside the library.  It runs the same step kernel as the
allocating deco_run_phase with DECO_KERNEL_GLOBAL, so its results must be
bit-identical to that call's, call after call -- a tolerance could hide stale
scratch contents or a wrong ping-pong parity leaking into a result column.
Nothing may be taken from the stream-ordered pool while it runs, and a
scratch allocation armed to fail must not be reached.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

import graphgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2509_18612_gb300 as deco  # noqa: E402

DEV = torch.device("cuda:0")


def _block(g, C, ld, seed, dtype):
    rng = np.random.default_rng(seed)
    Y = np.zeros((g.n, ld), np.float32)
    Y[:, :C] = rng.uniform(-1, 1, size=(g.n, C)) * np.where(rng.random(C) < 0.5, 1.0, 1e-3)
    V = np.zeros((g.n, ld), np.float32)
    V[:, :C] = rng.normal(size=(g.n, C)) * 0.1
    return torch.from_numpy(Y).to(DEV).to(dtype), torch.from_numpy(V).to(DEV)


@pytest.mark.parametrize("precision", [deco.DECO_PREC_FP32, deco.DECO_PREC_BF16])
def test_noalloc_phase_matches_allocating_phase_twice(precision):
    g = gg.er_graph(800, 0.06, 1)
    G = deco.graph_from(g)
    C, ld = 203, 208                      # ragged column count
    dtype = torch.bfloat16 if precision == deco.DECO_PREC_BF16 else torch.float32
    a = deco.step_args(deco.DECO_OBJ_MULTILINEAR01, precision, 0.01, 0.9)
    for call, (seed, steps) in enumerate([(1, 7), (2, 10)]):   # odd: result lands in the scratch; even: in y
        y0, v0 = _block(g, C, ld, seed, dtype)
        y_ref, v_ref = y0.clone(), v0.clone()
        deco.deco_run_phase(G, C, ld, y_ref, v_ref, steps, a, deco.DECO_KERNEL_GLOBAL)
        y, v = y0.clone(), v0.clone()
        flag = torch.zeros(1, dtype=torch.int32, device=DEV)
        torch.cuda.synchronize()
        deco.deco_debug_pool_usage(reset=True)
        used_before, _ = deco.deco_debug_pool_usage()
        deco.deco_debug_fail_scratch_alloc(1)     # the first scratch allocation would fail
        try:
            deco.deco_run_phase_noalloc(G, C, ld, y, v, steps, a, flag)
            torch.cuda.synchronize()
        finally:
            deco.deco_debug_fail_scratch_alloc(0)
        _, used_high = deco.deco_debug_pool_usage()
        assert used_high == used_before, (call, used_before, used_high)
        assert int(flag.item()) == 0, call
        assert torch.equal(y[:, :C], y_ref[:, :C]), call
        assert torch.equal(v[:, :C], v_ref[:, :C]), call
        # columns >= C of the caller's block are never written
        assert torch.equal(y[:, C:], y0[:, C:]), call


def test_noalloc_phase_refuses_blocks_beyond_its_scratch():
    g = gg.er_graph(20000, 0.0005, 3)
    G = deco.graph_from(g)
    C = ld = 256                          # 20000 x 256 x 4 B = 20.5 MB > 16 MiB
    y = torch.zeros(g.n, ld, device=DEV)
    a = deco.step_args(deco.DECO_OBJ_MULTILINEAR01, deco.DECO_PREC_FP32, 0.01, 0.0)
    with pytest.raises(deco.DecoError) as ei:
        deco.deco_run_phase_noalloc(G, C, ld, y, None, 3, a)
    assert ei.value.status == deco.DECO_ERR_UNSUPPORTED
    assert "16777216" in str(ei.value)
