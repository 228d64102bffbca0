"""Degenerate and boundary cases of the solver through the C ABI, against the
oracle: a single node, an edgeless graph, one starting point, phases of zero
steps, a lift of three (Eq. 11 summed in order), complete graphs (closed-form
optimum), a graph near the shared-memory limit of the on-chip kernel, and the
bounded device waits giving up (failure detection without a GPU fault)."""
import numpy as np
import pytest

import graphgen as gg
from oracle import deco_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2509_18612_gb300 as deco  # noqa: E402

DEV = torch.device("cuda:0")


def _agree(a, b):
    return float(np.mean(np.asarray(a) == np.asarray(b)))


@pytest.mark.parametrize("n", [1, 2, 50])
def test_edgeless_graphs_cut_zero(n):
    g = gg.from_edges(n, [], [])
    for kern in (deco.DECO_KERNEL_GLOBAL, deco.DECO_KERNEL_AUTO):
        res, z, pc = deco.deco_solve(deco.graph_from(g), 8, [(1, 20, 0.01, 0.9), (2, 5, 0.001, 0.9)],
                                     deco.params(init=deco.DECO_INIT_IDI, kernel=kern), 3)
        assert res.best_cut == 0 and (pc == 0).all() and z.shape == (n,)


def test_one_starting_point_and_zero_step_phases():
    g = gg.er_graph(100, 0.1, 0)
    G = deco.graph_from(g)
    x0 = gg.uniform_x0(g.n, 1, 4)
    sched = [(1, 0, 0.01, 0.0), (1, 50, 0.01, 0.0), (2, 0, 0.001, 0.0)]
    res, z, pc = deco.deco_solve(G, 1, sched, deco.params(init=deco.DECO_INIT_EXPLICIT), 2, x0=x0)
    ref = O.solve(g, 1, [O.Phase(*s) for s in sched], O.Params(init="explicit"), 2, x0=x0)
    np.testing.assert_array_equal(pc, np.array(ref.phase_cuts))
    assert res.best_cut == ref.best_cut == O.cut_value(g, z)
    assert res.edge_updates == g.nnz * 50


@pytest.mark.parametrize("precision", [deco.DECO_PREC_FP32, deco.DECO_PREC_BF16])
def test_lift_three_rounding_order(precision):
    # l = 3: the row sum is accumulated in the order i = 0, 1, 2 on both sides
    g = gg.er_graph(200, 0.05, 7)
    B, l = 40, 3
    rng = np.random.default_rng(3)
    Y = rng.uniform(-1, 1, size=(g.n, B * l)).astype(np.float32)
    dt = torch.bfloat16 if precision == deco.DECO_PREC_BF16 else torch.float32
    y = torch.from_numpy(Y).to(DEV).to(dt)
    zbits = torch.zeros(g.n * 2, dtype=torch.int32, device=DEV)
    cuts = torch.zeros(B, dtype=torch.int64, device=DEV)
    deco.deco_round_cut(deco.graph_from(g), B, l, B * l, precision, y, zbits, cuts)
    torch.cuda.synchronize()
    Yq = y.float().cpu().numpy()
    # the device sums in FP32 in order; the FP64 oracle's sum decides every row
    # whose FP32 and FP64 sums have the same sign (all but exact-zero ties)
    s32 = (Yq[:, 0::3] + Yq[:, 1::3]) + Yq[:, 2::3]
    ref = O.cut_values(g, (s32 >= 0).astype(np.uint8))
    np.testing.assert_array_equal(cuts.cpu().numpy(), ref)
    assert _agree(ref, O.cut_values(g, O.binarize(Yq, l))) >= 0.99


@pytest.mark.parametrize("n", [6, 9, 14])
def test_complete_graph_reaches_the_closed_form(n):
    u, v = np.triu_indices(n, 1)
    g = gg.from_edges(n, u, v)
    res, z, _ = deco.deco_solve(deco.graph_from(g), 64, [(1, 300, 0.01, 0.9), (2, 100, 0.002, 0.9)],
                                deco.params(init=deco.DECO_INIT_IDI_HALF_UNIFORM), 1)
    assert res.best_cut == (n // 2) * ((n + 1) // 2) == O.cut_value(g, z)


@pytest.mark.parametrize("precision", [deco.DECO_PREC_FP32, deco.DECO_PREC_BF16])
def test_graph_near_the_shared_memory_limit_on_chip_equals_global(precision):
    # n = 1200 with a cluster of 8: the 150 KB replica of the column slab plus
    # the staging, momentum and CSR image of 150 own rows fill ~215 KB of the
    # ~226 KB of shared memory a CTA may use
    g = gg.er_graph(1200, 0.006, 9)
    G = deco.graph_from(g)
    cols = 64 if precision == deco.DECO_PREC_BF16 else 32
    C, ld = 2 * cols - 3, 2 * cols
    rng = np.random.default_rng(1)
    Y = np.zeros((g.n, ld), np.float32)
    Y[:, :C] = rng.uniform(-1e-3, 1e-3, size=(g.n, C))
    dt = torch.bfloat16 if precision == deco.DECO_PREC_BF16 else torch.float32
    outs = []
    for kern in (deco.DECO_KERNEL_GLOBAL, deco.DECO_KERNEL_ONCHIP | (8 << 8)):
        y = torch.from_numpy(Y).to(DEV).to(dt)
        v = torch.zeros(g.n, ld, device=DEV)
        a = deco.step_args(deco.DECO_OBJ_MULTILINEAR01, precision, 0.01, 0.9)
        deco.deco_run_phase(G, C, ld, y, v, 12, a, kern)
        torch.cuda.synchronize()
        outs.append((y, v))
    assert torch.equal(outs[0][0][:, :C], outs[1][0][:, :C]) and torch.equal(outs[0][1][:, :C], outs[1][1][:, :C])


@pytest.mark.parametrize("which", [0, 1, 2])
def test_bounded_wait_gives_up_and_the_context_stays_usable(which):
    """Failure detection without a GPU fault: one of the kernels' own bounded
    waits (dense mbarrier wait, dense grid barrier, on-chip exchange wait)
    runs on something nothing ever completes.  It must give up after its 2 s
    limit, report DECO_ERR_TIMEOUT through the error flag, and leave the
    context usable: a solve right after it matches the oracle."""
    status, ms = deco.deco_probe_wait_timeout(which)
    assert status == deco.DECO_ERR_TIMEOUT, deco.last_error()
    # the dense waits give up on the 2 s clock; the on-chip exchange wait on
    # the clock or on its iteration cap, whichever comes first
    assert (1900.0 if which < 2 else 1.0) <= ms <= 6000.0, ms
    assert "gave up" in deco.last_error()
    g = gg.er_graph(100, 0.1, 0)
    x0 = gg.uniform_x0(g.n, 16, 0)
    res, z, pc = deco.deco_solve(deco.graph_from(g), 16, [(1, 50, 0.01, 0.0)],
                                 deco.params(init=deco.DECO_INIT_EXPLICIT), 0, x0=x0)
    ref = O.solve(g, 16, [O.Phase(1, 50, 0.01, 0.0)], O.Params(init="explicit"), 0, x0=x0)
    assert res.best_cut == O.cut_value(g, z)
    assert _agree(pc[0], ref.phase_cuts[0]) >= 0.99


def test_injected_scratch_allocation_failures_leave_the_library_usable():
    """Host-side fault injection: the k-th scratch allocation of a solve fails
    with DECO_ERR_OOM (k = 1, 2, ... until the solve needs fewer); each failed
    call releases what it took, and the next call, on the same graph handle,
    gives the same result as before the failures."""
    g = gg.er_graph(100, 0.1, 0)
    G = deco.graph_from(g)
    x0 = gg.uniform_x0(g.n, 16, 1)
    sched = [(1, 30, 0.01, 0.9), (2, 10, 0.001, 0.9)]
    p = deco.params(init=deco.DECO_INIT_EXPLICIT)
    base, zb, pcb = deco.deco_solve(G, 16, sched, p, 0, x0=x0)
    failed = 0
    try:
        for k in range(1, 64):
            deco.deco_debug_fail_scratch_alloc(k)
            try:
                res, z, pc = deco.deco_solve(G, 16, sched, p, 0, x0=x0)
            except deco.DecoError as e:
                assert e.status == deco.DECO_ERR_OOM and "injected" in str(e), str(e)
                failed += 1
                deco.deco_debug_fail_scratch_alloc(0)
                res, z, pc = deco.deco_solve(G, 16, sched, p, 0, x0=x0)
                assert res.best_cut == base.best_cut and (pc == pcb).all() and (z == zb).all()
            else:
                assert res.best_cut == base.best_cut and (pc == pcb).all()
                break
    finally:
        deco.deco_debug_fail_scratch_alloc(0)
    assert failed >= 10, failed


@pytest.mark.parametrize("where", ["first", "middle", "last", "none"])
@pytest.mark.parametrize("family", ["er", "ba"])
def test_large_graph_symmetry_check_on_the_device(where, family):
    # graphs of unit weights with nnz >= 2^20 are checked for symmetry on the
    # device: a removed mirror entry is reported at the lowest offending row,
    # as the host check reports it on small graphs; a symmetric graph passes.
    # The BA graph's first rows are hubs of hundreds of entries (several
    # passes of a warp's lanes).
    g = gg.er_graph_avg_degree(120_000, 10, 6) if family == "er" else gg.ba_graph(140_000, 4, 6)
    rp, ci = g.row_ptr.astype(np.int32), g.col_idx.astype(np.int32)
    assert ci.size >= 1 << 20
    if where != "none":
        v = {"first": 0, "middle": g.n // 2, "last": g.n - 1}[where]
        while rp[v + 1] == rp[v]:
            v += 1
        e = rp[v + 1] - 1                              # drop the last entry (v, u) of row v
        u = int(ci[e])
        ci = np.delete(ci, e)
        rp = rp.copy()
        rp[v + 1:] -= 1
        # (u, v) is now the one entry without a mirror: row u is the offending row
        with pytest.raises(deco.DecoError) as ei:
            deco.deco_create_graph(g.n, rp, ci, None)
        assert ei.value.status == deco.DECO_ERR_GRAPH
        assert f"({u},{v}) stored but ({v},{u}) missing" in deco.last_error(), deco.last_error()
    else:
        G = deco.deco_create_graph(g.n, rp, ci, None)
        G.close()


def test_smem_probe_rate_is_plausible():
    # the shared-memory load path of all SMs: below the 152 SMs x 128 B/clk
    # x 2.07 GHz the hardware can deliver at most (plus a margin for the
    # clock), and well above a tenth of it
    derived = 152 * 128 * 2.07e9 / 1e9
    for width in (8, 16):
        gbs = deco.deco_probe_smem_rate(width, 1 << 14)
        assert 0.1 * derived < gbs < 1.1 * derived, (width, gbs)
