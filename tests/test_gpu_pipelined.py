"""The pipelined form of the per-step kernel (DECO_KERNEL_PIPELINED): rows in
degree-sorted slices, each warp's items one stream of records, every
neighbour row staged in shared memory by cp.async ahead of its use.  It performs the same FP32 operations in the same order as
the lane-group form of DECO_KERNEL_GLOBAL, so every iterate and momentum
value must be bit-identical to it -- on graphs with hubs (rows split into
several parts), +-1 and general integral weights, isolated nodes, ragged and
wide column counts (several column chunks), per-column step sizes and step
budgets, both objectives, with and without momentum, every stage shape and
with column slabs; in the form with the shape read from the arguments, the
forms with 8 or 12 entries per item fixed at compile time, and the wide form
(two 16-byte vectors per lane).  The lane-group form itself is checked
against the FP64 oracle step by step in test_gpu_parity.py.
"""
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
OBJ = {O.OBJ_MULTILINEAR01: deco.DECO_OBJ_MULTILINEAR01, O.OBJ_LAPLACIAN: deco.DECO_OBJ_LAPLACIAN}
PIPE = deco.DECO_KERNEL_GLOBAL | deco.DECO_KERNEL_PIPELINED
FIX8 = PIPE | deco.DECO_KERNEL_PIPE_ENTRIES(1) | deco.DECO_KERNEL_PIPE_STAGES(1)    # 8 entries, 2 stages
FIX12 = PIPE | deco.DECO_KERNEL_PIPE_ENTRIES(3) | deco.DECO_KERNEL_PIPE_STAGES(1)   # 12 entries, 2 stages
WIDE = deco.DECO_KERNEL_PIPE_WIDE
FORMS = {"runtime": PIPE, "fixed8": FIX8, "fixed12": FIX12, "wide8": FIX8 | WIDE, "wide12": FIX12 | WIDE}


def _signed(n, p, seed, choices):
    g = gg.er_graph(n, p, seed)
    rng = np.random.default_rng(seed + 5)
    u, v, _ = g.edges()
    return gg.from_edges(n, u, v, rng.choice(np.array(choices), size=u.size))


def _hubs():
    # a few nodes joined to most others (degrees 100-300: rows of many parts)
    # on top of a sparse ER graph
    base = gg.er_graph(600, 0.01, 8)
    u, v, _ = base.edges()
    rng = np.random.default_rng(9)
    us, vs = list(u), list(v)
    for h, deg in ((0, 300), (1, 170), (2, 100), (3, 33)):
        for x in rng.choice(np.arange(4, 600), size=deg, replace=False):
            us.append(h)
            vs.append(int(x))
    e = {(min(a, b), max(a, b)) for a, b in zip(us, vs) if a != b}
    a, b = zip(*sorted(e))
    return gg.from_edges(600, a, b)


GRAPHS = {
    "er800": lambda: gg.er_graph(800, 0.06, 1),
    "torus": lambda: gg.torus_graph(40, 20, 2),                 # +-1 weights
    "ba": lambda: gg.ba_graph(700, 4, 3),                       # hubs of degree > 32
    "signed": lambda: _signed(300, 0.05, 4, (-2.0, -1.0, 1.0, 3.0)),
    "isolated": lambda: gg.from_edges(50, [0, 1, 2], [1, 2, 3]),
    "hubs": _hubs,
    "er_sparse": lambda: gg.er_graph_avg_degree(5000, 10, 11),  # the large workload's family
}


def _blocks(g, C, ld, precision, seed, mu):
    rng = np.random.default_rng(seed)
    Y = np.zeros((g.n, ld), np.float32)
    Y[:, :C] = rng.uniform(-1, 1, size=(g.n, C)) * np.where(rng.random(C) < 0.5, 1.0, 1e-3)
    Y[:, C:] = 7.0                                   # padding columns: must stay untouched
    dt = torch.bfloat16 if precision == deco.DECO_PREC_BF16 else torch.float32
    y = torch.from_numpy(Y).to(DEV).to(dt)
    v = None
    if mu:
        V = np.zeros((g.n, ld), np.float32)
        V[:, :C] = rng.normal(size=(g.n, C)) * 0.1
        v = torch.from_numpy(V).to(DEV)
    return y, v


def _phase(G, y, v, C, ld, steps, objective, precision, alpha, mu, kernel, alpha_cols=None, steps_cols=None):
    y = y.clone()
    v = None if v is None else v.clone()
    flag = torch.zeros(1, dtype=torch.int32, device=DEV)
    a = deco.step_args(OBJ[objective], precision, alpha, mu, alpha_cols, steps_cols)
    deco.deco_run_phase(G, C, ld, y, v, steps, a, kernel, flag)
    torch.cuda.synchronize()
    return y, v, int(flag.item())


def _same(ref, got, y0, C):
    assert ref[2] == got[2] == 0
    assert torch.equal(got[0][:, :C], ref[0][:, :C])
    assert torch.equal(got[0][:, C:], y0[:, C:])
    if ref[1] is not None:
        assert torch.equal(got[1][:, :C], ref[1][:, :C])


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("precision", [deco.DECO_PREC_FP32, deco.DECO_PREC_BF16])
@pytest.mark.parametrize("C,ld", [(128, 128), (203, 256), (24, 64), (520, 576)])
def test_pipelined_step_bitwise_equals_lane_groups(form, name, precision, C, ld):
    # (520 columns: several column chunks; 203: a ragged chunk whose second
    # vectors in the wide form lie partly or wholly past C)
    g = GRAPHS[name]()
    G = deco.graph_from(g)
    objective = O.OBJ_LAPLACIAN if name in ("signed", "torus") else O.OBJ_MULTILINEAR01
    mu = 0.9 if C != 128 else 0.0
    y, v = _blocks(g, C, ld, precision, 3, mu)
    for steps in (3, 4):                              # odd / even: the result in either buffer
        ref = _phase(G, y, v, C, ld, steps, objective, precision, 0.01, mu, deco.DECO_KERNEL_GLOBAL)
        got = _phase(G, y, v, C, ld, steps, objective, precision, 0.01, mu, FORMS[form])
        _same(ref, got, y, C)


@pytest.mark.parametrize("entries", [0, 1, 2, 3])
@pytest.mark.parametrize("stages", [0, 1, 2, 3])
@pytest.mark.parametrize("warps", [0, 1, 3])
@pytest.mark.parametrize("wide", [False, True])
def test_pipelined_shapes_bitwise(entries, stages, warps, wide):
    # every entries-per-item / stage-count / block shape on the graph with
    # rows of up to 300 entries (up to 38 parts of 8); stage code 3 is not
    # defined and is refused, and the wide form runs only with 8 or 12
    # entries in 2 stages
    fixed = stages == 1 and entries in (1, 3)
    if wide and stages != 3 and not fixed:
        with pytest.raises(deco.DecoError):
            deco.deco_run_phase(deco.graph_from(GRAPHS["er800"]()), 64, 64, torch.zeros(800, 64, device=DEV), None,
                                1, deco.step_args(), PIPE | WIDE | deco.DECO_KERNEL_PIPE_ENTRIES(entries)
                                | deco.DECO_KERNEL_PIPE_STAGES(stages))
        return
    if stages == 3:
        with pytest.raises(deco.DecoError):
            deco.deco_run_phase(deco.graph_from(GRAPHS["er800"]()), 64, 64, torch.zeros(800, 64, device=DEV), None,
                                1, deco.step_args(), PIPE | deco.DECO_KERNEL_PIPE_ENTRIES(entries)
                                | deco.DECO_KERNEL_PIPE_STAGES(stages))
        return
    g = GRAPHS["hubs"]()
    G = deco.graph_from(g)
    C, ld = 128, 128
    kern = (PIPE | deco.DECO_KERNEL_PIPE_ENTRIES(entries) | deco.DECO_KERNEL_PIPE_STAGES(stages)
            | deco.DECO_KERNEL_PIPE_WARPS(warps) | (WIDE if wide else 0))
    for precision in (deco.DECO_PREC_FP32, deco.DECO_PREC_BF16):
        y, v = _blocks(g, C, ld, precision, 4, 0.9)
        ref = _phase(G, y, v, C, ld, 5, O.OBJ_MULTILINEAR01, precision, 0.01, 0.9, deco.DECO_KERNEL_GLOBAL)
        got = _phase(G, y, v, C, ld, 5, O.OBJ_MULTILINEAR01, precision, 0.01, 0.9, kern)
        _same(ref, got, y, C)


@pytest.mark.parametrize("name", ["er800", "signed", "ba", "hubs"])
@pytest.mark.parametrize("precision", [deco.DECO_PREC_FP32, deco.DECO_PREC_BF16])
@pytest.mark.parametrize("s", [1, 2])
@pytest.mark.parametrize("form", ["runtime", "runtime_hints", "fixed8", "fixed8_hints", "wide8", "wide12_hints"])
@pytest.mark.parametrize("C,ld", [(200, 256), (128, 128)])
def test_pipelined_column_slabs_with_budgets_bitwise(name, precision, s, form, C, ld):
    # column slabs, per-column step sizes and budgets; with and without the L2
    # eviction priorities (a cache hint changes no value).  200 columns: a
    # ragged last slab; 128 columns in 4 slabs: two lanes per row in the wide
    # form
    g = GRAPHS[name]()
    G = deco.graph_from(g)
    objective = O.OBJ_LAPLACIAN if name == "signed" else O.OBJ_MULTILINEAR01
    y, v = _blocks(g, C, ld, precision, 4, 0.9)
    steps_cols = torch.from_numpy(np.random.default_rng(5).integers(0, 9, C).astype(np.int32)).to(DEV)
    alpha_cols = torch.from_numpy(np.random.default_rng(6).uniform(1e-3, 2e-2, C).astype(np.float32)).to(DEV)
    for steps in (7, 8):
        ref = _phase(G, y, v, C, ld, steps, objective, precision, 0.0, 0.9, deco.DECO_KERNEL_GLOBAL,
                     alpha_cols, steps_cols)
        got = _phase(G, y, v, C, ld, steps, objective, precision, 0.0, 0.9,
                     FORMS[form.replace("_hints", "")] | deco.DECO_KERNEL_COLUMN_SLABS(s)
                     | (deco.DECO_KERNEL_PIPE_L2_HINTS if form.endswith("_hints") else 0),
                     alpha_cols, steps_cols)
        _same(ref, got, y, C)


def test_pipelined_nonfinite_flag_and_single_node():
    # a non-finite start is flagged as by the lane-group form; a graph of one
    # isolated node takes a step of its own row only
    g = GRAPHS["er800"]()
    G = deco.graph_from(g)
    C = ld = 64
    y, _ = _blocks(g, C, ld, deco.DECO_PREC_FP32, 1, 0.0)
    y[5, 3] = float("inf")
    for kern in FORMS.values():
        _, _, flag = _phase(G, y, None, C, ld, 1, O.OBJ_MULTILINEAR01, deco.DECO_PREC_FP32, 0.01, 0.0, kern)
        assert flag & 1
    one = deco.graph_from(gg.from_edges(1, [], []))
    y1 = torch.full((1, 64), 0.5, device=DEV)
    got = _phase(one, y1, None, 64, 64, 3, O.OBJ_MULTILINEAR01, deco.DECO_PREC_FP32, 0.01, 0.0, PIPE)
    assert got[2] == 0 and torch.equal(got[0], y1)   # no neighbours: the multilinear gradient is 0


def test_pipelined_solve_equals_lane_group_solve():
    g = GRAPHS["er_sparse"]()
    G = deco.graph_from(g)
    sched = [(1, 60, 0.01, 0.9), (2, 20, 0.001, 0.9)]
    out = []
    for kern in (deco.DECO_KERNEL_GLOBAL, PIPE, PIPE | deco.DECO_KERNEL_COLUMN_SLABS(1), FIX8 | WIDE):
        for prec in (deco.DECO_PREC_FP32, deco.DECO_PREC_BF16):
            res, z, pc = deco.deco_solve(G, 64, sched, deco.params(init=deco.DECO_INIT_IDI, precision=prec,
                                                                    kernel=kern), 3)
            out.append((prec, res.best_cut, res.best_init, res.best_phase, z.tobytes(), pc.tobytes()))
    for prec in (deco.DECO_PREC_FP32, deco.DECO_PREC_BF16):
        runs = [o[1:] for o in out if o[0] == prec]
        assert runs[0] == runs[1] == runs[2] == runs[3]


@pytest.mark.parametrize("name", ["er800", "ba", "hubs", "isolated", "er_sparse"])
@pytest.mark.parametrize("C,ld", [(128, 128), (203, 256), (24, 64)])
@pytest.mark.parametrize("form", ["runtime", "fixed8", "fixed12", "wide8", "wide12"])
def test_pipelined_mixed_precision_add_bitwise(name, C, ld, form):
    # BF16 sums of unit-weight rows with the mixed-precision add instruction:
    # the same value as widening the BF16 operand and adding in FP32
    g = GRAPHS[name]()
    G = deco.graph_from(g)
    y, v = _blocks(g, C, ld, deco.DECO_PREC_BF16, 6, 0.9)
    ref = _phase(G, y, v, C, ld, 5, O.OBJ_MULTILINEAR01, deco.DECO_PREC_BF16, 0.01, 0.9, deco.DECO_KERNEL_GLOBAL)
    got = _phase(G, y, v, C, ld, 5, O.OBJ_MULTILINEAR01, deco.DECO_PREC_BF16, 0.01, 0.9,
                 FORMS[form] | deco.DECO_KERNEL_PIPE_MIXED_ADD)
    _same(ref, got, y, C)


