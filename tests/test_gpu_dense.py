"""Parity of the dense tensor-core kernel (DECO_KERNEL_DENSE) with the global
kernel and with the CPU oracle.

Tolerances
  * one step from a dyadic block (every y a multiple of 2^-6, |y| <= 1, integral
    weights): every partial sum of A Y is exact in FP32 whatever the summation
    order, so the dense kernel's step equals the global kernel's bit for bit
    (same fused FP32 update, same BF16 rounding).
  * steps from arbitrary BF16 blocks, against the FP64 oracle: the tensor
    cores sum row i of A Y in their own order, so
        |y_gpu - y_ref| <= 2^-8 |y_ref| + 1.01 alpha_eff gamma_i S_i + 1e-6 max(1, max|y_ref|)
    with S_i = sum_j |a_ij| |y_j| and gamma_i = 2 deg_i 2^-24 (twice the
    classical bound deg_i u of recursive FP32 summation, u = 2^-24, for an
    accumulator whose internal rounding is not specified), the first term
    being the BF16 rounding of the result; the momentum gets gamma_i S_i.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import graphgen as gg
from oracle import deco_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2509_18612_gb300 as deco  # noqa: E402

DEV = torch.device("cuda:0")
OBJ = {O.OBJ_MULTILINEAR01: deco.DECO_OBJ_MULTILINEAR01, O.OBJ_LAPLACIAN: deco.DECO_OBJ_LAPLACIAN}
BF16 = deco.DECO_PREC_BF16
DENSE = deco.DECO_KERNEL_DENSE


def signed_graph(n, p, seed, choices=(-2.0, -1.0, 1.0, 3.0)):
    g = gg.er_graph(n, p, seed)
    rng = np.random.default_rng(seed + 5)
    u, v, _ = g.edges()
    return gg.from_edges(n, u, v, rng.choice(np.array(choices), size=u.size))


GRAPHS = {
    "er100": lambda: gg.er_graph(100, 0.1, 0),            # one row tile, ragged
    "er1000_dense": lambda: gg.er_graph(1000, 0.5, 11),   # 8 row tiles, ragged
    "signed_dense": lambda: signed_graph(700, 0.4, 12),
    "torus": lambda: gg.torus_graph(40, 20, 2),           # +-1 weights
    "isolated": lambda: gg.from_edges(50, [0, 1, 2], [1, 2, 3]),
}


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def dyadic_block(n, C, ld, seed, mu):
    rng = np.random.default_rng(seed)
    Y = np.zeros((n, ld), np.float32)
    Y[:, :C] = rng.integers(-64, 65, size=(n, C)) / 64.0
    V = None
    if mu:
        V = np.zeros((n, ld), np.float32)
        V[:, :C] = rng.integers(-256, 257, size=(n, C)) / 64.0
    return Y, V


def run_phase(g, Y, V, C, ld, steps, objective, alpha, mu, kernel, alpha_cols=None, steps_cols=None, G=None):
    y = to_dev(Y).to(torch.bfloat16)
    v = None if V is None else to_dev(V)
    flag = torch.zeros(1, dtype=torch.int32, device=DEV)
    a = deco.step_args(OBJ[objective], BF16, alpha, mu, alpha_cols, steps_cols)
    deco.deco_run_phase(G if G is not None else deco.graph_from(g), C, ld, y, v, steps, a, kernel, flag)
    torch.cuda.synchronize()
    return y, v, int(flag.item())


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("C", [70, 136, 300])
@pytest.mark.parametrize("objective", [O.OBJ_MULTILINEAR01, O.OBJ_LAPLACIAN])
@pytest.mark.parametrize("mu", [0.0, 0.9])
def test_dense_step_bitwise_equals_global_on_dyadic_block(name, C, objective, mu):
    g = GRAPHS[name]()
    ld = (C + 63) // 64 * 64
    Y, V = dyadic_block(g.n, C, ld, 7, mu)
    alpha = 0.01 if objective == O.OBJ_MULTILINEAR01 else 0.003
    ref = run_phase(g, Y, V, C, ld, 1, objective, alpha, mu, deco.DECO_KERNEL_GLOBAL)
    G = deco.graph_from(g)
    for k, mode in [(k, m) for k in (0, 1, 2, 4, 8) for m in (0, deco.DECO_KERNEL_DENSE_PER_STEP)]:
        try:
            got = run_phase(g, Y, V, C, ld, 1, objective, alpha, mu, DENSE | (k << 8) | mode, G=G)
        except deco.DecoError as e:   # a split deeper than the contraction of a small graph
            assert e.status == deco.DECO_ERR_UNSUPPORTED and k > 1
            continue
        assert got[2] == ref[2] == 0
        assert torch.equal(got[0][:, :C], ref[0][:, :C]), (k, mode)
        if mu:
            assert torch.equal(got[1][:, :C], ref[1][:, :C]), (k, mode)
        assert torch.equal(got[0][:, C:], to_dev(Y).to(torch.bfloat16)[:, C:])   # padding columns untouched


@pytest.mark.parametrize("name", ["er1000_dense", "signed_dense", "er100"])
@pytest.mark.parametrize("k", [0, 1, 2, 4, 8])
def test_dense_phase_kernel_bitwise_equals_per_step_launches(name, k):
    # the persistent phase kernel and one launch per step split the
    # contraction the same way and add the partials in the same order
    g = GRAPHS[name]()
    C, ld = 136, 192
    rng = np.random.default_rng(10)
    Y = np.zeros((g.n, ld), np.float32)
    Y[:, :C] = rng.uniform(-1, 1, size=(g.n, C)) * np.where(rng.random(C) < 0.5, 1.0, 1e-3)
    V = np.zeros((g.n, ld), np.float32)
    V[:, :C] = rng.normal(size=(g.n, C)) * 0.1
    sc = to_dev(rng.integers(0, 30, C).astype(np.int32))
    ac = to_dev(rng.uniform(1e-5, 1e-3, C).astype(np.float32))
    objective = O.OBJ_LAPLACIAN if name == "signed_dense" else O.OBJ_MULTILINEAR01
    G = deco.graph_from(g)
    out = []
    for mode in (0, deco.DECO_KERNEL_DENSE_PER_STEP):
        try:
            out.append(run_phase(g, Y, V, C, ld, 24, objective, 0.0, 0.9, DENSE | (k << 8) | mode, ac, sc, G=G))
        except deco.DecoError as e:
            assert e.status == deco.DECO_ERR_UNSUPPORTED and k > 1
            pytest.skip("split deeper than the contraction")
    assert out[0][2] == out[1][2] == 0
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


def test_dense_per_column_alpha_and_budget_bitwise():
    g = GRAPHS["er1000_dense"]()
    C, ld = 96, 128
    Y, V = dyadic_block(g.n, C, ld, 8, 0.9)
    rng = np.random.default_rng(4)
    ac = to_dev(rng.uniform(1e-4, 1e-2, C).astype(np.float32))
    sc = to_dev(rng.integers(0, 2, C).astype(np.int32))   # budget 0: column frozen
    ref = run_phase(g, Y, V, C, ld, 1, O.OBJ_MULTILINEAR01, 0.0, 0.9, deco.DECO_KERNEL_GLOBAL, ac, sc)
    got = run_phase(g, Y, V, C, ld, 1, O.OBJ_MULTILINEAR01, 0.0, 0.9, DENSE, ac, sc)
    assert torch.equal(got[0][:, :C], ref[0][:, :C]) and torch.equal(got[1][:, :C], ref[1][:, :C])


def _tol(g, yin, ref, alpha_eff, rows_deg):
    Aabs = abs(O.adjacency(g))
    S = np.asarray(Aabs @ np.abs(yin))
    gamma = 2.0 * rows_deg[:, None] * 2.0 ** -24
    return 2.0 ** -8 * np.abs(ref) + 1.01 * alpha_eff * gamma * S \
        + 1e-6 * np.maximum(1.0, np.max(np.abs(ref), axis=0, keepdims=True)), gamma * S


@pytest.mark.parametrize("name", ["er1000_dense", "signed_dense", "er100"])
@pytest.mark.parametrize("objective", [O.OBJ_MULTILINEAR01, O.OBJ_LAPLACIAN])
@pytest.mark.parametrize("mu", [0.0, 0.9])
def test_dense_step_matches_oracle(name, objective, mu):
    # one step from a seeded BF16 block (and seeded momentum); several steps
    # are the composition of this step (the phase kernel equals one launch per
    # step bit for bit, and a multi-step call equals repeated one-step calls)
    g = GRAPHS[name]()
    C, ld = 136, 192
    rng = np.random.default_rng(9)
    Y = np.zeros((g.n, ld), np.float32)
    Y[:, :C] = rng.uniform(-1, 1, size=(g.n, C)) * np.where(rng.random(C) < 0.5, 1.0, 1e-3)
    V = np.zeros((g.n, ld), np.float32)
    if mu:
        V[:, :C] = rng.normal(size=(g.n, C)) * 0.1
    deg = np.diff(g.row_ptr).astype(np.float64)
    alpha = 2e-4 if objective == O.OBJ_MULTILINEAR01 else 1e-4
    alpha_eff = 2 * alpha if objective == O.OBJ_MULTILINEAR01 else alpha
    yin = torch.from_numpy(Y).to(torch.bfloat16).float().numpy()[:, :C].astype(np.float64)
    y, v, flag = run_phase(g, Y, V if mu else None, C, ld, 1, objective, alpha, mu, DENSE)
    ref, vref = O.pga_step(g, yin, alpha, objective, V[:, :C].astype(np.float64), mu)
    out = y[:, :C].float().cpu().numpy().astype(np.float64)
    tol, vtol = _tol(g, yin, ref, alpha_eff, deg)
    assert flag == 0
    assert np.all(np.abs(out - ref) <= tol)
    if mu:
        vout = v[:, :C].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(vout - vref) <= 1e-5 * np.maximum(1.0, np.abs(vref)) + vtol)


def test_dense_is_deterministic_and_multistep_runs_in_place():
    g = GRAPHS["er1000_dense"]()
    C, ld = 128, 128
    rng = np.random.default_rng(3)
    Y = rng.uniform(-1e-3, 1e-3, size=(g.n, ld)).astype(np.float32)
    V = np.zeros((g.n, ld), np.float32)
    a = run_phase(g, Y, V, C, ld, 25, O.OBJ_MULTILINEAR01, 1e-4, 0.9, DENSE)
    b = run_phase(g, Y, V, C, ld, 25, O.OBJ_MULTILINEAR01, 1e-4, 0.9, DENSE)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    # 25 steps in one call = 25 calls of one step (momentum carried through v)
    y, v = Y, V
    for _ in range(25):
        yy, vv, _ = run_phase(g, y, v, C, ld, 1, O.OBJ_MULTILINEAR01, 1e-4, 0.9, DENSE)
        y, v = yy.float().cpu().numpy(), vv.cpu().numpy()
    assert np.array_equal(y, a[0].float().cpu().numpy()) and np.array_equal(v, a[1].cpu().numpy())


def test_dense_nonfinite_flag():
    g = GRAPHS["er100"]()
    Y = np.zeros((g.n, 64), np.float32)
    Y[3, 2] = np.nan
    _, _, flag = run_phase(g, Y, None, 64, 64, 1, O.OBJ_LAPLACIAN, 0.01, 0.0, DENSE)
    assert flag == 1


def test_dense_limits():
    g = signed_graph(200, 0.3, 5, choices=(-300.0, 1.0))   # |w| = 300 is not exact in BF16
    Y = np.zeros((g.n, 64), np.float32)
    with pytest.raises(deco.DecoError) as ei:
        run_phase(g, Y, None, 64, 64, 1, O.OBJ_LAPLACIAN, 0.01, 0.0, DENSE)
    assert ei.value.status == deco.DECO_ERR_UNSUPPORTED
    g = GRAPHS["er100"]()   # 2 contraction chunks: a split of 4 does not fit
    with pytest.raises(deco.DecoError) as ei:
        run_phase(g, np.zeros((g.n, 64), np.float32), None, 64, 64, 1, O.OBJ_LAPLACIAN, 0.01, 0.0, DENSE | (4 << 8))
    assert ei.value.status == deco.DECO_ERR_UNSUPPORTED
    with pytest.raises(deco.DecoError) as ei:   # split modifiers are for ONCHIP / DENSE only
        run_phase(g, np.zeros((g.n, 64), np.float32), None, 64, 64, 1, O.OBJ_LAPLACIAN, 0.01, 0.0,
                  deco.DECO_KERNEL_GLOBAL | (2 << 8))
    assert ei.value.status == deco.DECO_ERR_ARG


def test_dense_solve_cuts_are_consistent_and_close_to_sparse():
    g = gg.er_graph(1000, 0.5, 21)
    G = deco.graph_from(g)
    sched = [(1, 200, 1e-4, 0.9), (2, 50, 2e-5, 0.9)]
    out = {}
    for kern in (deco.DECO_KERNEL_GLOBAL, DENSE):
        p = deco.params(init=deco.DECO_INIT_IDI_HALF_UNIFORM, precision=BF16, kernel=kern, polish_steps=10)
        res, z, pc = deco.deco_solve(G, 128, sched, p, 5)
        assert O.cut_value(g, z) == res.best_cut        # the assignment realises the reported cut
        out[kern] = res.best_cut
    # different summation order, same method: best cuts within 0.5 %
    assert abs(out[DENSE] - out[deco.DECO_KERNEL_GLOBAL]) <= 0.005 * out[deco.DECO_KERNEL_GLOBAL]


def test_dense_autotune_candidate_and_auto_reuse():
    g = GRAPHS["er1000_dense"]()
    G = deco.graph_from(g)
    C, ld = 128, 128
    sel, us = deco.deco_autotune(G, C, BF16, deco.DECO_OBJ_MULTILINEAR01, 0.9, 10)
    assert us > 0.0
    rng = np.random.default_rng(5)
    Y = rng.uniform(-1e-3, 1e-3, size=(g.n, ld)).astype(np.float32)
    V = np.zeros((g.n, ld), np.float32)
    ref = run_phase(g, Y, V, C, ld, 6, O.OBJ_MULTILINEAR01, 1e-4, 0.9, sel, G=G)
    got = run_phase(g, Y, V, C, ld, 6, O.OBJ_MULTILINEAR01, 1e-4, 0.9, deco.DECO_KERNEL_AUTO, G=G)
    assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])


# ---------------------------------------------- full size: ER(4096, 0.5), B = 128 / 256

@pytest.fixture(scope="module")
def er4096():
    g = gg.er_graph(4096, 0.5, 4096)
    return g, deco.graph_from(g)


@pytest.mark.parametrize("C", [128, 256])
def test_dense_full_size_step_bitwise_and_sampled_oracle(er4096, C):
    g, G = er4096
    ld = C
    Y, _ = dyadic_block(g.n, C, ld, 13, 0.0)
    ref = run_phase(g, Y, None, C, ld, 1, O.OBJ_MULTILINEAR01, 1e-4, 0.0, deco.DECO_KERNEL_GLOBAL, G=G)
    got = run_phase(g, Y, None, C, ld, 1, O.OBJ_MULTILINEAR01, 1e-4, 0.0, DENSE, G=G)
    assert torch.equal(got[0], ref[0])
    # the oracle's step (FP64) on 16 sampled columns, every row: columns are
    # independent, so the oracle runs only those
    cols = np.sort(np.random.default_rng(1).choice(C, 16, replace=False))
    ref_y, _ = O.pga_step(g, Y[:, cols].astype(np.float64), 1e-4, O.OBJ_MULTILINEAR01)
    out = got[0][:, torch.from_numpy(cols).to(got[0].device)].float().cpu().numpy().astype(np.float64)
    assert np.all(np.abs(out - ref_y) <= 2.0 ** -8 * np.abs(ref_y) + 1e-6)


def test_dense_full_size_step_with_momentum_matches_oracle(er4096):
    # one step of the phase kernel at the full size, every element, from a
    # seeded block and a seeded momentum
    g, G = er4096
    C, ld = 128, 128
    rng = np.random.default_rng(14)
    Y = rng.uniform(-1e-3, 1e-3, size=(g.n, ld)).astype(np.float32)
    V = (rng.normal(size=(g.n, ld)) * 0.05).astype(np.float32)
    deg = np.diff(g.row_ptr).astype(np.float64)
    alpha = 1e-4
    yin = torch.from_numpy(Y).to(torch.bfloat16).float().numpy().astype(np.float64)
    y, v, flag = run_phase(g, Y, V, C, ld, 1, O.OBJ_MULTILINEAR01, alpha, 0.9, DENSE, G=G)
    ref, vref = O.pga_step(g, yin, alpha, O.OBJ_MULTILINEAR01, V.astype(np.float64), 0.9)
    out = y.float().cpu().numpy().astype(np.float64)
    tol, vtol = _tol(g, yin, ref, 2 * alpha, deg)
    assert flag == 0
    assert np.all(np.abs(out - ref) <= tol)
    assert np.all(np.abs(v.cpu().numpy() - vref) <= 1e-5 * np.maximum(1.0, np.abs(vref)) + vtol)


def test_tensor_core_rate_probe():
    # the probe runs on every SM and reports a positive time per instruction;
    # the tensor core is the bound, not the issuing thread: twice the columns
    # take longer, and two issuers take about the time per instruction of one
    one = deco.deco_probe_mma_rate(128, 1, 2048)
    two = deco.deco_probe_mma_rate(128, 2, 2048)
    wide = deco.deco_probe_mma_rate(256, 1, 2048)
    assert 1.0 < one < 10000.0 and 1.0 < two < 10000.0 and 1.0 < wide < 10000.0
    assert wide > 1.3 * one
    assert 0.5 * one < two < 1.5 * one
    with pytest.raises(deco.DecoError):
        deco.deco_probe_mma_rate(96, 1, 16)
