"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances
  * cut values, rounding bits, argmax, IDI means: bit-exact.
  * one FP32 step: |y_gpu - y_oracle| <= 1e-5 * max(1, max|y_oracle|) per column
    (the oracle runs in FP64 from the same FP32 input).
  * one BF16 step: the oracle result rounded to bf16 may differ from the GPU's
    by one bf16 rounding of the FP32-computed value: |diff| <= 2^-8 |y| + 1e-6.
  * solves: final rounded cuts identical on >= 99% of (graph, start) pairs.
"""
import math

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


def signed_graph(n, p, seed, choices=(-2.0, -1.0, 1.0, 3.0)):
    g = gg.er_graph(n, p, seed)
    rng = np.random.default_rng(seed + 5)
    u, v, _ = g.edges()
    return gg.from_edges(n, u, v, rng.choice(np.array(choices), size=u.size))


GRAPHS = {
    "er100": lambda: gg.er_graph(100, 0.1, 0),
    "er800": lambda: gg.er_graph(800, 0.06, 1),
    "torus": lambda: gg.torus_graph(40, 20, 2),
    "ba": lambda: gg.ba_graph(700, 4, 3),
    "signed": lambda: signed_graph(300, 0.05, 4),
    "isolated": lambda: gg.from_edges(50, [0, 1, 2], [1, 2, 3]),   # mostly isolated nodes
}


def to_dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


# ------------------------------------------------------------------ cut (Eq. 1)

@pytest.mark.parametrize("name", list(GRAPHS))
def test_eval_cut_bit_exact(name):
    g = GRAPHS[name]()
    G = deco.graph_from(g)
    Z = gg.random_binary(g.n, 37, 11)          # ragged: 37 columns
    for j in range(3):
        assert deco.deco_eval_cut(G, Z[:, j]) == O.cut_value(g, Z[:, j])
    cuts = torch.zeros(37, dtype=torch.int64, device=DEV)
    deco.deco_eval_cuts(G, 37, to_dev(Z), cuts)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(cuts.cpu().numpy(), O.cut_values(g, Z))


def test_eval_cut_extremes():
    g = gg.er_graph(200, 0.3, 9)
    G = deco.graph_from(g)
    assert deco.deco_eval_cut(G, np.zeros(g.n, np.uint8)) == 0
    assert deco.deco_eval_cut(G, np.ones(g.n, np.uint8)) == 0
    # bipartite graph, true bipartition: every edge is cut
    u = np.repeat(np.arange(10), 10)
    v = np.tile(np.arange(10, 20), 10)
    kb = gg.from_edges(20, u, v)
    assert deco.deco_eval_cut(deco.graph_from(kb), (np.arange(20) < 10).astype(np.uint8)) == 100


# ------------------------------------------------------------ one step (Eq. 7/10)

def _run_step(g, Y, objective, alpha, mu=0.0, V=None, precision=deco.DECO_PREC_FP32, alpha_cols=None,
              steps_cols=None, t=0):
    n, C = Y.shape
    ld = (C + 7) // 8 * 8
    Yp = np.zeros((n, ld), np.float32)
    Yp[:, :C] = Y
    dt = torch.bfloat16 if precision == deco.DECO_PREC_BF16 else torch.float32
    yin = to_dev(Yp).to(dt)
    yout = torch.zeros_like(yin)
    v = None
    if mu != 0.0:
        Vp = np.zeros((n, ld), np.float32)
        if V is not None:
            Vp[:, :C] = V
        v = to_dev(Vp)
    flag = torch.zeros(1, dtype=torch.int32, device=DEV)
    ac = None if alpha_cols is None else to_dev(np.asarray(alpha_cols, np.float32))
    sc = None if steps_cols is None else to_dev(np.asarray(steps_cols, np.int32))
    args = deco.step_args(OBJ[objective], precision, alpha, mu, ac, sc, t)
    G = deco.graph_from(g)
    deco.deco_step(G, C, ld, yin, yout, v, args, flag)
    torch.cuda.synchronize()
    yin_used = yin.float().cpu().numpy()[:, :C].astype(np.float64)
    out = yout.float().cpu().numpy()[:, :C].astype(np.float64)
    vout = None if v is None else v.cpu().numpy()[:, :C].astype(np.float64)
    return yin_used, out, vout, int(flag.item())


def _fp32_tol(ref):
    scale = np.maximum(1.0, np.max(np.abs(ref), axis=0, keepdims=True))
    return 1e-5 * scale


@pytest.mark.parametrize("name", ["er100", "er800", "torus", "ba", "signed", "isolated"])
@pytest.mark.parametrize("objective", [O.OBJ_MULTILINEAR01, O.OBJ_LAPLACIAN])
@pytest.mark.parametrize("mu", [0.0, 0.9])
def test_step_fp32_parity(name, objective, mu):
    g = GRAPHS[name]()
    rng = np.random.default_rng(1)
    C = 70                                         # several vectors and a ragged tail
    Y = rng.uniform(-1, 1, size=(g.n, C)).astype(np.float32)
    Y[:, :5] = np.sign(Y[:, :5])                   # binary columns (clamp active)
    Y[:, 5:10] *= 1e-4                             # paper-scale small starts
    V = rng.normal(size=(g.n, C)).astype(np.float32) if mu else None
    alpha = 0.01 if objective == O.OBJ_MULTILINEAR01 else 0.003
    yin, out, vout, flag = _run_step(g, Y, objective, alpha, mu, V)
    ref, vref = O.pga_step(g, yin, alpha, objective, None if V is None else V.astype(np.float64), mu)
    assert flag == 0
    assert np.all(np.abs(out - ref) <= _fp32_tol(ref))
    if mu:
        assert np.all(np.abs(vout - vref) <= 1e-5 * np.maximum(1.0, np.abs(vref)))


@pytest.mark.parametrize("objective", [O.OBJ_MULTILINEAR01, O.OBJ_LAPLACIAN])
def test_step_bf16_parity(objective):
    g = gg.er_graph(800, 0.06, 1)
    rng = np.random.default_rng(2)
    C = 136
    Y = (rng.uniform(-1, 1, size=(g.n, C)) * np.where(rng.random(C) < 0.5, 1.0, 1e-4)).astype(np.float32)
    yin, out, _, flag = _run_step(g, Y, objective, 0.002, precision=deco.DECO_PREC_BF16)
    ref, _ = O.pga_step(g, yin, 0.002, objective)
    assert flag == 0
    tol = 2.0 ** -8 * np.abs(ref) + 1e-6 * np.maximum(1.0, np.max(np.abs(ref), axis=0, keepdims=True))
    assert np.all(np.abs(out - ref) <= tol)


def test_step_per_column_alpha_and_budget():
    g = gg.ba_graph(500, 4, 7)
    rng = np.random.default_rng(3)
    C = 24
    Y = rng.uniform(-1, 1, size=(g.n, C)).astype(np.float32)
    alpha = rng.uniform(1e-3, 3e-2, C).astype(np.float32)
    steps = rng.integers(0, 10, C).astype(np.int32)
    t = 5
    yin, out, _, _ = _run_step(g, Y, O.OBJ_MULTILINEAR01, 0.0, alpha_cols=alpha, steps_cols=steps, t=t)
    ref, _ = O.pga_step(g, yin, alpha.astype(np.float64), O.OBJ_MULTILINEAR01, active=steps > t)
    assert np.all(np.abs(out - ref) <= _fp32_tol(ref))
    assert np.array_equal(out[:, steps <= t], yin[:, steps <= t])


def test_paper_form_binary_points_are_fixed_on_gpu():
    g = gg.er_graph(300, 0.05, 3)
    Y = np.where(gg.random_binary(g.n, 64, 4) > 0, 1.0, -1.0).astype(np.float32)
    for alpha in (1e-3, 0.3, 5.0):
        yin, out, _, _ = _run_step(g, Y, O.OBJ_LAPLACIAN, alpha)
        assert np.array_equal(out, yin)


def test_nonfinite_flag():
    g = gg.er_graph(100, 0.1, 0)
    Y = np.zeros((g.n, 8), np.float32)
    Y[3, 2] = np.nan
    _, _, _, flag = _run_step(g, Y, O.OBJ_LAPLACIAN, 0.01)
    assert flag == 1


# -------------------------------------------------- rounding + cut + argmax

@pytest.mark.parametrize("lift", [1, 2, 3, 4, 8])
@pytest.mark.parametrize("precision", [deco.DECO_PREC_FP32, deco.DECO_PREC_BF16])
def test_round_cut_bit_exact(lift, precision):
    # l = 4 and 8: the lifting sweep's larger lifts (Table 2's ablation), where
    # the FP32 order of the row sum of Eq. 11 decides near-ties
    g = GRAPHS["signed"]() if lift == 3 else gg.er_graph(800, 0.06, 1)
    rng = np.random.default_rng(lift)
    B = 45
    C = B * lift
    ld = (C + 7) // 8 * 8
    Y = rng.uniform(-1, 1, size=(g.n, C)).astype(np.float32)
    Y[rng.random(Y.shape) < 0.05] = 0.0            # exact zeros: strict vs non-strict
    if lift == 2:
        pair = rng.random((g.n, B)) < 0.1          # exact cancellations y0 = -y1
        Y[:, 1::2] = np.where(pair, -Y[:, 0::2], Y[:, 1::2])
    if lift >= 4:
        # exact cancellations in pairs (sum exactly 0: rounds to 1) and
        # near-cancellations whose FP32 sum depends on the order
        pair = rng.random((g.n, B)) < 0.1
        for i in range(1, lift, 2):
            Y[:, i::lift] = np.where(pair, -Y[:, i - 1::lift], Y[:, i::lift])
        near = rng.random((g.n, B)) < 0.05
        Y[:, 0::lift] = np.where(near, np.float32(1.0), Y[:, 0::lift])
        Y[:, 1::lift] = np.where(near, np.float32(-1.0), Y[:, 1::lift])
        Y[:, 2::lift] = np.where(near, np.float32(2.0 ** -30), Y[:, 2::lift])
        Y[:, 3::lift] = np.where(near, np.float32(-2.0 ** -30), Y[:, 3::lift])
    Yp = np.zeros((g.n, ld), np.float32)
    Yp[:, :C] = Y
    dt = torch.bfloat16 if precision == deco.DECO_PREC_BF16 else torch.float32
    y = to_dev(Yp).to(dt)
    W = (B + 31) // 32
    zbits = torch.zeros(g.n * W, dtype=torch.int32, device=DEV)
    cuts = torch.zeros(B, dtype=torch.int64, device=DEV)
    best = torch.zeros(1, dtype=torch.int32, device=DEV)
    G = deco.graph_from(g)
    deco.deco_round_cut(G, B, lift, ld, precision, y, zbits, cuts, best)
    torch.cuda.synchronize()
    yused = y.float().cpu().numpy()[:, :C].astype(np.float64)
    if lift >= 3:
        # Eq. 11 summed in FP32 in order i = 0..l-1 (both sides take the
        # decision in the kernel's precision)
        s = np.zeros((g.n, B), np.float32)
        for i in range(lift):
            s = (s + yused[:, i::lift].astype(np.float32)).astype(np.float32)
        Z = (s >= 0).astype(np.uint8)
    else:
        Z = O.binarize(yused, lift)
    words = zbits.cpu().numpy().view(np.uint32).reshape(g.n, W)
    bits = ((words[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(g.n, W * 32)[:, :B]
    np.testing.assert_array_equal(bits, Z)
    ref = O.cut_values(g, Z)
    np.testing.assert_array_equal(cuts.cpu().numpy(), ref)
    assert int(best.item()) == O.best_of(ref)


@pytest.mark.parametrize("lift", [4, 8])
def test_lifted_phase_large_lift_matches_oracle(lift):
    # one pLUCO phase (Alg. 2) with l = 4 / 8 columns per start, momentum,
    # IDI starts drawn on the device: rounded cuts (Eq. 11) identical on >= 99 %
    # of the starts and the same best cut as the oracle's
    g = gg.er_graph(400, 0.05, 12)
    B = 64
    sched = [(lift, 150, 0.002, 0.9)]
    G = deco.graph_from(g)
    res, z, pc = deco.deco_solve(G, B, sched, deco.params(init=deco.DECO_INIT_IDI), 77)
    ref = O.solve(g, B, [O.Phase(*sched[0])], O.Params(init="idi"), 77)
    assert _agreement(pc[0], ref.phase_cuts[0]) >= 0.99
    assert res.best_cut == O.cut_value(g, z)
    assert res.best_cut == ref.best_cut
    assert res.edge_updates == g.nnz * B * lift * 150


def test_argmax_ties_lowest_index():
    g = gg.from_edges(4, [0, 1, 2], [1, 2, 3])
    B = 64
    Y = -np.ones((4, B), np.float32)
    Y[1, 7] = Y[1, 40] = Y[3, 40] = 1.0   # init 7 cut 2; init 40 cut 3 ... and 41 too
    Y[1, 41] = Y[3, 41] = 1.0
    y = to_dev(Y)
    zbits = torch.zeros(4 * 2, dtype=torch.int32, device=DEV)
    cuts = torch.zeros(B, dtype=torch.int64, device=DEV)
    best = torch.zeros(1, dtype=torch.int32, device=DEV)
    deco.deco_round_cut(deco.graph_from(g), B, 1, B, deco.DECO_PREC_FP32, y, zbits, cuts, best)
    torch.cuda.synchronize()
    assert cuts[40].item() == 3 and cuts[41].item() == 3 and int(best.item()) == 40


# ------------------------------------------------------------- initialisation

def test_idi_and_dui_means():
    for g in (gg.ba_graph(600, 4, 1), gg.torus_graph(40, 20, 2), signed_graph(300, 0.05, 4)):
        G = deco.graph_from(g)
        h = torch.zeros(g.n, dtype=torch.float32, device=DEV)
        for seed in (0, 12345678901):
            deco.deco_idi_mean(G, 0.2, seed, 1, h)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(h.cpu().numpy(), O.idi_mean(g, seed, 1, 0.2))
            deco.deco_dui_mean(G, seed, 2, h)
            torch.cuda.synchronize()
            np.testing.assert_allclose(h.cpu().numpy(), O.dui_mean(g, seed, 2), rtol=0, atol=1e-6)


@pytest.mark.parametrize("init", ["uniform", "idi", "dui", "idi_half_uniform", "mean", "explicit"])
@pytest.mark.parametrize("lift", [1, 2])
def test_init_block_parity(init, lift):
    g = gg.ba_graph(400, 4, 5)
    G = deco.graph_from(g)
    B, seed, phase = 40, 77, 0 if init != "mean" else 3
    C = B * lift
    ld = (C + 7) // 8 * 8
    kinds = {"uniform": deco.DECO_INIT_UNIFORM, "idi": deco.DECO_INIT_IDI, "dui": deco.DECO_INIT_DUI,
             "idi_half_uniform": deco.DECO_INIT_IDI_HALF_UNIFORM, "mean": deco.DECO_INIT_MEAN,
             "explicit": deco.DECO_INIT_EXPLICIT}
    p = deco.params(init=kinds[init], uniform_half_width=0.5)
    y = torch.zeros(g.n, ld, dtype=torch.float32, device=DEV)
    mean = None
    x0 = None
    if init == "mean":
        mean = np.random.default_rng(0).uniform(-1, 1, g.n).astype(np.float32)
    if init == "explicit":
        x0 = np.zeros((g.n, ld), np.float32)
        x0[:, :C] = gg.uniform_x0(g.n, C, 3)
    deco.deco_init_block(G, B, lift, ld, p, seed, phase, y,
                         mean=None if mean is None else to_dev(mean),
                         x0=None if x0 is None else to_dev(x0))
    torch.cuda.synchronize()
    got = y.cpu().numpy()[:, :C].astype(np.float64)
    op = O.Params(init=init, uniform_half_width=0.5, mean=mean)
    if init == "mean":
        ref = O.gaussian_block(mean.astype(np.float64), C, seed, phase, 0.8, 1e-4)
    else:
        ref = O.initial_block(g, B, lift, op, seed, None if x0 is None else x0[:, :C])
    # Gaussian starts are s * (h + sqrt(eta) eps) computed in FP32: the error is
    # relative to the magnitude of the summands (up to ~5 s), not of the sum,
    # which can cancel to nearly zero.
    atol = 2e-6 * 5 * 1e-4 if init != "uniform" and init != "explicit" else 1e-12
    np.testing.assert_allclose(got, ref, rtol=2e-6, atol=atol)


# ------------------------------------------------------------------- solves

def _agreement(a, b):
    return float(np.mean(np.asarray(a) == np.asarray(b)))


def test_solve_pquco_er100_b64_explicit():
    # ER(100, 0.1) seed 0, B = 64, x0 ~ U[0,1], T = 500, alpha = 0.01, plain PGA
    g = gg.er_graph(100, 0.1, 0)
    B, T = 64, 500
    x0 = gg.uniform_x0(g.n, B, 0)
    G = deco.graph_from(g)
    res, z, pc = deco.deco_solve(G, B, [(1, T, 0.01, 0.0)], deco.params(init=deco.DECO_INIT_EXPLICIT), 0, x0=x0)
    ref = O.solve(g, B, [O.Phase(1, T, 0.01, 0.0)], O.Params(init="explicit"), 0, x0=x0)
    assert _agreement(pc[0], ref.phase_cuts[0]) >= 0.99
    assert res.best_cut == O.cut_value(g, z) == int(pc[0].max())
    assert res.best_cut == ref.best_cut
    assert res.edge_updates == g.nnz * B * T


@pytest.mark.parametrize("objective", [O.OBJ_MULTILINEAR01, O.OBJ_LAPLACIAN])
def test_solve_pdeco_schedule(objective):
    # DECO alternation with momentum, IDI + uniform starts drawn on the device
    g = gg.er_graph(300, 0.06, 8)
    B = 96
    sched = [(1, 120, 0.01, 0.9), (2, 40, 0.001, 0.9), (1, 120, 0.01, 0.9), (2, 40, 0.001, 0.9)]
    G = deco.graph_from(g)
    p = deco.params(objective=OBJ[objective], init=deco.DECO_INIT_IDI_HALF_UNIFORM)
    res, z, pc = deco.deco_solve(G, B, sched, p, 4242)
    ref = O.solve(g, B, [O.Phase(*s) for s in sched], O.Params(objective=objective, init="idi_half_uniform"), 4242)
    assert res.best_cut == O.cut_value(g, z)
    for k in range(len(sched)):
        assert _agreement(pc[k], ref.phase_cuts[k]) >= 0.99, k
    assert res.best_cut == ref.best_cut
    assert (res.best_phase, res.best_init) == (ref.best_phase, ref.best_init)


def test_solve_intermediate_roundings_match_oracle():
    # eval_every = 30: roundings after steps 30, 60, 90 of the 120-step phases
    # (and after 30 of the 40-step ones) compete for the best; the phases'
    # final roundings, and so the iterates, are those of the plain solve
    g = gg.er_graph(300, 0.06, 8)
    B = 96
    sched = [(1, 120, 0.01, 0.9), (2, 40, 0.001, 0.9), (1, 120, 0.01, 0.9)]
    G = deco.graph_from(g)
    plain, _, pc0 = deco.deco_solve(G, B, sched, deco.params(init=deco.DECO_INIT_IDI_HALF_UNIFORM), 77)
    res, z, pc = deco.deco_solve(G, B, sched, deco.params(init=deco.DECO_INIT_IDI_HALF_UNIFORM, eval_every=30), 77)
    ref = O.solve(g, B, [O.Phase(*s) for s in sched], O.Params(init="idi_half_uniform", eval_every=30), 77)
    np.testing.assert_array_equal(pc, pc0)   # segmenting a phase does not change its iterate
    assert res.best_cut >= plain.best_cut and res.best_cut == O.cut_value(g, z)
    assert res.best_cut == ref.best_cut
    assert (res.best_phase, res.best_init) == (ref.best_phase, ref.best_init)
    for k in range(len(sched)):
        assert _agreement(pc[k], ref.phase_cuts[k]) >= 0.99, k


def test_solve_intermediate_roundings_across_the_fp32_polish():
    # BF16 phases with an FP32 polish of the last 25 steps: roundings every 20
    # steps fall on both sides of the precision switch; the iterate is the
    # plain solve's bit for bit
    g = gg.er_graph(400, 0.05, 3)
    B = 64
    sched = [(1, 100, 0.01, 0.9), (2, 50, 0.002, 0.9)]
    G = deco.graph_from(g)
    base = dict(init=deco.DECO_INIT_IDI, precision=deco.DECO_PREC_BF16, polish_steps=25)
    plain, _, pc0 = deco.deco_solve(G, B, sched, deco.params(**base), 5)
    res, z, pc = deco.deco_solve(G, B, sched, deco.params(**base, eval_every=20), 5)
    np.testing.assert_array_equal(pc, pc0)
    assert res.best_cut >= plain.best_cut and res.best_cut == O.cut_value(g, z)


def test_solve_fresh_later_phases_match_oracle():
    g = gg.er_graph(300, 0.06, 8)
    B = 96
    sched = [(1, 120, 0.01, 0.9), (2, 40, 0.001, 0.9), (1, 60, 0.01, 0.9)]
    G = deco.graph_from(g)
    for init, oinit in ((deco.DECO_INIT_IDI_HALF_UNIFORM, "idi_half_uniform"), (deco.DECO_INIT_DUI, "dui")):
        p = deco.params(init=init, phase_init=deco.DECO_PHASE_INIT_FRESH)
        res, z, pc = deco.deco_solve(G, B, sched, p, 4242)
        ref = O.solve(g, B, [O.Phase(*s) for s in sched], O.Params(init=oinit, phase_init="fresh"), 4242)
        assert res.best_cut == O.cut_value(g, z) == ref.best_cut
        for k in range(len(sched)):
            assert _agreement(pc[k], ref.phase_cuts[k]) >= 0.99, (oinit, k)
    with pytest.raises(deco.DecoError):   # an explicit block cannot be drawn afresh
        deco.deco_solve(G, 4, sched, deco.params(init=deco.DECO_INIT_EXPLICIT, phase_init=1), 0,
                        x0=gg.uniform_x0(g.n, 4, 0))


def test_solve_signed_torus_bf16_polish_cut_gap():
    g = gg.torus_graph(40, 20, 2)
    B = 128
    sched = [(1, 300, 0.01, 0.9), (2, 100, 0.001, 0.9)]
    G = deco.graph_from(g)
    f32, z32, pc32 = deco.deco_solve(G, B, sched, deco.params(init=deco.DECO_INIT_IDI_HALF_UNIFORM), 9)
    b16, z16, pc16 = deco.deco_solve(G, B, sched, deco.params(init=deco.DECO_INIT_IDI_HALF_UNIFORM,
                                                              precision=deco.DECO_PREC_BF16, polish_steps=50), 9)
    ref = O.solve(g, B, [O.Phase(*s) for s in sched], O.Params(init="idi_half_uniform"), 9)
    assert f32.best_cut == ref.best_cut
    assert b16.best_cut == O.cut_value(g, z16)
    # BF16 iterates with an FP32 polish: the cut gap against the FP64 oracle is small
    assert b16.best_cut >= 0.98 * ref.best_cut


def test_solve_nonfinite_explicit_start_reports_error():
    g = gg.er_graph(50, 0.2, 0)
    x0 = gg.uniform_x0(g.n, 8, 0)
    x0[4, 3] = np.inf
    with pytest.raises(deco.DecoError) as ei:
        deco.deco_solve(deco.graph_from(g), 8, [(1, 10, 0.01, 0.0)], deco.params(init=deco.DECO_INIT_EXPLICIT), 0, x0=x0)
    assert ei.value.status == deco.DECO_ERR_NONFINITE


def test_solve_brute_force_bound_small_graphs():
    for seed in range(3):
        g = gg.er_graph(18, 0.3, seed)
        opt, _ = O.brute_force_maxcut(g)
        res, z, _ = deco.deco_solve(deco.graph_from(g), 64, [(1, 200, 0.05, 0.9), (2, 50, 0.01, 0.9)],
                                    deco.params(init=deco.DECO_INIT_IDI), seed)
        assert res.best_cut <= opt
        assert res.best_cut == O.cut_value(g, z)
        assert res.best_cut >= 0.9 * opt


# ---------------------------------------------- one phase, on-chip kernel

def _phase_blocks(g, C, ld, precision, seed, mu):
    rng = np.random.default_rng(seed)
    Y = np.zeros((g.n, ld), np.float32)
    Y[:, :C] = rng.uniform(-1, 1, size=(g.n, C)) * np.where(rng.random(C) < 0.5, 1.0, 1e-3)
    Y[:, :4] = np.sign(Y[:, :4])
    dt = torch.bfloat16 if precision == deco.DECO_PREC_BF16 else torch.float32
    y = to_dev(Y).to(dt)
    v = None
    if mu:
        V = np.zeros((g.n, ld), np.float32)
        V[:, :C] = rng.normal(size=(g.n, C)) * 0.1
        v = to_dev(V)
    return y, v


def _run_phase(g, y, v, C, ld, steps, objective, precision, alpha, mu, kernel, alpha_cols=None, steps_cols=None):
    y = y.clone()
    v = None if v is None else v.clone()
    flag = torch.zeros(1, dtype=torch.int32, device=DEV)
    a = deco.step_args(OBJ[objective], precision, alpha, mu, alpha_cols, steps_cols)
    deco.deco_run_phase(deco.graph_from(g), C, ld, y, v, steps, a, kernel, flag)
    torch.cuda.synchronize()
    return y, v, int(flag.item())


@pytest.mark.parametrize("name", ["er800", "torus", "ba", "signed", "isolated", "er100"])
@pytest.mark.parametrize("precision", [deco.DECO_PREC_FP32, deco.DECO_PREC_BF16])
@pytest.mark.parametrize("k,xchg", [(0, 0), (1, 0), (2, 0), (4, 0), (8, 0), (2, 1), (4, 1), (8, 1),
                                    (1, 4), (2, 4), (4, 4)])
@pytest.mark.parametrize("pairs", [False, True])
def test_onchip_phase_bitwise_equals_global(name, precision, k, xchg, pairs):
    # xchg 4: the lean form (momentum in global memory, rows through L2);
    # pairs: the row-pair form (a half-warp per row)
    g = GRAPHS[name]()
    cols = 64 if precision == deco.DECO_PREC_BF16 else 32
    C = 3 * cols - 5                                # three slabs, ragged last slab
    ld = 3 * cols
    objective = O.OBJ_LAPLACIAN if name == "signed" else O.OBJ_MULTILINEAR01
    mu = 0.9
    y, v = _phase_blocks(g, C, ld, precision, 3, mu)
    steps_cols = to_dev(np.random.default_rng(1).integers(0, 12, C).astype(np.int32))
    alpha_cols = to_dev(np.random.default_rng(2).uniform(1e-3, 2e-2, C).astype(np.float32))
    ref_y, ref_v, f0 = _run_phase(g, y, v, C, ld, 9, objective, precision, 0.0, mu, deco.DECO_KERNEL_GLOBAL,
                                  alpha_cols, steps_cols)
    sel = deco.DECO_KERNEL_ONCHIP | (k << 8) | ((xchg & 3) << 14)   # xchg 1: DSMEM broadcast, 0: L2 (default)
    if xchg == 4:
        sel |= deco.DECO_KERNEL_LEAN
    if pairs:
        sel |= deco.DECO_KERNEL_ROW_PAIRS
    try:
        got_y, got_v, f1 = _run_phase(g, y, v, C, ld, 9, objective, precision, 0.0, mu, sel, alpha_cols, steps_cols)
    except deco.DecoError as e:
        assert e.status == deco.DECO_ERR_UNSUPPORTED and k in (1, 2)   # replica does not fit
        pytest.skip("cluster size does not fit this graph")
    assert f0 == f1 == 0
    assert torch.equal(got_y[:, :C], ref_y[:, :C])
    assert torch.equal(got_v[:, :C], ref_v[:, :C])


def _multi_step_bound(g, objective, alpha, mu, steps, eps_y, eps_v):
    """Sup-norm distance after `steps` steps between two runs from the same
    start when one of them adds at most eps_y / eps_v per step to the exact
    map: the gradient is Lipschitz in y with Lg = max_i (c_d |d_i| +
    sum_j |a_ij|) (c_d = 1 Laplacian, 0 multilinear), V' = mu V + grad and
    the projection is 1-Lipschitz, so b' <= mu b + Lg a + eps_v and
    a' <= a + alpha_eff b' + eps_y."""
    A = abs(O.adjacency(g))
    Lg = float(np.max(np.asarray(A.sum(axis=1)))) if g.nnz else 0.0
    if objective == O.OBJ_LAPLACIAN:
        Lg += float(np.max(np.abs(O.net_degree(g)))) if g.nnz else 0.0
    a_eff = 2.0 * alpha if objective == O.OBJ_MULTILINEAR01 else alpha
    a = b = 0.0
    for _ in range(steps):
        b = mu * b + Lg * a + eps_v
        a = a + a_eff * b + eps_y
    return a, b


@pytest.mark.parametrize("name", ["er800", "torus", "ba", "signed"])
@pytest.mark.parametrize("objective", [O.OBJ_MULTILINEAR01, O.OBJ_LAPLACIAN])
def test_onchip_steps_match_oracle(name, objective):
    # four steps of the on-chip kernel against four oracle steps, both from
    # the same seeded start; the distance is bounded by the one-step
    # tolerance propagated through the Lipschitz constant of the step
    g = GRAPHS[name]()
    C, ld = 64, 64
    mu, steps = 0.9, 4
    y, v = _phase_blocks(g, C, ld, deco.DECO_PREC_FP32, 5, mu)
    yin = y[:, :C].cpu().numpy().astype(np.float64)
    vin = v[:, :C].cpu().numpy().astype(np.float64)
    alpha = 0.01 if objective == O.OBJ_MULTILINEAR01 else 0.003
    out, vout, flag = _run_phase(g, y, v, C, ld, steps, objective, deco.DECO_PREC_FP32, alpha, mu,
                                 deco.DECO_KERNEL_ONCHIP)
    ref, vref = yin, vin
    vmax = 1.0
    for _ in range(steps):
        ref, vref = O.pga_step(g, ref, alpha, objective, vref, mu)
        vmax = max(vmax, float(np.max(np.abs(vref))))
    a, b = _multi_step_bound(g, objective, alpha, mu, steps, 1e-5, 1e-5 * vmax)
    assert flag == 0
    assert np.max(np.abs(out[:, :C].cpu().numpy() - ref)) <= a
    assert np.max(np.abs(vout[:, :C].cpu().numpy() - vref)) <= b


def test_solve_kernels_agree():
    g = gg.er_graph(800, 0.06, 1)
    sched = [(1, 100, 0.01, 0.9), (2, 30, 0.001, 0.9)]
    out = []
    for kern in (deco.DECO_KERNEL_GLOBAL, deco.DECO_KERNEL_ONCHIP):
        res, z, pc = deco.deco_solve(deco.graph_from(g), 256, sched,
                                     deco.params(init=deco.DECO_INIT_IDI_HALF_UNIFORM, kernel=kern), 5)
        out.append((res.best_cut, res.best_init, res.best_phase, z.tobytes(), pc.tobytes()))
    assert out[0] == out[1]


@pytest.mark.parametrize("name", ["er800", "signed", "ba"])
@pytest.mark.parametrize("precision", [deco.DECO_PREC_FP32, deco.DECO_PREC_BF16])
@pytest.mark.parametrize("s", [1, 2, 3])
def test_column_slab_schedule_bitwise_equals_global(name, precision, s):
    g = GRAPHS[name]()
    C, ld = 200, 256                                  # ragged last slab
    objective = O.OBJ_LAPLACIAN if name == "signed" else O.OBJ_MULTILINEAR01
    y, v = _phase_blocks(g, C, ld, precision, 4, 0.9)
    steps_cols = to_dev(np.random.default_rng(5).integers(0, 9, C).astype(np.int32))
    alpha_cols = to_dev(np.random.default_rng(6).uniform(1e-3, 2e-2, C).astype(np.float32))
    for steps in (7, 8):                              # odd / even: result in either buffer
        ref = _run_phase(g, y, v, C, ld, steps, objective, precision, 0.0, 0.9, deco.DECO_KERNEL_GLOBAL,
                         alpha_cols, steps_cols)
        got = _run_phase(g, y, v, C, ld, steps, objective, precision, 0.0, 0.9,
                         deco.DECO_KERNEL_GLOBAL | (s << 16), alpha_cols, steps_cols)
        assert torch.equal(got[0][:, :C], ref[0][:, :C])
        assert torch.equal(got[1][:, :C], ref[1][:, :C])
        assert torch.equal(got[0][:, C:], y[:, C:])   # padding columns untouched


# ------------------------------------------------------ batch + population

def _batch_case():
    graphs = [gg.ba_graph(n, 4, 30 + i) for i, n in enumerate([60, 90, 120, 75, 200])]
    graphs.append(gg.torus_graph(8, 6, 3))            # a +-1 graph in the same batch
    return graphs


@pytest.mark.parametrize("kernel", [deco.DECO_KERNEL_GLOBAL, deco.DECO_KERNEL_ONCHIP])
def test_batch_population_matches_oracle(kernel):
    graphs = _batch_case()
    handles = [deco.graph_from(g) for g in graphs]
    batch = deco.deco_create_batch(handles)
    B, P, rounds = 16, 4, 4
    pop = deco.population(candidates=P, rounds=rounds, t_lo=30, t_hi=60, e_lo=-3.0, e_hi=-1.5, momentum=0.9,
                          lifts=(1, 2))
    p = deco.params(init=deco.DECO_INIT_IDI_HALF_UNIFORM, kernel=kernel)
    res, best, ex = deco.deco_solve_batch(batch, B, p, pop, 2024, want_assignment=True, want_round_cuts=True)
    ref = O.solve_batch_population(graphs, B, P, rounds, [1, 2], 30, 60, -3.0, -1.5, 0.9,
                                   O.Params(init="idi_half_uniform"), 2024)
    for r in range(rounds):
        agree = np.mean(ex["round_cuts"][r] == ref.round_cuts[r])
        assert agree >= 0.99, (r, agree)
        np.testing.assert_array_equal(ex["round_scores"][r], ref.round_scores[r])
    np.testing.assert_array_equal(ex["final_T"], ref.final_T)
    np.testing.assert_array_equal(ex["final_e"], ref.final_e.astype(np.float32))
    assert list(best) == ref.best_cuts
    # the returned assignment realises every graph's best cut
    off = 0
    for g, bc in zip(graphs, best):
        assert O.cut_value(g, ex["assignment"][off:off + g.n]) == bc
        off += g.n


def test_batch_kernels_and_replay_agree():
    graphs = _batch_case()
    batch = deco.deco_create_batch([deco.graph_from(g) for g in graphs])
    pop = deco.population(candidates=4, rounds=5, t_lo=20, t_hi=20, e_lo=-2.5, e_hi=-1.5, lifts=(1, 2))
    outs = []
    for kernel in (deco.DECO_KERNEL_GLOBAL, deco.DECO_KERNEL_ONCHIP):
        res, best, ex = deco.deco_solve_batch(batch, 16, deco.params(init=deco.DECO_INIT_IDI, kernel=kernel), pop, 5,
                                              want_round_cuts=True)
        outs.append((best.tolist(), ex["round_cuts"].tobytes(), ex["round_scores"].tobytes()))
    assert outs[0] == outs[1]


@pytest.mark.parametrize("precision", [deco.DECO_PREC_FP32, deco.DECO_PREC_BF16])
@pytest.mark.parametrize("sizes", [(150, 300), (300, 1150)])
def test_batch_onchip_items_equal_the_union_per_step_kernel(precision, sizes):
    # 40 graphs whose union does not fit in shared memory while every member
    # does: the default runs one on-chip launch (row-pair form) with an item
    # per (graph, 128-byte column slab) -- with graphs of up to 1 150 rows in
    # the lean form (momentum in global memory, replica refreshed from L2); the
    # per-step kernel over the union performs the same FP32 operations in the
    # same order
    rng = np.random.default_rng(77)
    graphs = [gg.ba_graph(int(n), 4, 700 + i) for i, n in enumerate(rng.integers(sizes[0], sizes[1], 40))]
    batch = deco.deco_create_batch([deco.graph_from(g) for g in graphs])
    pop = deco.population(candidates=4, rounds=3, t_lo=20, t_hi=50, e_lo=-2.5, e_hi=-1.5, momentum=0.9,
                          lifts=(1, 2))
    outs = []
    for kernel in (deco.DECO_KERNEL_GLOBAL, deco.DECO_KERNEL_AUTO):
        p = deco.params(init=deco.DECO_INIT_IDI, precision=precision, kernel=kernel)
        res, best, ex = deco.deco_solve_batch(batch, 64, p, pop, 9, want_round_cuts=True)
        outs.append((best.tolist(), ex["round_cuts"].tobytes(), ex["round_scores"].tobytes(), res.kernel_launches))
    assert outs[0][:3] == outs[1][:3]
    assert outs[1][3] < outs[0][3]   # one launch per phase instead of one per step


def test_batch_rejects_bad_population():
    batch = deco.deco_create_batch([deco.graph_from(gg.ba_graph(50, 4, 1))])
    with pytest.raises(deco.DecoError) as ei:
        deco.deco_solve_batch(batch, 10, deco.params(), deco.population(candidates=4), 0)   # 10 % 4 != 0
    assert ei.value.status == deco.DECO_ERR_ARG


# ------------------------------------------------------------------ autotuner

@pytest.mark.parametrize("precision", [deco.DECO_PREC_FP32, deco.DECO_PREC_BF16])
def test_autotune_records_a_shape_that_keeps_results(precision):
    g = gg.torus_graph(40, 20, 2)
    G = deco.graph_from(g)
    C, ld = 256, 256
    sel, us = deco.deco_autotune(G, C, precision, deco.DECO_OBJ_LAPLACIAN, 0.9, 10)
    assert us > 0.0
    kind = sel & 0x3
    assert kind in (deco.DECO_KERNEL_GLOBAL, deco.DECO_KERNEL_ONCHIP)
    y, v = _phase_blocks(g, C, ld, precision, 9, 0.9)
    ref = _run_phase(g, y, v, C, ld, 6, O.OBJ_LAPLACIAN, precision, 0.003, 0.9, deco.DECO_KERNEL_GLOBAL)
    # the tuned shape is used by DECO_KERNEL_AUTO on the same handle
    y2, v2 = y.clone(), v.clone()
    a = deco.step_args(deco.DECO_OBJ_LAPLACIAN, precision, 0.003, 0.9)
    deco.deco_run_phase(G, C, ld, y2, v2, 6, a, deco.DECO_KERNEL_AUTO)
    torch.cuda.synchronize()
    assert torch.equal(y2[:, :C], ref[0][:, :C]) and torch.equal(v2[:, :C], ref[1][:, :C])
    with pytest.raises(deco.DecoError):
        deco.deco_set_tuning(G, C, precision, 0x7777)
    deco.deco_set_tuning(G, C, precision, deco.DECO_KERNEL_GLOBAL)
