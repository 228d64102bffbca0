"""Parity of the greedy comparator and the 1-flip local search with the oracle.

Both are integer algorithms with deterministic rules (the greedy orderings are
a Philox-keyed Feistel bijection, the local search flips the local maxima of
(gain, -index) among positive-gain neighbours), so every assignment, cut and
round count must be identical.
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


def signed_graph(n, p, seed, choices=(-2.0, -1.0, 1.0, 3.0)):
    g = gg.er_graph(n, p, seed)
    rng = np.random.default_rng(seed + 5)
    u, v, _ = g.edges()
    return gg.from_edges(n, u, v, rng.choice(np.array(choices), size=u.size))


GRAPHS = {
    "er100": lambda: gg.er_graph(100, 0.1, 0),
    "ba": lambda: gg.ba_graph(300, 4, 3),
    "torus": lambda: gg.torus_graph(12, 9, 2),
    "signed": lambda: signed_graph(120, 0.08, 4),
    "isolated": lambda: gg.from_edges(50, [0, 1, 2], [1, 2, 3]),
    "single": lambda: gg.from_edges(1, [], []),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_greedy_bit_exact(name):
    g = GRAPHS[name]()
    B, seed = 37, 2024
    z = torch.zeros(g.n * B, dtype=torch.uint8, device=DEV)
    cuts = torch.zeros(B, dtype=torch.int64, device=DEV)
    deco.deco_greedy(deco.graph_from(g), B, seed, z, cuts)
    torch.cuda.synchronize()
    Zr, cr = O.greedy_batch(g, B, seed)
    np.testing.assert_array_equal(z.cpu().numpy().reshape(g.n, B), Zr)
    np.testing.assert_array_equal(cuts.cpu().numpy(), cr)
    w = g.edges()[2]
    if (w >= 0).all():
        assert (2 * cr >= w.sum()).all()   # the greedy guarantee (non-negative weights)


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("rounds", [1, 3, 200])
def test_local_search_bit_exact(name, rounds):
    g = GRAPHS[name]()
    B = 70                                   # three words, ragged
    Z = (np.random.default_rng(6).random((g.n, B)) < 0.5).astype(np.uint8)
    z = torch.from_numpy(Z.reshape(-1).copy()).to(DEV)
    cuts = torch.zeros(B, dtype=torch.int64, device=DEV)
    r = deco.deco_local_search(deco.graph_from(g), B, z, rounds, cuts)
    Zr, rr = O.local_search(g, Z, rounds)
    np.testing.assert_array_equal(z.cpu().numpy().reshape(g.n, B), Zr)
    np.testing.assert_array_equal(cuts.cpu().numpy(), O.cut_values(g, Zr))
    assert r == rr
    if rr < rounds:
        assert not (O.flip_gains(g, Zr) > 0).any()


def test_local_search_zero_rounds_keeps_the_vectors():
    g = GRAPHS["er100"]()
    Z = (np.random.default_rng(1).random((g.n, 8)) < 0.5).astype(np.uint8)
    z = torch.from_numpy(Z.reshape(-1).copy()).to(DEV)
    assert deco.deco_local_search(deco.graph_from(g), 8, z, 0) == 0
    np.testing.assert_array_equal(z.cpu().numpy().reshape(g.n, 8), Z)


def test_solve_with_local_search_matches_oracle():
    g = gg.er_graph(100, 0.1, 0)
    x0 = gg.uniform_x0(g.n, 64, 0)
    sched = [(1, 300, 0.01, 0.0), (2, 60, 0.002, 0.0)]
    p = deco.params(init=deco.DECO_INIT_EXPLICIT, local_search=40)
    res, z, pc = deco.deco_solve(deco.graph_from(g), 64, sched, p, 5, x0=x0)
    ref = O.solve(g, 64, [O.Phase(*s) for s in sched], O.Params(init="explicit", local_search=40), 5, x0=x0)
    assert res.best_cut == ref.best_cut == O.cut_value(g, z)
    for k in range(len(sched)):
        assert np.mean(pc[k] == ref.phase_cuts[k]) >= 0.99
    # the polish never lowers a rounded vector's cut (first phase: same starts)
    plain, _, pc0 = deco.deco_solve(deco.graph_from(g), 64, sched, deco.params(init=deco.DECO_INIT_EXPLICIT), 5, x0=x0)
    assert (pc[0] >= pc0[0]).all()


@pytest.mark.parametrize("opt", [dict(local_search=5), dict(phase_init=1), dict(eval_every=10)])
def test_solve_only_options_rejected_in_batched_solves(opt):
    graphs = [gg.ba_graph(60, 4, 1), gg.ba_graph(80, 4, 2)]
    batch = deco.deco_create_batch([deco.graph_from(g) for g in graphs])
    with pytest.raises(deco.DecoError) as ei:
        deco.deco_solve_batch(batch, 8, deco.params(**opt), deco.population(candidates=2, rounds=1), 0)
    assert ei.value.status == deco.DECO_ERR_UNSUPPORTED


def test_greedy_and_local_search_at_eval_size():
    # the learned-proposal evaluation graph ER(5000, 0.002): sampled greedy runs
    # against the oracle
    g = gg.er_graph(5000, 0.002, 9002)
    G = deco.graph_from(g)
    B = 256
    z = torch.zeros(g.n * B, dtype=torch.uint8, device=DEV)
    cuts = torch.zeros(B, dtype=torch.int64, device=DEV)
    deco.deco_greedy(G, B, 77, z, cuts)
    Zg = z.cpu().numpy().reshape(g.n, B)
    for b in (0, 101, 255):
        zr = O.greedy_maxcut(g, O.feistel_order(g.n, b, 77))
        np.testing.assert_array_equal(Zg[:, b], zr)
    np.testing.assert_array_equal(cuts.cpu().numpy(), O.cut_values(g, Zg))
    # the local search of 256 seeded columns, in full
    Z0 = (np.random.default_rng(12).random((g.n, B)) < 0.5).astype(np.uint8)
    z = torch.from_numpy(Z0.reshape(-1).copy()).to(DEV)
    r = deco.deco_local_search(G, B, z, 500, cuts)
    Zr, rr = O.local_search(g, Z0, 500)
    assert r == rr
    np.testing.assert_array_equal(z.cpu().numpy().reshape(g.n, B), Zr)
    np.testing.assert_array_equal(cuts.cpu().numpy(), O.cut_values(g, Zr))


def test_budget_solve_repetitions_match_oracle():
    g = gg.er_graph(100, 0.1, 0)
    G = deco.graph_from(g)
    sched = [(1, 200, 0.01, 0.9), (2, 50, 0.001, 0.9)]
    p = deco.params(init=deco.DECO_INIT_IDI)
    res, z, reps = deco.deco_solve_budget(G, 64, sched, p, 21, budget_ms=1e9, max_repeats=3)
    assert reps == 3
    cut, zr = O.solve_repeated(g, 64, [O.Phase(*s) for s in sched], O.Params(init="idi"), 21, 3)
    assert res.best_cut == cut == O.cut_value(g, z)


def test_budget_solve_stops_on_time_and_resumes():
    g = gg.er_graph(800, 0.06, 1)
    G = deco.graph_from(g)
    sched = [(1, 100, 0.01, 0.9)]
    p = deco.params(init=deco.DECO_INIT_IDI)
    r0, z0, n0 = deco.deco_solve_budget(G, 128, sched, p, 5, budget_ms=0.0)
    assert n0 == 1 and r0.best_cut == O.cut_value(g, z0)
    r1, z1, n1 = deco.deco_solve_budget(G, 128, sched, p, 6, budget_ms=5.0, max_repeats=1000)
    assert 1 <= n1 < 1000 and r1.device_ms >= 5.0
    # resume from the first call's assignment: never below it
    r2, z2, n2 = deco.deco_solve_budget(G, 128, sched, p, 7, budget_ms=0.0, warm=z0)
    assert r2.best_cut >= r0.best_cut and r2.best_cut == O.cut_value(g, z2)
