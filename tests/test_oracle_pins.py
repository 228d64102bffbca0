"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a library
routine (networkx), a textbook closed form, exhaustive enumeration, an exact
finite difference, a closed-form matrix power, or a fixed-point
characterisation.  A dropped term, a wrong sign or a transposed operand in the
oracle fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest

import graphgen as gg
from oracle import deco_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_graphs():
    out = []
    with open(os.path.join(GOLDEN, "maxcut_closed_forms.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            name, n, best = parts[0], int(parts[1]), int(parts[2])
            us, vs = zip(*(tuple(map(int, e.split("-"))) for e in parts[3:]))
            out.append((name, gg.from_edges(n, us, vs, name=name), best))
    return out


def _signed_random(n, p, seed):
    g = gg.er_graph(n, p, seed)
    rng = np.random.default_rng(seed + 99)
    u, v, _ = g.edges()
    w = rng.choice([-2.0, -1.0, 1.0, 3.0], size=u.size)
    return gg.from_edges(n, u, v, w)


# ---------------------------------------------------------------- cut (Eq. 1)

@pytest.mark.parametrize("weighted", [False, True])
def test_cut_matches_networkx(weighted):
    nx = pytest.importorskip("networkx")
    for seed in range(5):
        g = _signed_random(30, 0.2, seed) if weighted else gg.er_graph(30, 0.2, seed)
        G = nx.Graph()
        G.add_nodes_from(range(g.n))
        u, v, w = g.edges()
        for a, b, c in zip(u, v, w):
            G.add_edge(int(a), int(b), weight=float(c))
        z = gg.random_binary(g.n, 4, seed + 7)
        for j in range(4):
            S = [i for i in range(g.n) if z[i, j]]
            ref = nx.cut_size(G, S, weight="weight" if weighted else None)
            assert O.cut_value(g, z[:, j]) == int(round(ref))
        assert list(O.cut_values(g, z)) == [O.cut_value(g, z[:, j]) for j in range(4)]


@pytest.mark.parametrize("name,g,best", _golden_graphs(), ids=lambda x: x if isinstance(x, str) else "")
def test_brute_force_closed_forms(name, g, best):
    val, z = O.brute_force_maxcut(g)
    assert val == best
    assert O.cut_value(g, z) == best


def test_brute_force_vs_subset_enumeration():
    nx = pytest.importorskip("networkx")
    for seed in range(3):
        g = gg.er_graph(9, 0.4, seed)
        G = nx.Graph()
        G.add_nodes_from(range(g.n))
        u, v, _ = g.edges()
        G.add_edges_from(zip(u.tolist(), v.tolist()))
        ref = max(nx.cut_size(G, S) for r in range(g.n + 1)
                  for S in itertools.combinations(range(g.n), r)) if g.m else 0
        assert O.brute_force_maxcut(g)[0] == ref


# ------------------------------------------------ objectives at binary points

def test_vertex_identity_multilinear_and_laplacian():
    for seed in range(4):
        g = _signed_random(25, 0.3, seed)
        z = gg.random_binary(g.n, 6, seed)
        for j in range(6):
            c = O.cut_value(g, z[:, j])
            x = z[:, j].astype(np.float64)
            assert O.objective_multilinear(g, x) == pytest.approx(c, abs=1e-9)
            y = 2.0 * x - 1.0
            assert O.objective_quco(g, y) == pytest.approx(4.0 * c, abs=1e-9)
            # Eq. (3) summand with each unordered edge once: sum w (y_u - y_v)^2 = 4 Cut
            u, v, w = g.edges()
            assert float(np.sum(w * (y[u] - y[v]) ** 2)) == pytest.approx(4.0 * c, abs=1e-9)


def test_laplacian_annihilates_constants():
    # Lemma 2: L e_n = 0, so constant vectors are stationary.
    g = _signed_random(40, 0.2, 3)
    for c in (-1.0, 0.3, 1.0):
        assert np.allclose(O.grad_quco(g, np.full(g.n, c)), 0.0, atol=1e-12)


def test_laplacian_psd_unit_weights():
    # Lemma 1: with non-negative weights L is PSD.
    g = gg.er_graph(40, 0.2, 5)
    ev = np.linalg.eigvalsh(O.laplacian(g).toarray())
    assert ev.min() > -1e-9


# ------------------------------------------------------- gradients (Eq. 6)

def test_gradient_finite_difference():
    rng = np.random.default_rng(0)
    for seed in range(3):
        g = _signed_random(20, 0.3, seed)
        x = rng.uniform(0.0, 1.0, g.n)
        y = rng.uniform(-1.0, 1.0, g.n)
        gm = O.grad_multilinear(g, x)
        gl = O.grad_quco(g, y)
        h = 0.125
        for v in range(g.n):
            e = np.zeros(g.n)
            e[v] = h
            # F is affine in each coordinate: the central difference is exact
            fd = (O.objective_multilinear(g, x + e) - O.objective_multilinear(g, x - e)) / (2 * h)
            assert fd == pytest.approx(gm[v], abs=1e-9)
            # f = y^T L y is quadratic: the central difference is exact and equals 2 L y
            fd = (O.objective_quco(g, y + e) - O.objective_quco(g, y - e)) / (2 * h)
            assert fd == pytest.approx(2.0 * gl[v], abs=1e-9)


# ----------------------------------------- update rule in the box interior

@pytest.mark.parametrize("objective", [O.OBJ_LAPLACIAN, O.OBJ_MULTILINEAR01])
@pytest.mark.parametrize("mu", [0.0, 0.9])
def test_interior_closed_form(objective, mu):
    g = _signed_random(24, 0.3, 11)
    rng = np.random.default_rng(1)
    Y0 = rng.uniform(-1e-6, 1e-6, size=(g.n, 3))
    alpha, T = 0.01, 12
    A = O.adjacency(g).toarray()
    L = O.laplacian(g).toarray()
    I = np.eye(g.n)
    if objective == O.OBJ_LAPLACIAN:
        M, a = L, alpha              # V <- mu V + L Y ; Y <- Y + alpha V
    else:
        M, a = -A, 2.0 * alpha       # in y = 2x-1: V <- mu V - A Y ; Y <- Y + 2 alpha V
    big = np.block([[I + a * M, a * mu * I], [M, mu * I]])
    state = np.vstack([Y0, np.zeros_like(Y0)])
    ref = np.linalg.matrix_power(big, T) @ state
    Y, V = Y0.copy(), None
    for _ in range(T):
        Y, V = O.pga_step(g, Y, alpha, objective, V, mu)
    assert np.max(np.abs(Y)) < 0.5          # stayed in the interior
    # the multilinear oracle steps in x = (1+y)/2 ~ 0.5, whose FP64 spacing is
    # 1.1e-16: compare there at that absolute precision (the entries are ~1e-6)
    atol = 1e-18 if objective == O.OBJ_LAPLACIAN else 1e-13
    np.testing.assert_allclose(Y, ref[: g.n], rtol=1e-9, atol=atol)
    assert np.max(np.abs(ref[: g.n])) > 1e4 * atol


def test_per_column_alpha_and_active_mask():
    g = gg.er_graph(30, 0.2, 2)
    rng = np.random.default_rng(3)
    Y = rng.uniform(-1, 1, size=(g.n, 4))
    a = np.array([0.01, 0.02, 0.03, 0.04])
    Yn, _ = O.pga_step(g, Y, a, O.OBJ_MULTILINEAR01, active=np.array([1, 0, 1, 0], bool))
    for j in range(4):
        if j % 2:
            assert np.array_equal(Yn[:, j], Y[:, j])
        else:
            ref, _ = O.pga_step(g, Y[:, j:j + 1], a[j], O.OBJ_MULTILINEAR01)
            assert np.array_equal(Yn[:, j], ref[:, 0])


# ----------------------------------------------- fixed points (Def. 2, Thm. 1)

def test_paper_form_every_binary_is_fixed():
    # Def. 2 / Sec. 3.1: for w >= 0, y_v (L y)_v = d_v - y_v (A y)_v >= 0 at binary
    # y, so the projected step returns the same point for any alpha > 0.
    g = gg.er_graph(10, 0.4, 1)
    for code in range(1 << g.n):
        y = np.array([1.0 if (code >> i) & 1 else -1.0 for i in range(g.n)])[:, None]
        for alpha in (1e-3, 0.3, 5.0):
            Yn, _ = O.pga_step(g, y, alpha, O.OBJ_LAPLACIAN)
            assert np.array_equal(Yn, y)


def test_multilinear_fixed_points_are_one_flip_optimal():
    # In the multilinear form a binary x is unchanged by the projected step iff
    # no single-vertex flip increases the cut (F is affine in each coordinate).
    for seed in range(3):
        g = _signed_random(9, 0.5, seed)
        for code in range(1 << g.n):
            z = np.array([(code >> i) & 1 for i in range(g.n)], dtype=np.uint8)
            y = (2.0 * z - 1.0)[:, None]
            Yn, _ = O.pga_step(g, y, 0.05, O.OBJ_MULTILINEAR01)
            fixed = np.array_equal(Yn, y)
            c = O.cut_value(g, z)
            improving = False
            for v in range(g.n):
                z2 = z.copy()
                z2[v] ^= 1
                if O.cut_value(g, z2) > c:
                    improving = True
                    break
            # a zero gain leaves the coordinate unchanged as well
            assert fixed == (not improving)


def test_multilinear_fixed_point_cut_at_least_half_edges():
    for seed in range(3):
        g = gg.er_graph(60, 0.1, seed)
        Y = gg.uniform_x0(g.n, 8, seed) * 2.0 - 1.0
        Y = O.run_phase(g, Y.astype(np.float64), O.Phase(1, 2000, 0.05), O.OBJ_MULTILINEAR01)
        Z = O.binarize(Y)
        binary = np.all(np.abs(Y) == 1.0, axis=0)
        for j in np.flatnonzero(binary):
            assert O.cut_value(g, Z[:, j]) * 2 >= g.m


def test_lifted_constant_rows_round_to_cut_zero():
    # Thm. 1 proof: X = e_n c^T rounds to a constant z, cut 0.
    g = gg.er_graph(20, 0.3, 4)
    for c in itertools.product([-1.0, 1.0], repeat=2):
        X = np.tile(np.array(c), (g.n, 1))
        z = O.binarize(X, 2)
        assert len(set(z[:, 0])) == 1
        assert O.cut_values(g, z)[0] == 0
        Xn, _ = O.pga_step(g, X, 0.1, O.OBJ_LAPLACIAN)
        assert np.array_equal(Xn, X)


def test_lifted_columns_update_independently():
    # Remark after Eq. (11): every column of X follows the unlifted update.
    g = gg.er_graph(30, 0.2, 6)
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, size=(g.n, 6))
    for obj in (O.OBJ_LAPLACIAN, O.OBJ_MULTILINEAR01):
        Xn, _ = O.pga_step(g, X, 0.02, obj)
        for j in range(6):
            yj, _ = O.pga_step(g, X[:, j:j + 1], 0.02, obj)
            np.testing.assert_array_equal(Xn[:, j], yj[:, 0])


def test_binarize_strict_and_nonstrict():
    Y = np.array([[0.0, 0.0], [1e-300, -1e-300], [-0.5, 0.5]])
    assert O.binarize(Y, 1).tolist() == [[0, 0], [1, 0], [0, 1]]
    # lifted: row sums 0, 0, 0 -> all >= 0
    assert O.binarize(Y, 2).ravel().tolist() == [1, 1, 1]
    assert O.binarize(np.array([[-1.0, 0.9]]), 2).ravel().tolist() == [0]


def test_best_of_lowest_index():
    assert O.best_of([3, 7, 7, 1]) == 1
    assert O.best_of([5]) == 0


# ------------------------------------------------------- initialisation

def test_idi_star_is_optimal():
    # a hub with k leaves: the hub is the only important node; every leaf sees
    # the hub on one side and joins the other -> the cut is all k edges.
    k = 12
    g = gg.from_edges(k + 1, [0] * k, list(range(1, k + 1)))
    imp = O.important_set(g, 0.2)
    assert imp.tolist() == [True] + [False] * k
    for seed in range(6):
        h = O.idi_mean(g, seed)
        z = (h > 0).astype(np.uint8)
        assert O.cut_value(g, z) == k
        assert np.all(h[1:] == -h[0])


def test_idi_rule_on_hand_built_graph():
    # two hubs 0 and 1 (degree 5); node 2 touches only hub 0, node 3 touches both,
    # nodes 4..7 touch hub 1 and hub 0 as listed.
    edges = [(0, 2), (0, 3), (1, 3), (0, 4), (1, 4), (1, 5), (1, 6), (0, 7)]
    g = gg.from_edges(8, *zip(*edges))
    imp = O.important_set(g, 0.2)
    assert imp.tolist() == [True, True] + [False] * 6
    for seed in range(16):
        h = O.idi_mean(g, seed)
        p0, p1 = h[0], h[1]
        assert abs(p0) == 1 and abs(p1) == 1
        assert h[2] == -p0 and h[7] == -p0 and h[5] == -p1 and h[6] == -p1
        if p0 == p1:
            assert h[3] == -p0 and h[4] == -p0
        else:
            assert abs(h[3]) == 1 and abs(h[4]) == 1   # ties: coin


def test_idi_regular_graph_all_ties():
    g = gg.torus_graph(6, 5, 0, signed=False)
    assert not O.important_set(g).any()
    hs = np.stack([O.idi_mean(g, s) for s in range(40)])
    assert set(np.unique(hs)) == {-1.0, 1.0}
    assert abs(hs.mean()) < 0.1


def test_degree_moments_match_numpy():
    g = gg.ba_graph(300, 4, 1)
    deg = O.degree_count(g).astype(np.float64)
    m, s = O.degree_moments(g)
    assert m == pytest.approx(deg.mean(), rel=1e-15)
    assert s == pytest.approx(deg.std(), rel=1e-12)


def test_dui_range():
    g = gg.ba_graph(200, 4, 2)
    deg = O.degree_count(g)
    h = O.dui_mean(g, 5)
    hw = 1.0 - deg / deg.max()
    assert np.all(np.abs(h) <= hw + 1e-15)
    assert np.all(h[deg == deg.max()] == 0.0)
    assert np.std(h / np.where(hw > 0, hw, 1)) > 0.4   # spread over the interval


def test_philox_uniform_and_normal_distribution():
    stats = pytest.importorskip("scipy.stats")
    r = np.arange(400, dtype=np.uint64)[:, None]
    c = np.arange(500, dtype=np.uint64)[None, :]
    u = O.draw_uniform(r, c, 0, O.STREAM_INIT, 1234).ravel()
    assert u.min() > 0.0 and u.max() < 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    z = O.draw_normal(r, c, 3, O.STREAM_INIT, 99).ravel()
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.01
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # distinct phases / streams / seeds give unrelated draws
    u2 = O.draw_uniform(r, c, 1, O.STREAM_INIT, 1234).ravel()
    u3 = O.draw_uniform(r, c, 0, O.STREAM_IDI, 1234).ravel()
    u4 = O.draw_uniform(r, c, 0, O.STREAM_INIT, 1235).ravel()
    for other in (u2, u3, u4):
        assert abs(np.corrcoef(u, other)[0, 1]) < 0.01


def _philox_kat():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append([int(w, 16) for w in line.split()])
    return rows


def test_philox_known_answer_vectors():
    # the generator's published known-answer vectors (tests/golden), not
    # values computed by the oracle
    rows = _philox_kat()
    assert len(rows) == 3
    for r in rows:
        ctr = [np.array([x], dtype=np.uint64) for x in r[:4]]
        out = O.philox4x32_10(*ctr, r[4], r[5])
        assert [int(o[0]) for o in out] == r[6:10]


def test_philox_round_is_a_bijection():
    # Each Philox round is invertible: lo words give c0, c2 back through the odd
    # multipliers' inverses mod 2^32, then c1, c3 follow from the hi words.
    rng = np.random.default_rng(0)
    c = rng.integers(0, 2**32, size=(4, 1000), dtype=np.uint64)
    k0, k1 = 0x12345678, 0x9ABCDEF0
    # one round = philox with the key schedule truncated: compare 10 rounds of
    # the oracle with a hand-inverted reconstruction round by round.
    M0, M1 = 0xD2511F53, 0xCD9E8D57
    inv0, inv1 = pow(M0, -1, 2**32), pow(M1, -1, 2**32)
    out = O.philox4x32_10(c[0], c[1], c[2], c[3], k0, k1)
    s = [x.astype(object) for x in out]
    keys = [((k0 + r * 0x9E3779B9) & 0xFFFFFFFF, (k1 + r * 0xBB67AE85) & 0xFFFFFFFF) for r in range(10)]
    for r in reversed(range(10)):
        kk0, kk1 = keys[r]
        n0, n1, n2, n3 = s
        c2 = np.array([(int(x) * inv1) & 0xFFFFFFFF for x in n1], dtype=object)
        c0 = np.array([(int(x) * inv0) & 0xFFFFFFFF for x in n3], dtype=object)
        c1 = np.array([((int(a) * M1) >> 32) ^ int(b) ^ kk0 for a, b in zip(c2, n0)], dtype=object)
        c3 = np.array([((int(a) * M0) >> 32) ^ int(b) ^ kk1 for a, b in zip(c0, n2)], dtype=object)
        s = [c0, c1, c2, c3]
    for i in range(4):
        assert [int(x) for x in s[i]] == [int(x) for x in c[i]]


def test_gaussian_block_scaling_and_clip():
    g = gg.er_graph(50, 0.1, 0)
    h = O.idi_mean(g, 3)
    Y = O.gaussian_block(h, 64, 3, 0, 0.8, 1e-4)
    assert np.all(np.abs(Y) <= 1.0)
    # mean over columns tracks s*h, spread tracks s*sqrt(eta)
    np.testing.assert_allclose(Y.mean(axis=1), 1e-4 * h, atol=1e-4 * 0.5)
    assert Y.std() == pytest.approx(1e-4 * math.sqrt(1.0 * 0.8 + 1.0), rel=0.1)
    big = O.gaussian_block(h, 64, 3, 0, 0.8, 10.0)
    assert np.all(np.abs(big) <= 1.0) and np.any(np.abs(big) == 1.0)


# ------------------------------------------------------------ evolution

def test_evolution_rules():
    rng = np.random.default_rng(0)
    e = rng.uniform(-4, -1, 6)
    T = rng.integers(3000, 10001, 6)
    scores = np.array([5, 9, 1, 9, 3, 7])
    eps = np.array([20.0, -20.0, 0.5])
    epsp = np.array([0.0, 1.0, 0.5])
    ne, nT, keep = O.evolve(e, T, scores, eps, epsp, 3000, 10000)
    assert keep == [1, 3, 5]                 # top half, ties by lower index
    for i in keep:
        assert ne[i] == e[i] and nT[i] == T[i]
    drop = [0, 4, 2][::-1]                    # scores 5,3,1 -> worst first is 2
    worst_first = [2, 4, 0]
    assert sorted(drop) == sorted(worst_first)
    for j, victim in enumerate(worst_first):
        src = keep[j]
        assert -4.0 <= ne[victim] <= -1.0
        assert ne[victim] == min(max(e[src] + 0.2 * eps[j], -4.0), -1.0)
        assert nT[victim] == min(max(math.floor(T[src] * (1 + 0.2 * (2 * epsp[j] - 1))), 3000), 10000)
    assert ne[worst_first[0]] == -1.0 and ne[worst_first[1]] == -4.0


def test_population_draws_in_range_and_batch_bookkeeping():
    e, T = O.population_init(64, 500, 2000, -4.0, -1.0, 7)
    assert np.all((e >= -4.0) & (e <= -1.0)) and np.all((T >= 500) & (T <= 2000))
    assert len(set(T.tolist())) > 30 and np.std(e) > 0.5
    eps, epsp = O.population_perturbations(1000, 3, 7)
    assert abs(eps.mean()) < 0.1 and abs(eps.std() - 1.0) < 0.1 and 0.0 < epsp.min() and epsp.max() < 1.0
    graphs = [gg.ba_graph(n, 4, s) for s, n in enumerate([40, 60, 50])]
    res = O.solve_batch_population(graphs, 8, 4, 3, [1, 2], 20, 40, -3.0, -1.5, 0.9,
                                   O.Params(init="idi_half_uniform"), 11)
    for gi, g in enumerate(graphs):
        # the best cut is the best over rounds and starts, never above the optimum
        assert res.best_cuts[gi] == max(int(rc[gi].max()) for rc in res.round_cuts)
        assert res.best_cuts[gi] * 2 >= g.m
    for rc, sc in zip(res.round_cuts, res.round_scores):
        for k in range(4):
            assert sc[k] == sum(int(rc[gi, 2 * k:2 * k + 2].max()) for gi in range(3))
    # rounds after the first use the evolved population
    e1, T1 = res.populations[1]
    keep = sorted(range(4), key=lambda k: (-res.round_scores[0][k], k))[:2]
    e0, T0 = res.populations[0]
    for k in keep:
        assert e1[k] == e0[k] and T1[k] == T0[k]


# -------------------------------------------------------------- solvers

def test_solve_never_beats_brute_force_and_reports_consistently():
    for seed in range(3):
        g = gg.er_graph(16, 0.35, seed)
        opt, _ = O.brute_force_maxcut(g)
        res = O.solve(g, 16, [O.Phase(1, 150, 0.05, 0.9), O.Phase(2, 60, 0.01, 0.9),
                              O.Phase(1, 150, 0.05, 0.9)],
                      O.Params(objective=O.OBJ_LAPLACIAN, init="idi"), seed)
        assert res.best_cut <= opt
        assert res.best_cut == O.cut_value(g, res.assignment)
        assert res.best_cut >= 0.8 * opt
        for k, cuts in enumerate(res.phase_cuts):
            assert cuts.max() <= res.best_cut


def test_er100_b64_shape_solve_runs():
    g = gg.er_graph(100, 0.1, 0)
    x0 = gg.uniform_x0(g.n, 64, 0)
    res = O.solve(g, 64, [O.Phase(1, 500, 0.01, 0.0)],
                  O.Params(objective=O.OBJ_MULTILINEAR01, init="explicit"), 0, x0=x0)
    assert res.best_cut * 2 >= g.m
    assert res.best_cut == O.cut_value(g, res.assignment)


def test_greedy_half_guarantee():
    for seed in range(3):
        g = gg.er_graph(80, 0.1, seed)
        z = O.greedy_maxcut(g, np.random.default_rng(seed).permutation(g.n))
        assert 2 * O.cut_value(g, z) >= g.m


# ------------------------------------------------ greedy comparator (App. C.1) and 1-flip local search

@pytest.mark.parametrize("n", [1, 2, 3, 5, 16, 17, 100, 1000])
def test_feistel_order_is_a_permutation(n):
    for b in range(3):
        o = O.feistel_order(n, b, 12345)
        assert sorted(o.tolist()) == list(range(n))


def test_feistel_orders_differ_and_spread():
    n, runs = 50, 400
    first = np.array([O.feistel_order(n, b, 9)[0] for b in range(runs)])
    # the first vertex of a run is close to uniform over the nodes
    counts = np.bincount(first, minlength=n)
    assert counts.max() < 5 * runs / n
    assert len({tuple(O.feistel_order(n, b, 9)[:10]) for b in range(20)}) == 20


def test_greedy_complete_graph_closed_form():
    # identity order on K_n alternates sides: floor(n/2) * ceil(n/2) = max cut of K_n
    for n in (2, 5, 8, 11):
        u, v = np.triu_indices(n, 1)
        g = gg.from_edges(n, u, v)
        z = O.greedy_maxcut(g, np.arange(n))
        assert O.cut_value(g, z) == (n // 2) * ((n + 1) // 2)


def _signed(n, p, seed):
    g = gg.er_graph(n, p, seed)
    u, v, _ = g.edges()
    w = np.random.default_rng(seed).choice([-2.0, -1.0, 1.0, 3.0], size=u.size)
    return gg.from_edges(n, u, v, w)


@pytest.mark.parametrize("signed", [False, True])
def test_flip_gain_is_the_cut_change_of_one_flip(signed):
    g = _signed(30, 0.2, 2) if signed else gg.er_graph(30, 0.2, 2)
    Z = (np.random.default_rng(3).random((g.n, 4)) < 0.5).astype(np.uint8)
    G = O.flip_gains(g, Z)
    base = O.cut_values(g, Z)
    for v in range(g.n):
        Zf = Z.copy()
        Zf[v] ^= 1
        np.testing.assert_array_equal(O.cut_values(g, Zf) - base, G[v].astype(np.int64))


@pytest.mark.parametrize("signed", [False, True])
def test_local_search_rounds_flip_independent_sets_and_add_their_gains(signed):
    g = _signed(80, 0.08, 4) if signed else gg.er_graph(80, 0.08, 4)
    Z = (np.random.default_rng(5).random((g.n, 6)) < 0.5).astype(np.uint8)
    u, v, _ = g.edges()
    for _ in range(30):
        G = O.flip_gains(g, Z)
        Z1, r = O.local_search(g, Z, 1)
        flipped = Z1 != Z
        if r == 0:
            assert not (G > 0).any() and not flipped.any()
            break
        assert not (flipped[u] & flipped[v]).any()                 # no two neighbours in one column
        assert (G[flipped] > 0).all()
        gain = np.where(flipped, G, 0).sum(axis=0).astype(np.int64)
        np.testing.assert_array_equal(O.cut_values(g, Z1) - O.cut_values(g, Z), gain)
        Z = Z1
    else:
        pytest.fail("local search did not converge in 30 rounds")


def test_local_search_reaches_one_flip_optima_below_the_optimum():
    for seed in range(3):
        g = gg.er_graph(14, 0.35, 20 + seed)
        opt, _ = O.brute_force_maxcut(g)
        Z = (np.random.default_rng(seed).random((g.n, 16)) < 0.5).astype(np.uint8)
        Z2, r = O.local_search(g, Z, 1000)
        assert not (O.flip_gains(g, Z2) > 0).any()
        assert (O.cut_values(g, Z2) <= opt).all() and (O.cut_values(g, Z2) >= O.cut_values(g, Z)).all()
        Z3, r3 = O.local_search(g, Z2, 10)                          # a local optimum is left alone
        assert r3 == 0 and np.array_equal(Z3, Z2)


def test_one_flip_optima_are_fixed_points_of_the_multilinear_step():
    # binaries with no improving single flip are the fixed points of the
    # multilinear PGA step (F is affine in each coordinate)
    g = gg.er_graph(40, 0.15, 6)
    Z = (np.random.default_rng(7).random((g.n, 8)) < 0.5).astype(np.uint8)
    Z, _ = O.local_search(g, Z, 1000)
    Y = 2.0 * Z - 1.0
    Yn, _ = O.pga_step(g, Y, 0.3, O.OBJ_MULTILINEAR01)
    np.testing.assert_array_equal(Yn, Y)


def test_solve_with_local_search_never_lowers_the_phase_cuts():
    g = gg.er_graph(60, 0.1, 8)
    sched = [O.Phase(1, 40, 0.01, 0.0), O.Phase(2, 10, 0.001, 0.0)]
    a = O.solve(g, 16, sched, O.Params(init="idi"), 3)
    b = O.solve(g, 16, sched[:1], O.Params(init="idi", local_search=50), 3)
    # first phase identical up to the polish: every polished cut >= the raw cut
    assert (b.phase_cuts[0] >= a.phase_cuts[0]).all()
    assert b.best_cut == O.cut_value(g, b.assignment)


def test_repeated_solve_keeps_an_optimal_warm_start_and_never_loses_ground():
    g = gg.er_graph(14, 0.35, 31)
    opt, zopt = O.brute_force_maxcut(g)
    sched = [O.Phase(1, 30, 0.01, 0.0)]
    cut, z = O.solve_repeated(g, 4, sched, O.Params(init="idi"), 2, 2, warm=zopt)
    assert cut == opt and O.cut_value(g, z) == opt
    c1, _ = O.solve_repeated(g, 4, sched, O.Params(init="idi"), 2, 1)
    c3, z3 = O.solve_repeated(g, 4, sched, O.Params(init="idi"), 2, 3)
    assert opt >= c3 >= c1 and O.cut_value(g, z3) == c3


# ---------------------------------------------------------------- intermediate roundings, fresh phases

def test_eval_every_beyond_the_phase_changes_nothing():
    g = gg.er_graph(60, 0.15, 1)
    ph = [O.Phase(1, 40, 0.01, 0.9), O.Phase(2, 10, 0.002, 0.9)]
    a = O.solve(g, 16, ph, O.Params(init="idi"), 3)
    b = O.solve(g, 16, ph, O.Params(init="idi", eval_every=40), 3)
    assert (a.best_cut, a.best_init, a.best_phase) == (b.best_cut, b.best_init, b.best_phase)
    for x, y in zip(a.phase_cuts, b.phase_cuts):
        np.testing.assert_array_equal(x, y)


def test_eval_every_best_is_the_best_of_independently_recomputed_roundings():
    # one phase from an explicit start: the rounding after m E steps is the
    # rounding of a fresh m E-step run from the same start (the iteration is
    # deterministic and its momentum starts at zero), so the best over
    # {m E < T} and the final rounding must be what solve reports, ties to
    # the earliest rounding, then the lowest start
    g = gg.er_graph(50, 0.2, 4)
    B, T, E = 12, 45, 10
    x0 = gg.uniform_x0(g.n, B, 2)
    ph = O.Phase(1, T, 0.01, 0.9)
    res = O.solve(g, B, [ph], O.Params(init="explicit", eval_every=E), 0, x0=x0)
    Y0 = 2.0 * np.asarray(x0, dtype=np.float64) - 1.0
    best = None
    for steps in list(range(E, T, E)) + [T]:
        cuts = O.cut_values(g, O.binarize(O.run_phase(g, Y0, O.Phase(1, steps, 0.01, 0.9), O.OBJ_MULTILINEAR01), 1))
        b = int(np.argmax(cuts))
        if best is None or cuts[b] > best[0]:
            best = (int(cuts[b]), b)
    assert (res.best_cut, res.best_init, res.best_phase) == (best[0], best[1], 0)
    final = O.cut_values(g, O.binarize(O.run_phase(g, Y0, ph, O.OBJ_MULTILINEAR01), 1))
    np.testing.assert_array_equal(res.phase_cuts[0], final)   # phase cuts stay the final rounding's
    assert res.best_cut >= int(final.max())


def test_fresh_later_phases_do_not_depend_on_earlier_ones():
    g = gg.er_graph(60, 0.15, 5)
    p = O.Params(init="idi_half_uniform", phase_init="fresh")
    a = O.solve(g, 16, [O.Phase(1, 30, 0.01, 0.9), O.Phase(2, 20, 0.002, 0.9)], p, 9)
    b = O.solve(g, 16, [O.Phase(1, 5, 0.02, 0.0), O.Phase(2, 20, 0.002, 0.9)], p, 9)
    np.testing.assert_array_equal(a.phase_cuts[1], b.phase_cuts[1])
    # the default (around the previous best) does depend on them
    q = O.Params(init="idi_half_uniform")
    c = O.solve(g, 16, [O.Phase(1, 30, 0.01, 0.9), O.Phase(2, 20, 0.002, 0.9)], q, 9)
    np.testing.assert_array_equal(c.phase_cuts[0], a.phase_cuts[0])
    with pytest.raises(ValueError):
        O.solve(g, 4, [O.Phase(1, 3, 0.01, 0.0), O.Phase(1, 3, 0.01, 0.0)],
                O.Params(init="explicit", phase_init="fresh"), 0, x0=gg.uniform_x0(g.n, 4, 0))


# ------------------------------------------------- starts of later phases

def _random_signs_graph():
    # unit-weight ER graph whose phase-0 starts (uniform signs) give distinct cuts
    return gg.er_graph(40, 0.2, 21)


@pytest.mark.parametrize("objective", [O.OBJ_MULTILINEAR01, O.OBJ_LAPLACIAN])
def test_later_phase_starts_at_the_best_vector_mapped_to_plus_minus_one(objective):
    # Sec. 4.2: a later batch is drawn around the previous batch's best binary
    # vector z*, mapped to the box's vertex 2 z* - 1.  With eta = 0 the draw is
    # the centre itself, scaled by s, so the next phase's start (0 steps) is
    # exactly s (2 z* - 1).  Centring on z* (0/1), on another start's vector or
    # on a negated vector fails here.
    g = _random_signs_graph()
    s = 0.25
    p = O.Params(objective=objective, init="uniform", uniform_half_width=1.0, eta=0.0, scale=s)
    res = O.solve(g, 16, [O.Phase(1, 0, 0.01), O.Phase(1, 0, 0.01)], p, 5, keep_final=True)
    cuts0 = res.phase_cuts[0]
    assert len(set(cuts0.tolist())) > 3            # the starts really differ
    b = int(np.argmax(cuts0))                       # lowest index among the best
    Y0 = O.initial_block(g, 16, 1, p, 5)
    z = (Y0[:, b] > 0).astype(np.float64)           # Eq. 5 of the best start
    expect = float(np.float32(s)) * (2.0 * z - 1.0)
    assert np.array_equal(res.final_Y, np.repeat(expect[:, None], 16, axis=1))


def test_later_lifted_phase_rounds_every_start_to_the_previous_best():
    # The same centre seen through Eq. 11: a lifted start s (2 z* - 1) in both
    # components rounds to z* in every start (row sums -2s < 0 or 2s >= 0), so
    # every start of the lifted phase cuts exactly the previous best cut.  A
    # 0/1 centre would give zero rows, which Eq. 11's >= 0 rounds to 1 (cut 0).
    g = _random_signs_graph()
    p = O.Params(init="uniform", uniform_half_width=1.0, eta=0.0, scale=1e-4)
    res = O.solve(g, 12, [O.Phase(1, 0, 0.01), O.Phase(2, 0, 0.01)], p, 9)
    assert np.all(res.phase_cuts[1] == res.phase_cuts[0].max())


def test_batch_search_later_round_rounds_every_start_to_each_graphs_best():
    # Sec. 4.2 inside the batched search (Sec. 4.3): round r > 0 of graph i is
    # drawn around 2 z_i* - 1, z_i* that graph's best vector of round r - 1.
    # With zero steps (T_l = T_u = 0) and eta = 0, a lifted round 1 rounds
    # every start of graph i to z_i*, so every cut equals graph i's round-0
    # best.  A 0/1 centre (cut 0), the worst start's vector or another graph's
    # vector fails.
    graphs = [gg.er_graph(n, 0.2, 30 + n) for n in (24, 31, 40)]
    p = O.Params(init="uniform", uniform_half_width=1.0, eta=0.0)
    res = O.solve_batch_population(graphs, 8, 4, 2, [1, 2], 0, 0, -3.0, -1.0, 0.0, p, 4)
    r0, r1 = res.round_cuts
    for gi in range(len(graphs)):
        assert len(set(r0[gi].tolist())) > 2
        assert np.all(r1[gi] == r0[gi].max())


def test_uniform_block_is_an_affine_map_of_the_uniform_draws():
    # y = h (2u - 1): the values fill (-h, h) uniformly (a map onto [0, h], a
    # missing factor 2 or h, or a shift fails the range or the KS test), and
    # column c of a block with a column offset k is column c + k of the plain
    # block (the counter's column is the global column index).
    stats = pytest.importorskip("scipy.stats")
    h = 0.375
    Y = O.uniform_block(300, 64, 17, 0, h)
    assert Y.min() > -h and Y.max() < h
    assert Y.min() < -0.99 * h and Y.max() > 0.99 * h
    assert stats.kstest(Y.ravel(), "uniform", args=(-h, 2 * h)).pvalue > 1e-4
    assert abs(Y.mean()) < 0.01 * h
    np.testing.assert_array_equal(O.uniform_block(300, 40, 17, 0, h, col_offset=24), Y[:, 24:])
    # two rows of the draw, written out: u from the pinned generator's u01 map
    u = O.draw_uniform(np.array([[3]], dtype=np.uint64), np.array([[5]], dtype=np.uint64), 0, O.STREAM_INIT, 17)
    assert Y[3, 5] == float(np.float32(h)) * (2.0 * float(u[0, 0]) - 1.0)


@pytest.mark.parametrize("lift", [1, 2])
def test_idi_plus_uniform_split_of_the_starts(lift):
    # Reading of the "IDI + random" starts: starting points [0, B/2) are
    # Gaussian around s h_IDI, starting points [B/2, B) uniform s (2u - 1);
    # with lift l a starting point owns l adjacent columns.
    stats = pytest.importorskip("scipy.stats")
    g = gg.er_graph(120, 0.08, 6)
    B, s = 40, 1e-3
    h = O.idi_mean(g, 8, 0, 0.2)
    half = (B // 2) * lift
    # eta = 0: the IDI half is exactly s h (|y| = s), the uniform half lies
    # strictly inside (-s, s) and fills it
    Y = O.initial_block(g, B, lift, O.Params(init="idi_half_uniform", eta=0.0, scale=s), 8)
    assert Y.shape == (g.n, B * lift)
    sf = float(np.float32(s))
    assert np.array_equal(Y[:, :half], np.repeat((sf * h)[:, None], half, axis=1))
    U = Y[:, half:]
    assert np.all(np.abs(U) < sf)
    assert stats.kstest(U.ravel(), "uniform", args=(-sf, 2 * sf)).pvalue > 1e-4
    # eta = 0.8: the IDI half's row means track s h, the uniform half's track 0
    Y = O.initial_block(g, 2000, lift, O.Params(init="idi_half_uniform", eta=0.8, scale=s), 8)
    half = 1000 * lift
    np.testing.assert_allclose(Y[:, :half].mean(axis=1), sf * h, atol=0.15 * sf)
    np.testing.assert_allclose(Y[:, half:].mean(axis=1), 0.0, atol=0.15 * sf)
