"""Pins of the CPU oracle of the learned proposal (message-passing network):
finite-difference gradients, brute-force mean aggregation, the sign symmetry
of the loss, the closed form of Adam's first step, feature and initialiser
ranges."""
import math

import numpy as np
import pytest

import graphgen as gg
from oracle import mpnn_oracle as M


def _small():
    g = gg.ba_graph(40, 3, 2)
    X = M.features(g, 5)
    z = gg.random_binary(g.n, 1, 3)[:, 0]
    return g, X, z


def test_gradient_matches_central_differences():
    g, X, z = _small()
    hidden, layers = 8, 2
    rng = np.random.default_rng(0)
    theta = M.init_params(1, hidden, layers) + rng.normal(scale=0.05, size=M.n_params(hidden, layers))
    L, grad = M.loss_grad(theta, g, X, z, hidden=hidden, layers=layers)
    idx = rng.choice(theta.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        lp, _ = M.loss_grad(theta + e, g, X, z, hidden=hidden, layers=layers)
        lm, _ = M.loss_grad(theta - e, g, X, z, hidden=hidden, layers=layers)
        fd = (lp - lm) / (2 * h)
        assert fd == pytest.approx(grad[i], rel=1e-4, abs=1e-8)


def test_batch_loss_is_mean_of_graph_losses():
    ga, gb = gg.ba_graph(30, 3, 1), gg.er_graph(25, 0.2, 2)
    za, zb = gg.random_binary(ga.n, 1, 4)[:, 0], gg.random_binary(gb.n, 1, 5)[:, 0]
    oa, ob = np.random.default_rng(1).normal(size=ga.n), np.random.default_rng(2).normal(size=gb.n)
    la, _ = M.loss_and_dout(oa, za)
    lb, _ = M.loss_and_dout(ob, zb)
    gid = np.concatenate([np.zeros(ga.n, int), np.ones(gb.n, int)])
    l2, _ = M.loss_and_dout(np.concatenate([oa, ob]), np.concatenate([za, zb]), gid, 2)
    assert l2 == pytest.approx((la + lb) / 2, rel=1e-12)


def test_loss_sign_symmetry():
    rng = np.random.default_rng(3)
    o = rng.normal(size=50)
    z = rng.integers(0, 2, 50)
    l1, d1 = M.loss_and_dout(o, z)
    l2, d2 = M.loss_and_dout(o, 1 - z)
    l3, _ = M.loss_and_dout(-o, z)
    assert l1 == pytest.approx(l2) and l1 == pytest.approx(l3)
    np.testing.assert_allclose(d1, d2)
    # a perfect (or perfectly flipped) logit pattern has a small loss
    lp, _ = M.loss_and_dout(20.0 * (2 * z - 1), z)
    lf, _ = M.loss_and_dout(-20.0 * (2 * z - 1), z)
    assert lp < 1e-6 and lf < 1e-6


def test_mean_aggregation_brute_force():
    g, X, z = _small()
    theta = M.init_params(2, 8, 1)
    o, cache = M.forward(theta, g, X, 8, 1)
    H0, Mx = cache["H"][0], cache["M"][0]
    for v in range(g.n):
        nb = g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]
        ref = H0[nb].mean(axis=0) if nb.size else np.zeros(8)
        np.testing.assert_allclose(Mx[v], ref, rtol=1e-12, atol=1e-15)


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    th, m, v = M.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 0.01)
    np.testing.assert_allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)


def test_features_and_init_ranges():
    g = gg.ba_graph(200, 4, 7)
    X = M.features(g, 11)
    assert X.shape == (g.n, M.F_IN)
    assert np.all((X[:, 0] > 0) & (X[:, 0] <= 1)) and X[:, 0].max() == 1.0
    assert X[:, 1].mean() == pytest.approx(1.0, rel=1e-6)
    assert np.all((X[:, 3:] > -1) & (X[:, 3:] < 1))
    assert not np.allclose(X[:, 3:], M.features(g, 12)[:, 3:])
    theta = M.init_params(3)
    p = M.unpack(theta)
    a = math.sqrt(6.0 / (M.F_IN + 64))
    assert np.all(np.abs(p["W0"]) <= a) and np.abs(p["W0"]).max() > 0.9 * a
    assert np.all(p["b0"] == 0) and np.all(p["b1"] == 0) and p["bo"][0] == 0
    assert theta.size == M.n_params() == 8 * 64 + 64 + 3 * (2 * 64 * 64 + 64) + 65


def test_trained_proposal_beats_a_random_assignment():
    """What training buys (FP64 network): after 100 Adam steps on the best
    assignments of the plain solver on 8 small ER / BA graphs, the rounded
    proposal sign(o) of unseen graphs cuts well over the m / 2 edges a random
    assignment cuts on average (binomial spread ~1.5 % of m here); the
    untrained network proposes one side for every node (cut 0)."""
    from oracle import deco_oracle as O
    rng = np.random.default_rng(11)
    train = [gg.ba_graph(int(rng.integers(60, 121)), 4, 100 + i) if i % 2
             else gg.er_graph(int(rng.integers(60, 121)), 0.08, 100 + i) for i in range(8)]
    labels = [O.solve(g, 16, [O.Phase(1, 100, 0.02, 0.9), O.Phase(2, 30, 0.002, 0.9)], O.Params(init="idi"),
                      7 + i).assignment for i, g in enumerate(train)]
    us, vs, off = [], [], 0
    for g in train:
        u, v, _ = g.edges()
        us.append(u + off)
        vs.append(v + off)
        off += g.n
    U = gg.from_edges(off, np.concatenate(us), np.concatenate(vs))
    X = np.concatenate([M.features(g, 7) for g in train])
    z = np.concatenate(labels)
    gid = np.concatenate([np.full(g.n, i) for i, g in enumerate(train)])
    held_out = [gg.ba_graph(300, 4, 900 + s) for s in range(3)] + [gg.er_graph(300, 0.03, 950 + s) for s in range(3)]

    def cut_fractions(theta):
        fr = []
        for g in held_out:
            o, _ = M.forward(theta, g, M.features(g, 7))
            fr.append(O.cut_value(g, (o > 0).astype(np.uint8)) / g.m)
        return np.array(fr)

    theta = M.init_params(5)
    assert np.all(cut_fractions(theta) == 0.0)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    for t in range(1, 101):
        _, gr = M.loss_grad(theta, U, X, z, gid, len(train))
        theta, m, v = M.adam_step(theta, gr, m, v, t, 3e-3)
    fr = cut_fractions(theta)
    assert fr.min() > 0.56 and fr.mean() > 0.59, fr
