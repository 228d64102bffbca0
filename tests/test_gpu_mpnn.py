"""Parity of the learned-proposal kernels (through the C ABI) with the FP64
oracle: initial parameters (exact), inference, loss and full gradient, one
Adam step, batched graphs; training lowers the loss.

Tolerances: parameters are bit-exact FP32; forward outputs within 1e-5 of
the FP64 values (FP32 arithmetic over 64-wide dot products and neighbour
means); gradients within 1e-4 of the largest gradient entry plus 1e-6
(FP32 reductions over all nodes)."""
import numpy as np
import pytest

import graphgen as gg
from oracle import mpnn_oracle as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2509_18612_gb300 as deco  # noqa: E402

DEV = torch.device("cuda:0")


def signed(n, p, seed):
    g = gg.er_graph(n, p, seed)
    u, v, _ = g.edges()
    return gg.from_edges(n, u, v, np.random.default_rng(seed).choice([-1.0, 1.0], size=u.size))


GRAPHS = {"ba": lambda: gg.ba_graph(300, 4, 1), "er": lambda: gg.er_graph(250, 0.04, 2),
          "torus": lambda: gg.torus_graph(12, 10, 3), "signed": lambda: signed(150, 0.05, 4),
          "isolated": lambda: gg.from_edges(40, [0, 1, 2, 5], [1, 2, 3, 9])}


def test_initial_parameters_exact():
    m = deco.Mpnn(64, 3, 1234)
    assert m.n_params == M.n_params()
    np.testing.assert_array_equal(m.get_params().astype(np.float64), M.init_params(1234))


@pytest.mark.parametrize("name", list(GRAPHS))
def test_inference_matches_oracle(name):
    g = GRAPHS[name]()
    m = deco.Mpnn(64, 3, 7)
    theta = m.get_params().astype(np.float64)
    h = torch.zeros(g.n, device=DEV)
    m.infer(deco.graph_from(g), h, feat_seed=99)
    torch.cuda.synchronize()
    o, _ = M.forward(theta, g, M.features(g, 99))
    np.testing.assert_allclose(h.cpu().numpy(), np.tanh(o), rtol=0, atol=1e-5)
    # BF16 activations: close to the FP32 proposal
    hb = torch.zeros(g.n, device=DEV)
    m.infer(deco.graph_from(g), hb, feat_seed=99, precision=deco.DECO_PREC_BF16)
    torch.cuda.synchronize()
    assert np.max(np.abs(hb.cpu().numpy() - np.tanh(o))) < 0.05


@pytest.mark.parametrize("name", list(GRAPHS))
def test_loss_and_gradient_match_oracle(name):
    g = GRAPHS[name]()
    m = deco.Mpnn(64, 3, 8)
    rng = np.random.default_rng(5)
    theta = (m.get_params() + rng.normal(scale=0.05, size=m.n_params)).astype(np.float32)
    m.set_params(theta)
    z = gg.random_binary(g.n, 1, 6)[:, 0]
    grad = torch.zeros(m.n_params, device=DEV)
    loss = m.loss_grad(deco.graph_from(g), torch.from_numpy(z).to(DEV), grad, feat_seed=3)
    torch.cuda.synchronize()
    L, gref = M.loss_grad(theta.astype(np.float64), g, M.features(g, 3), z)
    assert loss == pytest.approx(L, rel=1e-5, abs=1e-7)
    gg_ = grad.cpu().numpy().astype(np.float64)
    tol = 1e-4 * np.max(np.abs(gref)) + 1e-6
    assert np.max(np.abs(gg_ - gref)) <= tol


def test_batch_loss_gradient_and_adam_step():
    graphs = [gg.ba_graph(120, 4, 11), gg.er_graph(90, 0.06, 12), gg.torus_graph(8, 7, 13)]
    batch = deco.deco_create_batch([deco.graph_from(g) for g in graphs])
    m = deco.Mpnn(64, 3, 21)
    theta = m.get_params().astype(np.float64)
    zs = [gg.random_binary(g.n, 1, 30 + i)[:, 0] for i, g in enumerate(graphs)]
    z = np.concatenate(zs)
    U = gg.from_edges(sum(g.n for g in graphs),
                      *[np.concatenate(x) for x in zip(*[(u + off, v + off, w) for g, off in
                                                          zip(graphs, np.cumsum([0] + [g.n for g in graphs])[:-1])
                                                          for (u, v, w) in [g.edges()]])])
    # oracle: features per graph with key feat_seed + i, one loss per graph
    X = np.concatenate([M.features(g, 40 + i) for i, g in enumerate(graphs)])
    gid = np.concatenate([np.full(g.n, i) for i, g in enumerate(graphs)])
    L, gref = M.loss_grad(theta, U, X, z, gid=gid, n_graphs=len(graphs))
    grad = torch.zeros(m.n_params, device=DEV)
    zd = torch.from_numpy(z).to(DEV)
    loss = m.loss_grad(batch, zd, grad, feat_seed=40)
    torch.cuda.synchronize()
    assert loss == pytest.approx(L, rel=1e-5)
    assert np.max(np.abs(grad.cpu().numpy() - gref)) <= 1e-4 * np.max(np.abs(gref)) + 1e-6
    # one Adam step from zero moments
    m.train_step(batch, zd, lr=1e-3, feat_seed=40)
    torch.cuda.synchronize()
    th1, _, _ = M.adam_step(theta, gref, np.zeros_like(theta), np.zeros_like(theta), 1, 1e-3)
    got = m.get_params().astype(np.float64)
    # first Adam step moves every parameter by ~lr * sign(g): compare where |g| is not tiny
    big = np.abs(gref) > 1e-3 * np.max(np.abs(gref))
    np.testing.assert_allclose(got[big], th1[big], rtol=0, atol=2e-6)


def test_training_lowers_the_loss():
    g = gg.er_graph(300, 0.03, 9)
    G = deco.graph_from(g)
    res, z, _ = deco.deco_solve(G, 64, [(1, 300, 0.02, 0.9)], deco.params(init=deco.DECO_INIT_IDI), 1,
                                want_phase_cuts=False)
    zd = torch.from_numpy(z).to(DEV)
    m = deco.Mpnn(64, 3, 3)
    losses = [m.train_step(G, zd, lr=3e-3, feat_seed=1) for _ in range(60)]
    assert losses[-1] < 0.8 * losses[0]


def test_trained_proposal_against_random_and_idi_starts():
    """What training buys, through the C ABI: the network trained for 100 Adam
    steps on the solver's best assignments of 8 small ER / BA graphs proposes,
    on unseen graphs, a sign pattern h > 0 that cuts well over the m / 2 edges
    of a random assignment (binomial spread ~1.5 % of m); before training it
    puts every node on one side (cut 0)."""
    rng = np.random.default_rng(11)
    train = [gg.ba_graph(int(rng.integers(60, 121)), 4, 100 + i) if i % 2
             else gg.er_graph(int(rng.integers(60, 121)), 0.08, 100 + i) for i in range(8)]
    handles = [deco.graph_from(g) for g in train]
    labels = []
    for i, G in enumerate(handles):
        _, z, _ = deco.deco_solve(G, 16, [(1, 100, 0.02, 0.9), (2, 30, 0.002, 0.9)],
                                  deco.params(init=deco.DECO_INIT_IDI), 7 + i, want_phase_cuts=False)
        labels.append(z)
    batch = deco.deco_create_batch(handles)
    zb = torch.from_numpy(np.concatenate(labels)).to(DEV)
    held_out = [gg.ba_graph(300, 4, 900 + s) for s in range(3)] + [gg.er_graph(300, 0.03, 950 + s) for s in range(3)]

    def cut_fractions(model):
        fr = []
        for g in held_out:
            G = deco.graph_from(g)
            h = torch.zeros(g.n, device=DEV)
            model.infer(G, h, feat_seed=7)
            torch.cuda.synchronize()
            fr.append(deco.deco_eval_cut(G, (h > 0).to(torch.uint8).cpu().numpy()) / g.m)
        return np.array(fr)

    model = deco.Mpnn(64, 3, 5)
    assert np.all(cut_fractions(model) == 0.0)
    model.train(batch, zb, steps=100, lr=3e-3, feat_seed=7)
    fr = cut_fractions(model)
    assert fr.min() > 0.56 and fr.mean() > 0.59, fr
    # Against the method's own start (IDI, Sec. 4.1.2) rounded the same way,
    # z = 1{h_IDI > 0}, averaged over four IDI draws: IDI's greedy rounding
    # cuts about 0.59 - 0.64 m on these graphs, and the trained proposal lands
    # in the same range, not clearly above it -- what the network buys here is
    # a start as good as IDI's without its greedy pass, not a better one.
    idi = []
    for g in held_out:
        G = deco.graph_from(g)
        hi = torch.zeros(g.n, device=DEV)
        vals = []
        for s in range(4):
            deco.deco_idi_mean(G, 0.2, 40 + s, 0, hi)
            torch.cuda.synchronize()
            vals.append(deco.deco_eval_cut(G, (hi > 0).to(torch.uint8).cpu().numpy()) / g.m)
        idi.append(np.mean(vals))
    idi = np.array(idi)
    assert np.all(idi > 0.56), idi
    assert fr.mean() > 0.92 * idi.mean(), (fr, idi)
