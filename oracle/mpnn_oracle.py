"""CPU oracle of the learned initial-mean proposal (message-passing network).

TEST INFRASTRUCTURE ONLY (imported by the tests, the smoke check and the
benchmark's CPU leg, never by the product library).

The paper's method is training-free; this proposal is the optional learned
start that feeds the same solver (a Gaussian start around a given mean h,
Sec. 4.2).  It is written here in FP64 NumPy, step by step:

  features   x_v = [d_v / Delta, d_v / mean(d), 1 / sqrt(d_v + 1), r_v1 .. r_v5]
             d_v = |N(v)|, r ~ U(-1, 1) from Philox counter (v, j, 0, STREAM_FEAT)
  layer 0    H0 = relu(X W0 + b0)                                 (8 -> 64)
  layer l    M = D^-1 A H_{l-1} (mean of the neighbours; 0 for isolated nodes)
             H_l = relu(H_{l-1} Ws_l + M Wn_l + b_l)              (64 -> 64), l = 1..L
  head       o = H_L wo + bo;   proposal h = tanh(o)
  loss       per graph, with targets t = 2 z* - 1 from the solver's best
             assignment and the sign symmetry of a cut (z and 1 - z cut the
             same edges): L_g = min(mean_v softplus(-t_v o_v), mean_v softplus(t_v o_v));
             the loss of a batch is the mean of L_g over its graphs
  Adam       beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected
  init       W ~ U(-a, a), a = sqrt(6 / (fan_in + fan_out)) from Philox counter
             (flat index, 0, 0, STREAM_PARAM); biases 0

Parameter layout (one flat FP32 vector): W0 [F x H], b0 [H], then for each
message-passing layer Ws [H x H], Wn [H x H], b [H], then wo [H], bo [1].
"""
from __future__ import annotations

import math

import numpy as np

from .deco_oracle import adjacency, degree_count, draw_uniform, seed_key

STREAM_FEAT = 4
STREAM_PARAM = 5
F_IN = 8
N_RANDOM = 5


def param_shapes(hidden: int = 64, layers: int = 3, f_in: int = F_IN):
    shapes = [("W0", (f_in, hidden)), ("b0", (hidden,))]
    for l in range(1, layers + 1):
        shapes += [(f"Ws{l}", (hidden, hidden)), (f"Wn{l}", (hidden, hidden)), (f"b{l}", (hidden,))]
    shapes += [("wo", (hidden,)), ("bo", (1,))]
    return shapes


def n_params(hidden: int = 64, layers: int = 3) -> int:
    return sum(int(np.prod(s)) for _, s in param_shapes(hidden, layers))


def unpack(theta, hidden=64, layers=3):
    out, o = {}, 0
    for name, shp in param_shapes(hidden, layers):
        k = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + k], dtype=np.float64).reshape(shp)
        o += k
    return out


def pack(p, hidden=64, layers=3):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in param_shapes(hidden, layers)])


def init_params(seed: int, hidden: int = 64, layers: int = 3) -> np.ndarray:
    """Xavier-uniform weights, zero biases, rounded to FP32 (the stored type)."""
    theta = np.zeros(n_params(hidden, layers))
    o = 0
    for name, shp in param_shapes(hidden, layers):
        k = int(np.prod(shp))
        if len(shp) == 2 or name == "wo":
            fan_in, fan_out = (shp[0], shp[1]) if len(shp) == 2 else (hidden, 1)
            a = math.sqrt(6.0 / (fan_in + fan_out))
            u = draw_uniform(np.arange(o, o + k, dtype=np.uint64), 0, 0, STREAM_PARAM, seed)
            theta[o:o + k] = ((2.0 * u - 1.0) * a).astype(np.float32)
        o += k
    return theta


def features(g, seed: int) -> np.ndarray:
    """Node features (see module docstring); FP32 values, as stored."""
    deg = degree_count(g).astype(np.float64)
    delta = max(float(deg.max()), 1.0) if g.n else 1.0
    mean = float(deg.mean()) if g.n else 1.0
    mean = mean if mean > 0 else 1.0
    X = np.zeros((g.n, F_IN))
    X[:, 0] = deg / delta
    X[:, 1] = deg / mean
    X[:, 2] = 1.0 / np.sqrt(deg + 1.0)
    v = np.arange(g.n, dtype=np.uint64)
    for j in range(N_RANDOM):
        X[:, 3 + j] = 2.0 * draw_uniform(v, j, 0, STREAM_FEAT, seed) - 1.0
    return X.astype(np.float32).astype(np.float64)


def _relu(x):
    return np.maximum(x, 0.0)


def forward(theta, g, X, hidden=64, layers=3):
    """Returns (o, cache); h = tanh(o) is the proposal."""
    p = unpack(theta, hidden, layers)
    A = adjacency(g)
    deg = degree_count(g).astype(np.float64)
    dinv = np.where(deg > 0, 1.0 / np.maximum(deg, 1.0), 0.0)
    cache = {"X": X, "pre": [], "H": [], "M": [], "dinv": dinv, "A": A}
    pre0 = X @ p["W0"] + p["b0"]
    H = _relu(pre0)
    cache["pre"].append(pre0)
    cache["H"].append(H)
    for l in range(1, layers + 1):
        M = dinv[:, None] * (A @ H)
        pre = H @ p[f"Ws{l}"] + M @ p[f"Wn{l}"] + p[f"b{l}"]
        H = _relu(pre)
        cache["M"].append(M)
        cache["pre"].append(pre)
        cache["H"].append(H)
    o = H @ p["wo"] + p["bo"][0]
    return o, cache


def softplus(x):
    return np.maximum(x, 0.0) + np.log1p(np.exp(-np.abs(x)))


def sigmoid(x):
    return np.where(x >= 0, 1.0 / (1.0 + np.exp(-np.where(x >= 0, x, 0))),
                    np.exp(np.where(x < 0, x, 0)) / (1.0 + np.exp(np.where(x < 0, x, 0))))


def loss_and_dout(o, z, gid=None, n_graphs=1):
    """Sign-symmetric logistic loss (module docstring) and dL/do."""
    o = np.asarray(o, dtype=np.float64)
    t = 2.0 * np.asarray(z, dtype=np.float64) - 1.0
    gid = np.zeros(o.size, dtype=np.int64) if gid is None else np.asarray(gid)
    dout = np.zeros_like(o)
    total = 0.0
    for gi in range(n_graphs):
        sel = gid == gi
        ng = int(sel.sum())
        lp = float(np.mean(softplus(-t[sel] * o[sel])))
        lm = float(np.mean(softplus(t[sel] * o[sel])))
        s = 1.0 if lp <= lm else -1.0
        total += min(lp, lm)
        # d softplus(-s t o) / do = -s t sigmoid(-s t o)
        dout[sel] = -s * t[sel] * sigmoid(-s * t[sel] * o[sel]) / (ng * n_graphs)
    return total / n_graphs, dout


def backward(theta, cache, dout, hidden=64, layers=3):
    """Gradient of the loss with respect to the flat parameter vector."""
    p = unpack(theta, hidden, layers)
    grads = {}
    H = cache["H"][-1]
    grads["wo"] = H.T @ dout
    grads["bo"] = np.array([dout.sum()])
    dH = np.outer(dout, p["wo"])
    A, dinv = cache["A"], cache["dinv"]
    for l in range(layers, 0, -1):
        pre = cache["pre"][l]
        dpre = dH * (pre > 0)
        Hprev = cache["H"][l - 1]
        M = cache["M"][l - 1]
        grads[f"Ws{l}"] = Hprev.T @ dpre
        grads[f"Wn{l}"] = M.T @ dpre
        grads[f"b{l}"] = dpre.sum(axis=0)
        dM = dpre @ p[f"Wn{l}"].T
        # M = D^-1 A H  =>  dH = A^T D^-1 dM = A (D^-1 dM), A symmetric
        dH = dpre @ p[f"Ws{l}"].T + A @ (dinv[:, None] * dM)
    dpre0 = dH * (cache["pre"][0] > 0)
    grads["W0"] = cache["X"].T @ dpre0
    grads["b0"] = dpre0.sum(axis=0)
    return pack(grads, hidden, layers)


def loss_grad(theta, g, X, z, gid=None, n_graphs=1, hidden=64, layers=3):
    o, cache = forward(theta, g, X, hidden, layers)
    L, dout = loss_and_dout(o, z, gid, n_graphs)
    return L, backward(theta, cache, dout, hidden, layers)


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One bias-corrected Adam update (t counts from 1)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
