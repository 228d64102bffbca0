"""CPU oracle for the DECO MaxCut hot path (arXiv 2509.18612).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check in
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this module.  The product path (the C-ABI library and its Python binding)
never calls it, and this module never calls the product path: the two share
no code.  Inputs come from ``graphgen`` (seeded generators, no arithmetic of
the method).

Everything is plain FP64 NumPy / scipy.sparse, written to be checked by eye
against the paper:

* cut value ........................ Def. 1, Eq. (1)
* relaxed objective / gradient ..... Eq. (QUCO), Eq. (6)  (paper form, x in [-1,1])
* multilinear objective ............ F(x) = sum_{(i,j) in E} w_ij (x_i + x_j - 2 x_i x_j)
                                     on [0,1]^n, gradient d - 2 A x (the box form
                                     of the same cut relaxation used by the solver's
                                     default objective)
* projected gradient ascent ........ Eq. (7) unlifted, Eq. (10) lifted, with
                                     heavy-ball momentum (Sec. 4.2 says momentum
                                     PGA is used in practice)
* binarisation ..................... Eq. (5) unlifted (x_v > 0), Eq. (11) lifted
                                     (row sum >= 0)
* pQUCO / pLUCO / pDECO ............ Algorithms 1, 2, 3
* DUI / IDI initialisation ......... Eq. (12), Sec. 4.1.2
* batch Gaussian initialisation .... Sec. 4.2 (first batch around h with
                                     covariance eta I, later batches around the
                                     previous batch's best binary vector),
                                     initial vectors scaled down (Sec. 5)
* evolution-based search ........... Sec. 4.3
* Philox4x32-10 counter RNG ........ Salmon, Moraes, Dror & Shaw, "Parallel
                                     random numbers: as easy as 1, 2, 3" (SC'11)

Readings of places where the paper is ambiguous are listed where they are
used (marked "Reading:").

State convention.  The iterate is kept in *centred* coordinates y in [-1,1]
for both objectives; for the multilinear objective the oracle converts to
x = (1 + y) / 2 and takes the step literally in x (an independent check on the
device's centred algebra), then converts back.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import scipy.sparse as sp

OBJ_MULTILINEAR01 = "multilinear01"
OBJ_LAPLACIAN = "laplacian"

# Stream identifiers of the counter-based generator (fourth counter word).
STREAM_INIT = 0      # per-(row, column) draws of the starting block
STREAM_IDI = 1       # per-node coins of the IDI mean
STREAM_DUI = 2       # per-node uniform draw of the DUI mean
STREAM_EVOLVE = 3    # perturbations of the evolution-based search
STREAM_ORDER = 6     # random vertex orderings of the greedy comparator


# ----------------------------------------------------------------------------
# Graph algebra (Sec. 2 notation: A adjacency, D degree matrix, L = D - A)
# ----------------------------------------------------------------------------

def adjacency(g) -> sp.csr_matrix:
    """Weighted symmetric adjacency A as FP64 CSR (unit weights when None)."""
    w = np.ones(g.nnz) if g.weights is None else np.asarray(g.weights, dtype=np.float64)
    return sp.csr_matrix((w, g.col_idx.astype(np.int64), g.row_ptr.astype(np.int64)),
                         shape=(g.n, g.n))


def net_degree(g) -> np.ndarray:
    """d_v = sum_u w_vu.

    Reading: the paper defines d_v for unweighted graphs (Sec. 2).  For signed
    weights the net weighted degree keeps L e_n = 0 and y^T L y = 4 Cut at
    binary y, which is what Eq. (QUCO) relies on.
    """
    return np.asarray(adjacency(g).sum(axis=1)).ravel()


def degree_count(g) -> np.ndarray:
    """|N(v)|, the number of incident edges (used by DUI and IDI, Sec. 4.1)."""
    return np.diff(g.row_ptr).astype(np.int64)


def laplacian(g) -> sp.csr_matrix:
    """L = D - A (Eq. QUCO)."""
    return (sp.diags(net_degree(g)) - adjacency(g)).tocsr()


# ----------------------------------------------------------------------------
# Cut value (Def. 1, Eq. 1) and objectives
# ----------------------------------------------------------------------------

def cut_value(g, z) -> int:
    """Cut(S) for S = {v : z_v = 1}: every crossing edge counted once, weighted.

    Eq. (1) sums 1{(v,u) in E} over v in S, u not in S; with weights each
    crossing edge contributes w_uv.  Returned as a Python int (exact).
    """
    z = np.asarray(z).astype(bool)
    u, v, w = g.edges()
    cross = z[u] != z[v]
    return int(np.sum(w[cross].astype(np.int64)))


def cut_values(g, Z) -> np.ndarray:
    """Cut value of every column of a binary block Z (n x B), int64."""
    Z = np.asarray(Z).astype(bool)
    u, v, w = g.edges()
    cross = Z[u, :] != Z[v, :]
    return (w.astype(np.int64)[:, None] * cross).sum(axis=0).astype(np.int64)


def objective_quco(g, y) -> float:
    """f(x) = x^T L x on [-1,1]^n (Eq. QUCO)."""
    y = np.asarray(y, dtype=np.float64)
    return float(y @ (laplacian(g) @ y))


def objective_multilinear(g, x) -> float:
    """F(x) = sum over unordered edges of w (x_i + x_j - 2 x_i x_j), x in [0,1]^n."""
    x = np.asarray(x, dtype=np.float64)
    u, v, w = g.edges()
    return float(np.sum(w * (x[u] + x[v] - 2.0 * x[u] * x[v])))


def grad_quco(g, y) -> np.ndarray:
    """g(x) = L x (Eq. 6).

    Reading: the true gradient of x^T L x is 2 L x; the paper writes L x and
    the step size absorbs the factor 2.  We keep the paper's literal form.
    """
    return laplacian(g) @ np.asarray(y, dtype=np.float64)


def grad_multilinear(g, x) -> np.ndarray:
    """dF/dx = d - 2 A x for the multilinear objective."""
    x = np.asarray(x, dtype=np.float64)
    return net_degree(g) - 2.0 * (adjacency(g) @ x)


# ----------------------------------------------------------------------------
# Projected gradient ascent step (Eq. 7 / Eq. 10) with momentum (Sec. 4.2)
# ----------------------------------------------------------------------------

def pga_step(g, Y, alpha, objective=OBJ_MULTILINEAR01, V=None, momentum=0.0,
             active=None, A=None, d=None):
    """One projected gradient ascent step on every column of the block Y.

    Y: n x C centred iterate in [-1,1].  alpha: scalar or per-column array.
    V: momentum buffer (same shape, None = zeros).  active: optional bool[C];
    inactive columns are left unchanged (their step budget is exhausted).

    Laplacian form (Eq. 7 / 10):   J = L Y;  V <- mu V + J;  Y <- Proj[-1,1](Y + alpha V)
    Multilinear form, taken in x = (1+Y)/2:
                                   G = d - 2 A X;  V <- mu V + G;  X <- Proj[0,1](X + alpha V)

    Reading (momentum): heavy ball, projection after the step, V reset at
    the start of each phase (Sec. 4.2 and 5 give only "momentum 0.9").
    Reading (evaluation order): the product with A is formed first and the
    step size applied afterwards, alpha * (L Y), never (alpha L) Y.
    """
    Y = np.asarray(Y, dtype=np.float64)
    n, C = Y.shape
    A = adjacency(g) if A is None else A
    d = net_degree(g) if d is None else d
    alpha = np.broadcast_to(np.asarray(alpha, dtype=np.float64), (C,))
    if V is None:
        V = np.zeros_like(Y)
    if objective == OBJ_LAPLACIAN:
        J = d[:, None] * Y - (A @ Y)
        Vn = momentum * V + J
        Yn = np.clip(Y + alpha[None, :] * Vn, -1.0, 1.0)
    elif objective == OBJ_MULTILINEAR01:
        X = (1.0 + Y) / 2.0
        G = d[:, None] - 2.0 * (A @ X)
        Vn = momentum * V + G
        Xn = np.clip(X + alpha[None, :] * Vn, 0.0, 1.0)
        Yn = 2.0 * Xn - 1.0
    else:
        raise ValueError(objective)
    if active is not None:
        act = np.asarray(active, dtype=bool)[None, :]
        Yn = np.where(act, Yn, Y)
        Vn = np.where(act, Vn, V)
    return Yn, Vn


# ----------------------------------------------------------------------------
# Binarisation (Eq. 5 / Eq. 11), best of the batch (the rounding and selection steps of Alg. 1 and Alg. 2)
# ----------------------------------------------------------------------------

def binarize(Y, lift: int = 1) -> np.ndarray:
    """z from the iterate.

    lift == 1: z_v = 1{x_v > 0} (Eq. 5), strict.
    lift >= 2: columns b*l .. b*l+l-1 belong to init b; z_v = 1{sum_i X_{v,i} >= 0}
               (Eq. 11), non-strict, summed in order i = 0 .. l-1 in FP64.
    """
    Y = np.asarray(Y, dtype=np.float64)
    if lift == 1:
        return (Y > 0.0).astype(np.uint8)
    n, C = Y.shape
    if C % lift:
        raise ValueError("column count not a multiple of the lift")
    s = np.zeros((n, C // lift))
    for i in range(lift):
        s = s + Y[:, i::lift]
    return (s >= 0.0).astype(np.uint8)


def best_of(cuts) -> int:
    """argmax over inits, lowest index on ties (the selection step of Alg. 1; reading for ties)."""
    cuts = np.asarray(cuts)
    return int(np.flatnonzero(cuts == cuts.max())[0])


# ----------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11) and the draws built on it
# ----------------------------------------------------------------------------

_PHILOX_M0 = 0xD2511F53
_PHILOX_M1 = 0xCD9E8D57
_PHILOX_W0 = 0x9E3779B9
_PHILOX_W1 = 0xBB67AE85
_MASK32 = 0xFFFFFFFF


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on counter (c0..c3) with key (k0, k1); arrays of uint32.

    One round: (c0,c1,c2,c3) -> (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2),
                                  hi(M0*c0) ^ c3 ^ k1, lo(M0*c0));
    the key is advanced by the Weyl constants (W0, W1) between rounds.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK32
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = np.uint64(k0 & _MASK32)
    k1 = np.uint64(k1 & _MASK32)
    m0 = np.uint64(_PHILOX_M0)
    m1 = np.uint64(_PHILOX_M1)
    mask = np.uint64(_MASK32)
    sh = np.uint64(32)
    for r in range(10):
        p0 = m0 * c0
        p1 = m1 * c2
        n0 = (p1 >> sh) ^ c1 ^ k0
        n1 = p1 & mask
        n2 = (p0 >> sh) ^ c3 ^ k1
        n3 = p0 & mask
        c0, c1, c2, c3 = n0, n1, n2, n3
        k0 = np.uint64((int(k0) + _PHILOX_W0) & _MASK32)
        k1 = np.uint64((int(k1) + _PHILOX_W1) & _MASK32)
    return c0, c1, c2, c3


def seed_key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & _MASK32, (seed >> 32) & _MASK32


def u01_from_bits(x) -> np.ndarray:
    """Uniform in (0,1): (2 * (x >> 9) + 1) * 2^-24, exact in FP32 and FP64."""
    k = (np.asarray(x, dtype=np.uint64) >> np.uint64(9)).astype(np.float64)
    return (2.0 * k + 1.0) * 2.0 ** -24


def draw_words(rows, cols, phase, stream, seed):
    """Philox output words for counter (row, col, phase, stream), key = seed."""
    k0, k1 = seed_key(seed)
    return philox4x32_10(rows, cols, np.uint64(phase), np.uint64(stream), k0, k1)


def draw_uniform(rows, cols, phase, stream, seed) -> np.ndarray:
    """U(0,1) from word 0."""
    x0, _, _, _ = draw_words(rows, cols, phase, stream, seed)
    return u01_from_bits(x0)


def draw_normal(rows, cols, phase, stream, seed) -> np.ndarray:
    """N(0,1) by the Box-Muller transform of words 0 and 1:
    sqrt(-2 ln u1) cos(2 pi u2)."""
    x0, x1, _, _ = draw_words(rows, cols, phase, stream, seed)
    u1 = u01_from_bits(x0)
    u2 = u01_from_bits(x1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ----------------------------------------------------------------------------
# Initialisation (Sec. 4.1, Sec. 4.2, Sec. 5)
# ----------------------------------------------------------------------------

def degree_moments(g):
    """Mean and population standard deviation of |N(v)| (Sec. 4.1.2).

    Computed from integer power sums so that every implementation obtains
    the same FP64 values: mean = S1/n, var = (n S2 - S1^2) / n^2.
    """
    deg = degree_count(g)
    n = g.n
    s1 = int(deg.sum())
    s2 = int((deg * deg).sum())
    mean = float(s1) / float(n)
    var = float(n * s2 - s1 * s1) / float(n * n)
    return mean, math.sqrt(var)


def important_set(g, beta: float = 0.2) -> np.ndarray:
    """I = {v : d_v > mean + beta * sigma} (Sec. 4.1.2), as a bool mask."""
    mean, sigma = degree_moments(g)
    thresh = mean + float(np.float32(beta)) * sigma
    return degree_count(g).astype(np.float64) > thresh


def idi_mean(g, seed: int, phase: int = 0, beta: float = 0.2) -> np.ndarray:
    """h_IDI in {-1,+1}^n (Sec. 4.1.2).

    Important nodes take p_i ~ U{-1,1}.  a, b are the indicators of the two
    sides of the important nodes; an unimportant node i compares (A a)_i with
    (A b)_i: +1 if (A a)_i < (A b)_i, -1 if greater, a fair coin if equal.

    Reading: A is the weighted adjacency (signed graphs included); a and b are
    zero outside I.  Coins: bit 0 of word 2 for p_i, bit 0 of word 3 for the
    tie (counter = (i, 0, phase, STREAM_IDI)); bit 1 means +1.
    """
    n = g.n
    v = np.arange(n, dtype=np.uint64)
    _, _, x2, x3 = draw_words(v, 0, phase, STREAM_IDI, seed)
    coin_p = np.where((x2 & np.uint64(1)) == 1, 1.0, -1.0)
    coin_t = np.where((x3 & np.uint64(1)) == 1, 1.0, -1.0)
    imp = important_set(g, beta)
    p = np.where(imp, coin_p, 0.0)
    a = (p == 1.0).astype(np.float64)
    b = (p == -1.0).astype(np.float64)
    A = adjacency(g)
    Aa = A @ a
    Ab = A @ b
    r = np.where(Aa < Ab, 1.0, np.where(Aa > Ab, -1.0, coin_t))
    return np.where(imp, p, r)


def dui_mean(g, seed: int, phase: int = 0) -> np.ndarray:
    """h_DUI,v ~ U[-(1 - d_v/Delta), (1 - d_v/Delta)] (Eq. 12).

    Reading: a node with d_v = Delta gets 0 (the interval collapses).
    The uniform draw is u = word 0 of counter (v, 0, phase, STREAM_DUI).
    """
    deg = degree_count(g).astype(np.float64)
    delta = float(deg.max()) if g.n else 1.0
    halfwidth = 1.0 - deg / delta
    v = np.arange(g.n, dtype=np.uint64)
    u = draw_uniform(v, 0, phase, STREAM_DUI, seed)
    return (2.0 * u - 1.0) * halfwidth


def gaussian_block(mean, C: int, seed: int, phase: int, eta: float, scale: float,
                   col_offset: int = 0) -> np.ndarray:
    """Y[v,c] = Proj[-1,1]( s * (h_v + sqrt(eta) * N(0,1)) ) (Sec. 4.2, Sec. 5).

    Reading: the down-scaling of the initial vectors (Sec. 5) applies to the
    whole Gaussian draw (mean plus noise); the projection keeps the result in
    the box.
    Noise for column c uses counter (v, c + col_offset, phase, STREAM_INIT).
    eta and scale are given as FP32 values and widened to FP64.
    """
    mean = np.asarray(mean, dtype=np.float64)
    n = mean.shape[0]
    rows = np.arange(n, dtype=np.uint64)[:, None]
    cols = (np.arange(C, dtype=np.uint64) + np.uint64(col_offset))[None, :]
    eps = draw_normal(rows, cols, phase, STREAM_INIT, seed)
    eta = float(np.float32(eta))
    scale = float(np.float32(scale))
    return np.clip(scale * (mean[:, None] + math.sqrt(eta) * eps), -1.0, 1.0)


def uniform_block(n: int, C: int, seed: int, phase: int, half_width: float,
                  col_offset: int = 0) -> np.ndarray:
    """Y[v,c] = half_width * (2 u - 1) with u from counter (v, c, phase, STREAM_INIT)."""
    rows = np.arange(n, dtype=np.uint64)[:, None]
    cols = (np.arange(C, dtype=np.uint64) + np.uint64(col_offset))[None, :]
    u = draw_uniform(rows, cols, phase, STREAM_INIT, seed)
    return float(np.float32(half_width)) * (2.0 * u - 1.0)


# ----------------------------------------------------------------------------
# pQUCO / pLUCO / pDECO (Algorithms 1-3)
# ----------------------------------------------------------------------------

@dataclass
class Phase:
    lift: int          # 1 = unlifted (Alg. 1), l >= 2 = lifted (Alg. 2)
    steps: int
    alpha: float
    momentum: float = 0.0


@dataclass
class Params:
    objective: str = OBJ_MULTILINEAR01
    init: str = "uniform"     # uniform | idi | dui | idi_half_uniform | explicit | mean
    eta: float = 0.8
    scale: float = 1e-4
    beta: float = 0.2
    uniform_half_width: float = 1.0
    mean: Optional[np.ndarray] = None   # for init == "mean" (e.g. a learned proposal)
    local_search: int = 0     # rounds of 1-flip local search on every phase's rounded vectors (0: off)
    phase_init: str = "best"  # later phases: "best" (around 2 z* - 1, Sec. 4.2) | "fresh" (like phase 0)
    eval_every: int = 0       # > 0: also round after steps E, 2E, ... < T_k (best-so-far tracking)


@dataclass
class SolveResult:
    best_cut: int
    best_init: int
    best_phase: int
    assignment: np.ndarray
    phase_cuts: List[np.ndarray] = field(default_factory=list)
    phase_best: List[int] = field(default_factory=list)
    final_Y: Optional[np.ndarray] = None


def initial_block(g, B: int, lift: int, params: Params, seed: int, x0=None, phase: int = 0) -> np.ndarray:
    """Starting block of the first phase (n x B*lift, centred coordinates);
    with phase k > 0 the same kind of start with every random draw taken with
    phase index k in its counter (fresh later phases)."""
    n = g.n
    C = B * lift
    if params.init == "explicit" and phase > 0:
        raise ValueError("fresh later phases need a drawn initialisation")
    if params.init == "explicit":
        X0 = np.asarray(x0, dtype=np.float64)
        if X0.shape != (n, C):
            raise ValueError("explicit start must be n x (B*lift)")
        return 2.0 * X0 - 1.0 if params.objective == OBJ_MULTILINEAR01 else X0.copy()
    if params.init == "uniform":
        return uniform_block(n, C, seed, phase, params.uniform_half_width)
    if params.init == "idi":
        return gaussian_block(idi_mean(g, seed, phase, params.beta), C, seed, phase, params.eta, params.scale)
    if params.init == "dui":
        return gaussian_block(dui_mean(g, seed, phase), C, seed, phase, params.eta, params.scale)
    if params.init == "mean":
        return gaussian_block(params.mean, C, seed, phase, params.eta, params.scale)
    if params.init == "idi_half_uniform":
        # Reading: inits [0, B/2) are IDI-centred Gaussians, inits [B/2, B) are
        # uniform draws scaled like the Gaussian ones.
        Y = uniform_block(n, C, seed, phase, params.scale)
        half = (B // 2) * lift
        Y[:, :half] = gaussian_block(idi_mean(g, seed, phase, params.beta), half, seed, phase,
                                     params.eta, params.scale)
        return Y
    raise ValueError(params.init)


def run_phase(g, Y, phase: Phase, objective: str, alpha_cols=None, active_steps=None):
    """T_k projected gradient steps on the whole block (the step loop of Alg. 1 / Alg. 2)."""
    A = adjacency(g)
    d = net_degree(g)
    V = np.zeros_like(Y)
    alpha = phase.alpha if alpha_cols is None else alpha_cols
    for t in range(phase.steps):
        active = None if active_steps is None else (np.asarray(active_steps) > t)
        Y, V = pga_step(g, Y, alpha, objective, V, phase.momentum, active=active, A=A, d=d)
    return Y


def solve(g, B: int, phases: Sequence[Phase], params: Params, seed: int, x0=None,
          keep_final=False) -> SolveResult:
    """pDECO (Alg. 3) over an explicit phase list; pQUCO/pLUCO are one-phase lists.

    Phase 0 starts from ``initial_block``.  Every later phase starts from
    Gaussian draws around 2 z* - 1 with z* the best binary vector of the
    previous phase (Sec. 4.2: later batches are centred on the best binary
    vector of the previous batch; Alg. 3 feeds pLUCO's result to pQUCO).
    After each phase the block is binarised (Eq. 5 / 11), every init's cut is
    evaluated (Eq. 1) and the best is kept; the global best is the first
    strictly larger cut over phases (ties keep the earlier phase).
    params.phase_init == "fresh": later phases start like phase 0, with phase
    index k in the random draws.  params.eval_every = E > 0: the block is also
    binarised after steps E, 2E, ... < T_k of every phase; those cuts compete
    for the global best (ties keep the earlier rounding), while phase_cuts and
    the next phase's centre stay the final roundings'.
    """
    best = {"cut": None, "init": -1, "phase": -1, "z": None}

    def rounding(Yk, k, lift):
        Z = binarize(Yk, lift)
        if params.local_search > 0:
            Z, _ = local_search(g, Z, params.local_search)
        cuts = cut_values(g, Z)
        b = best_of(cuts)
        if best["cut"] is None or int(cuts[b]) > best["cut"]:
            best.update(cut=int(cuts[b]), init=b, phase=k, z=Z[:, b].copy())
        return Z, cuts, b

    phase_cuts, phase_best = [], []
    prev_best_z = None
    Y = None
    for k, ph in enumerate(phases):
        if k == 0 or params.phase_init == "fresh":
            Y = initial_block(g, B, ph.lift, params, seed, x0, phase=k)
        else:
            h = 2.0 * prev_best_z.astype(np.float64) - 1.0
            Y = gaussian_block(h, B * ph.lift, seed, k, params.eta, params.scale)
        if params.eval_every > 0:
            A, d = adjacency(g), net_degree(g)
            V = np.zeros_like(Y)
            for t in range(ph.steps):
                Y, V = pga_step(g, Y, ph.alpha, params.objective, V, ph.momentum, A=A, d=d)
                if t + 1 < ph.steps and (t + 1) % params.eval_every == 0:
                    rounding(Y, k, ph.lift)
        else:
            Y = run_phase(g, Y, ph, params.objective)
        Z, cuts, b = rounding(Y, k, ph.lift)
        phase_cuts.append(cuts)
        phase_best.append(b)
        prev_best_z = Z[:, b].copy()
    best_cut, best_init, best_phase, assignment = best["cut"], best["init"], best["phase"], best["z"]
    return SolveResult(best_cut=best_cut, best_init=best_init, best_phase=best_phase,
                       assignment=assignment, phase_cuts=phase_cuts, phase_best=phase_best,
                       final_Y=Y if keep_final else None)


def solve_repeated(g, B: int, phases: Sequence[Phase], params: Params, seed: int, repeats: int, warm=None):
    """pDECO repeated ``repeats`` times (Alg. 3 repeats its schedule while its
    time budget lasts; here the budget is a number of repetitions).
    Repetition r solves with seed + r; it starts as ``params.init`` says, or
    around 2 z* - 1 (init "mean") once a best vector z* exists (the warm
    start, or an earlier repetition's best).  Returns (best cut, best z)."""
    from dataclasses import replace
    best_z = None if warm is None else np.asarray(warm, dtype=np.uint8).copy()
    best_cut = -1 if warm is None else cut_value(g, best_z)
    for r in range(repeats):
        p = params if best_z is None else replace(params, init="mean", mean=2.0 * best_z.astype(np.float64) - 1.0)
        res = solve(g, B, phases, p, seed + r)
        if res.best_cut > best_cut:
            best_cut, best_z = res.best_cut, res.assignment.copy()
    return best_cut, best_z


# ----------------------------------------------------------------------------
# Evolution-based hyper-parameter search (Sec. 4.3)
# ----------------------------------------------------------------------------

def evolve(exponents, steps, scores, eps, eps_prime, t_lo: int, t_hi: int,
           e_lo: float = -4.0, e_hi: float = -1.0):
    """One evolution round on a population of (e, T) pairs, alpha = 10^e.

    Rank by score (descending; ties keep the lower index), keep the top half,
    replace the bottom half by perturbed copies of the kept members:
        e' = Proj[e_lo, e_hi](e + 0.2 eps),  eps ~ N(0,1)
        T' = floor(T0 (1 + 0.2 (2 eps' - 1))),  eps' ~ U(0,1)
    Reading: the j-th worst member is replaced from the j-th best kept member
    (pairing unstated in the paper); T' is clipped to [t_lo, t_hi] (the
    paper clips only e').  eps, eps_prime: one value per replaced member.
    """
    e = np.asarray(exponents, dtype=np.float64)
    T = np.asarray(steps, dtype=np.int64)
    s = np.asarray(scores)
    P = e.size
    order = sorted(range(P), key=lambda i: (-s[i], i))
    keep = order[: P // 2]
    drop = order[P // 2:]
    ne, nT = e.copy(), T.copy()
    for j, victim in enumerate(drop[::-1]):
        src = keep[j % len(keep)]
        ne[victim] = min(max(e[src] + 0.2 * eps[j], e_lo), e_hi)
        t = math.floor(T[src] * (1.0 + 0.2 * (2.0 * eps_prime[j] - 1.0)))
        nT[victim] = min(max(t, t_lo), t_hi)
    return ne, nT, keep


def population_init(P: int, t_lo: int, t_hi: int, e_lo: float, e_hi: float, seed: int):
    """Initial population of Sec. 4.3: T ~ U{T_l, T_u}, e ~ U[e_l, e_u], alpha = 10^e.

    Draws: counter (k, 0, 0, STREAM_EVOLVE) for candidate k; e from word 0
    (e_l + (e_u - e_l) u), T from word 1 (T_l + word mod (T_u - T_l + 1)).
    """
    k = np.arange(P, dtype=np.uint64)
    x0, x1, _, _ = draw_words(k, 0, 0, STREAM_EVOLVE, seed)
    e = e_lo + (e_hi - e_lo) * u01_from_bits(x0)
    T = t_lo + (x1.astype(np.int64) % (t_hi - t_lo + 1))
    return e.astype(np.float64), T.astype(np.int64)


def population_perturbations(n_replaced: int, round_idx: int, seed: int):
    """eps ~ N(0,1) and eps' ~ U(0,1) of the j-th replaced member in a round:
    counter (j, round, 1, STREAM_EVOLVE); eps by Box-Muller of words 0 and 1,
    eps' from word 2."""
    j = np.arange(n_replaced, dtype=np.uint64)
    x0, x1, x2, _ = draw_words(j, round_idx, 1, STREAM_EVOLVE, seed)
    u1, u2 = u01_from_bits(x0), u01_from_bits(x1)
    eps = np.array([math.sqrt(-2.0 * math.log(a)) * math.cos(2.0 * math.pi * b) for a, b in zip(u1, u2)])
    return eps, u01_from_bits(x2)


def alpha_of(e) -> np.ndarray:
    """alpha = 10^e, evaluated with the C library's pow and rounded to FP32 (the
    step size the iteration uses)."""
    return np.array([np.float32(math.pow(10.0, float(x))) for x in np.atleast_1d(e)], dtype=np.float64)


@dataclass
class BatchResult:
    best_cuts: List[int]
    round_cuts: List[np.ndarray]      # per round: n_graphs x B
    round_scores: List[np.ndarray]    # per round: P
    populations: List[tuple]          # per round: (e, T) used in that round
    final_e: np.ndarray = None
    final_T: np.ndarray = None


def solve_batch_population(graphs, B: int, P: int, rounds: int, lifts, t_lo: int, t_hi: int,
                           e_lo: float, e_hi: float, momentum: float, params: Params, seed: int) -> BatchResult:
    """Batched pDECO with the evolution-based search of Sec. 4.3, one shared
    population for all graphs of the batch.

    Candidate k owns starts [k B/P, (k+1) B/P); in a round it runs T_k steps
    with alpha_k = 10^{e_k} (per-column step size and step budget).  Round r
    uses lift lifts[r mod len(lifts)] (Alg. 3 alternation).  Its starts are
    drawn per graph (round 0: params.init; later rounds: Gaussian around
    2 z* - 1 of that graph's best binary vector of the previous round,
    Sec. 4.2).  After the round every start is rounded and cut per graph; the
    score of candidate k is the sum over graphs of the best cut among its
    starts; the population then evolves (``evolve``) with T' clipped to
    [t_lo, t_hi].  Readings: the population is shared by the batch (one
    hyper-parameter set for a dataset); random draws as in
    ``population_init`` / ``population_perturbations``; graph i draws its
    starts with key seed + i, counters indexed by its own rows, and the
    phase index of those counters is the round index.
    """
    e, T = population_init(P, t_lo, t_hi, e_lo, e_hi, seed)
    per = B // P
    best = [None] * len(graphs)
    prev_z = [None] * len(graphs)
    res = BatchResult(best_cuts=[], round_cuts=[], round_scores=[], populations=[])
    for r in range(rounds):
        lift = lifts[r % len(lifts)]
        C = B * lift
        cand_of_col = (np.arange(C) // lift) // per
        alpha_cols = alpha_of(e)[cand_of_col]
        steps_cols = T[cand_of_col]
        res.populations.append((e.copy(), T.copy()))
        cuts_r = np.zeros((len(graphs), B), dtype=np.int64)
        for gi, g in enumerate(graphs):
            gseed = (seed + gi) & 0xFFFFFFFFFFFFFFFF
            if r == 0:
                Y = initial_block(g, B, lift, params, gseed)
            else:
                Y = gaussian_block(2.0 * prev_z[gi].astype(np.float64) - 1.0, C, gseed, r, params.eta, params.scale)
            Y = run_phase(g, Y, Phase(lift, int(steps_cols.max()), 0.0, momentum), params.objective,
                          alpha_cols=alpha_cols, active_steps=steps_cols)
            Z = binarize(Y, lift)
            cuts = cut_values(g, Z)
            cuts_r[gi] = cuts
            b = best_of(cuts)
            prev_z[gi] = Z[:, b].copy()
            if best[gi] is None or int(cuts[b]) > best[gi]:
                best[gi] = int(cuts[b])
        scores = np.array([int(cuts_r[:, k * per:(k + 1) * per].max(axis=1).sum()) for k in range(P)])
        res.round_cuts.append(cuts_r)
        res.round_scores.append(scores)
        if r + 1 < rounds:
            n_rep = P - P // 2
            eps, epsp = population_perturbations(n_rep, r, seed)
            e, T, _ = evolve(e, T, scores, eps, epsp, t_lo, t_hi, e_lo, e_hi)
    res.best_cuts = best
    res.final_e, res.final_T = e, T
    return res


# ----------------------------------------------------------------------------
# Exhaustive and greedy references
# ----------------------------------------------------------------------------

def brute_force_maxcut(g):
    """Exact maximum cut by enumerating all 2^(n-1) assignments with z_0 = 0 (n <= 22)."""
    n = g.n
    if n > 22:
        raise ValueError("brute force limited to n <= 22")
    if n <= 1:
        return 0, np.zeros(n, dtype=np.uint8)
    u, v, w = g.edges()
    w = w.astype(np.int64)
    best, best_code = None, 0
    total = 1 << (n - 1)
    chunk = 1 << 16
    for start in range(0, total, chunk):
        codes = np.arange(start, min(total, start + chunk), dtype=np.int64)
        bits = ((codes[:, None] << 1) >> np.arange(n, dtype=np.int64)[None, :]) & 1
        cross = bits[:, u] != bits[:, v]
        vals = cross.astype(np.int64) @ w
        i = int(np.argmax(vals))
        if best is None or vals[i] > best:
            best, best_code = int(vals[i]), int(codes[i])
    z = (((best_code << 1) >> np.arange(n)) & 1).astype(np.uint8)
    return best, z


def greedy_maxcut(g, order) -> np.ndarray:
    """Sahni-Gonzalez greedy (App. C.1): place vertices in the given order on the
    side that maximises the cut among already placed vertices."""
    A = adjacency(g).tocsr()
    side = np.full(g.n, -1, dtype=np.int64)
    for k, v in enumerate(order):
        if k == 0:
            side[v] = 1
            continue
        lo, hi = A.indptr[v], A.indptr[v + 1]
        nb = A.indices[lo:hi]
        wt = A.data[lo:hi]
        placed = side[nb] >= 0
        gain1 = float(np.sum(wt[placed & (side[nb] == 0)]))   # put v in S (side 1)
        gain0 = float(np.sum(wt[placed & (side[nb] == 1)]))   # put v in S-bar
        side[v] = 1 if gain1 >= gain0 else 0
    return side.astype(np.uint8)


def feistel_order(n: int, b: int, seed: int) -> np.ndarray:
    """A random ordering of the n vertices for greedy run b (App. C.1 draws a
    fresh random ordering for every run).

    The ordering is the bijection k -> pi_b(k) of [0, n): a 4-round balanced
    Feistel network on [0, 4^h) (h >= 1 bits per half, 4^h >= n) whose round i
    maps (L, R) to (R, L xor (F_i(R) mod 2^h)), F_i(R) = word 0 of Philox
    counter (R, b, i, STREAM_ORDER), key seed; values >= n are walked through
    the network again until they fall in [0, n) (cycle walking keeps the map a
    bijection).  Returns order[k] = pi_b(k).
    """
    h = 1
    while 4 ** h < n:
        h += 1
    mask = np.uint64((1 << h) - 1)
    k0, k1 = seed_key(seed)

    def net(x):
        L, R = x >> np.uint64(h), x & mask
        for i in range(4):
            f, _, _, _ = philox4x32_10(R, np.uint64(b), np.uint64(i), np.uint64(STREAM_ORDER), k0, k1)
            L, R = R, L ^ (f.astype(np.uint64) & mask)
        return (L << np.uint64(h)) | R

    x = np.arange(n, dtype=np.uint64)
    todo = np.ones(n, dtype=bool)
    while todo.any():
        x[todo] = net(x[todo])
        todo = x >= np.uint64(n)
    return x.astype(np.int64)


def greedy_batch(g, B: int, seed: int):
    """B runs of the greedy algorithm (App. C.1), run b on ordering
    ``feistel_order(n, b, seed)``.  Returns (Z n x B uint8, cuts int64[B])."""
    Z = np.zeros((g.n, B), dtype=np.uint8)
    for b in range(B):
        Z[:, b] = greedy_maxcut(g, feistel_order(g.n, b, seed))
    return Z, cut_values(g, Z)


def flip_gains(g, Z) -> np.ndarray:
    """Change of the cut when node v alone changes side, per column:
    gain_v = sum_u w_vu s_u s_v with s = 1 - 2 z (the edges to same-side
    neighbours become cut, the cut edges stop being cut)."""
    S = 1.0 - 2.0 * np.asarray(Z, dtype=np.float64)
    return S * (adjacency(g) @ S)


def local_search(g, Z, max_rounds: int):
    """1-flip local search on every column of Z (n x B, 0/1), at most
    ``max_rounds`` rounds.  A round computes every gain and flips every node
    whose gain is positive and beats the gain of each neighbour with a
    positive gain (ties: the lower index wins); those nodes are pairwise
    non-adjacent, so the cut grows by the sum of their gains.  Stops early
    when no node has a positive gain (a 1-flip local optimum).  Returns
    (Z', rounds that flipped at least one node).
    """
    Z = np.array(Z, dtype=np.uint8, copy=True)
    # every (node v, neighbour u) pair of the adjacency
    v = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    u = g.col_idx.astype(np.int64)
    done = 0
    for _ in range(max_rounds):
        G = flip_gains(g, Z)
        pos = G > 0
        # u beats v in column c when G[u,c] > 0 and (G[u,c] > G[v,c] or (equal and u < v))
        gu, gv = G[u], G[v]
        beats = (gu > 0) & ((gu > gv) | ((gu == gv) & (u < v)[:, None]))
        beaten = np.zeros_like(pos)
        np.logical_or.at(beaten, v, beats)
        flip = pos & ~beaten
        if not flip.any():
            break
        Z[flip] ^= 1
        done += 1
    return Z, done

