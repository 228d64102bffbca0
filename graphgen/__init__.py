"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only *produces inputs*: graphs in CSR form and explicit starting
points.  It contains none of the method's arithmetic (no gradient, no
projection, no rounding, no cut), so the CPU oracle and the CUDA path can both
consume its output without sharing any computation.

Graph families follow the workloads the paper evaluates (Sec. 5: Erdos-Renyi
graphs made with a G(n, p) generator, Gset-like sparse graphs) and the shapes
the build measures: a 2-D torus with +-1 weights, Barabasi-Albert graphs with
m = 4 attachments, a sparse 10^6-node ER graph and a dense ER graph.
Every generator is deterministic in its integer seed.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

__all__ = [
    "Graph", "from_edges", "er_graph", "er_graph_avg_degree", "torus_graph",
    "ba_graph", "uniform_x0", "random_binary", "graph_family",
]


@dataclasses.dataclass
class Graph:
    """Undirected graph in symmetric CSR form (both orientations stored).

    row_ptr: int32[n+1], col_idx: int32[nnz] sorted and unique within a row,
    no self loops.  weights: None for unit weights, else float64[nnz] holding
    integral values (the same value on (u,v) and (v,u)).
    """
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    weights: Optional[np.ndarray] = None
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def m(self) -> int:
        return self.nnz // 2

    def edges(self):
        """Unordered edge list (u < v) with weights (1 for unit graphs)."""
        rows = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr))
        cols = self.col_idx.astype(np.int64)
        keep = rows < cols
        w = np.ones(self.nnz) if self.weights is None else self.weights
        return rows[keep], cols[keep], w[keep]


def from_edges(n: int, u, v, w=None, name: str = "") -> Graph:
    """Build symmetric CSR from an unordered edge list (duplicates removed)."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    if u.size:
        if np.any(u == v):
            raise ValueError("self loops are not allowed")
        if u.min() < 0 or v.min() < 0 or u.max() >= n or v.max() >= n:
            raise ValueError("node index out of range")
    a = np.minimum(u, v)
    b = np.maximum(u, v)
    key = a * n + b
    key, first = np.unique(key, return_index=True)
    a = key // n
    b = key % n
    wv = None if w is None else np.asarray(w, dtype=np.float64)[first]
    rows = np.concatenate([a, b])
    cols = np.concatenate([b, a])
    order = np.lexsort((cols, rows))
    rows = rows[order]
    cols = cols[order]
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32")
    weights = None
    if wv is not None:
        weights = np.concatenate([wv, wv])[order]
    return Graph(n=n, row_ptr=row_ptr.astype(np.int32), col_idx=cols.astype(np.int32),
                 weights=weights, name=name)


def _pairs_from_linear(k: np.ndarray):
    """Map a linear index over the strict lower triangle to (row, col), row > col.

    Index k enumerates pairs (1,0), (2,0), (2,1), (3,0), ...; row r starts at
    r (r - 1) / 2.
    """
    r = np.floor((1.0 + np.sqrt(1.0 + 8.0 * k.astype(np.float64))) / 2.0).astype(np.int64)
    # repair the float estimate so that r (r-1)/2 <= k < r (r+1)/2 exactly
    r = np.where(r * (r - 1) // 2 > k, r - 1, r)
    r = np.where((r + 1) * r // 2 <= k, r + 1, r)
    c = k - r * (r - 1) // 2
    return r, c


def er_graph(n: int, p: float, seed: int, name: str = "") -> Graph:
    """G(n, p) by geometric skipping over the n(n-1)/2 candidate pairs.

    Batagelj & Brandes (2005): gaps between successive present pairs are
    geometric with parameter p, so the cost is O(n + m) instead of O(n^2).
    """
    rng = np.random.default_rng(seed)
    total = n * (n - 1) // 2
    if p <= 0.0 or total == 0:
        return from_edges(n, [], [], name=name or f"er{n}")
    if p >= 1.0:
        ks = np.arange(total, dtype=np.int64)
    else:
        chunks = []
        pos = -1
        expect = int(total * p + 10 * math.sqrt(total * p + 1) + 16)
        while True:
            gaps = rng.geometric(p, size=max(expect, 1024)).astype(np.int64)
            ks = pos + np.cumsum(gaps)
            inside = ks[ks < total]
            chunks.append(inside)
            if inside.size < ks.size:
                break
            pos = int(ks[-1])
            expect = max(1024, expect // 4)
        ks = np.concatenate(chunks)
    r, c = _pairs_from_linear(ks)
    return from_edges(n, r, c, name=name or f"er{n}_p{p:g}_s{seed}")


def er_graph_avg_degree(n: int, avg_degree: float, seed: int) -> Graph:
    """G(n, p) with p = avg_degree / (n - 1)."""
    return er_graph(n, avg_degree / (n - 1), seed, name=f"er{n}_d{avg_degree:g}_s{seed}")


def torus_graph(nx_: int, ny: int, seed: int, signed: bool = True) -> Graph:
    """2-D toroidal grid nx_ x ny (4-regular); weights +-1 drawn uniformly if signed."""
    rng = np.random.default_rng(seed)
    idx = np.arange(nx_ * ny, dtype=np.int64).reshape(nx_, ny)
    right = np.roll(idx, -1, axis=0)
    down = np.roll(idx, -1, axis=1)
    u = np.concatenate([idx.ravel(), idx.ravel()])
    v = np.concatenate([right.ravel(), down.ravel()])
    w = None
    if signed:
        w = rng.choice(np.array([-1.0, 1.0]), size=u.size)
    return from_edges(nx_ * ny, u, v, w, name=f"torus{nx_}x{ny}_s{seed}")


def ba_graph(n: int, m: int, seed: int) -> Graph:
    """Barabasi-Albert preferential attachment.

    Starts from a clique on m+1 nodes; every further node links to m distinct
    earlier nodes drawn with probability proportional to their degree.
    """
    if n <= m:
        raise ValueError("BA graph needs n > m")
    rng = np.random.default_rng(seed)
    n_edges = (m + 1) * m // 2 + (n - m - 1) * m
    us = np.empty(n_edges, dtype=np.int64)
    vs = np.empty(n_edges, dtype=np.int64)
    pool = np.empty(2 * n_edges, dtype=np.int64)   # every edge end once: degree-proportional draws
    k = 0
    for a in range(m + 1):
        for b in range(a):
            us[k], vs[k] = a, b
            pool[2 * k], pool[2 * k + 1] = a, b
            k += 1
    for node in range(m + 1, n):
        size = 2 * k
        chosen = []
        while len(chosen) < m:
            for t in pool[rng.integers(0, size, size=2 * m)]:
                t = int(t)
                if t not in chosen and len(chosen) < m:
                    chosen.append(t)
        for t in sorted(chosen):
            us[k], vs[k] = node, t
            pool[2 * k], pool[2 * k + 1] = node, t
            k += 1
    return from_edges(n, us, vs, name=f"ba{n}_m{m}_s{seed}")


def uniform_x0(n: int, cols: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Explicit starting block, n x cols float32, uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(n, cols)).astype(np.float32)


def random_binary(n: int, cols: int, seed: int) -> np.ndarray:
    """n x cols uint8 block of independent fair bits."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2, size=(n, cols), dtype=np.uint8)


def graph_family(kind: str, n: int, seed: int, **kw) -> Graph:
    """Named family helper used by tests and the benchmark."""
    if kind == "er":
        return er_graph(n, kw["p"], seed)
    if kind == "er_deg":
        return er_graph_avg_degree(n, kw["avg_degree"], seed)
    if kind == "ba":
        return ba_graph(n, kw.get("m", 4), seed)
    if kind == "torus":
        return torus_graph(kw["nx"], kw["ny"], seed, signed=kw.get("signed", True))
    raise ValueError(kind)
