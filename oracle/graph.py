"""The graph model of Sec. 2 and the matrices built from it.

* G = (V, E, w): connected, undirected, weighted; self-loops and edge
  directions are ignored (Sec. 6.3).  Parallel edges are read as parallel
  conductances: their weights add.
* L = D - A with D_ii = sum_j w_ij (Sec. 2).
* B: m x n incidence matrix with B(e, u) = +1, B(e, v) = -1 for e = {u, v};
  the orientation is free (Sec. 5.2); the reading taken here is u = min(e),
  v = max(e).  Edge ids are the ranks of (min, max) in lexicographic order.
* W = diag(w) (Sec. 5.2).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csgraph


class NotConnected(ValueError):
    pass


@dataclass
class Graph:
    n: int
    u: np.ndarray  # (m,) int64, u < v, lexicographically sorted
    v: np.ndarray  # (m,) int64
    w: np.ndarray  # (m,) float64 > 0

    @property
    def m(self) -> int:
        return int(self.u.size)


def canonical_graph(n, src, dst, w=None, check_connected=True) -> Graph:
    """Edge list -> canonical G: drop self-loops, orient every edge as
    (min, max), sum the weights of repeated pairs, sort lexicographically.
    Raises NotConnected for a disconnected graph (the method assumes a
    connected G, Sec. 2)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    w = np.ones(src.size) if w is None else np.asarray(w, dtype=np.float64)
    if n < 2:
        raise ValueError("need n >= 2")
    if src.size and (src.min() < 0 or dst.min() < 0 or src.max() >= n or dst.max() >= n):
        raise ValueError("endpoint out of range")
    if np.any(~np.isfinite(w)) or np.any(w <= 0):
        raise ValueError("weights must be positive and finite")
    keep = src != dst
    a = np.minimum(src, dst)[keep]
    b = np.maximum(src, dst)[keep]
    ww = w[keep]
    key = a * n + b
    uniq, inv = np.unique(key, return_inverse=True)
    wsum = np.zeros(uniq.size)
    np.add.at(wsum, inv, ww)
    g = Graph(n=int(n), u=uniq // n, v=uniq % n, w=wsum)
    if check_connected and not is_connected(g):
        raise NotConnected("graph is not connected")
    return g


def is_connected(g: Graph) -> bool:
    a = sp.coo_matrix((np.ones(g.m), (g.u, g.v)), shape=(g.n, g.n))
    ncomp, _ = csgraph.connected_components(a, directed=False)
    return ncomp == 1


def adjacency(g: Graph) -> sp.csr_matrix:
    """Symmetric weighted adjacency A (Sec. 2)."""
    r = np.concatenate([g.u, g.v])
    c = np.concatenate([g.v, g.u])
    x = np.concatenate([g.w, g.w])
    return sp.csr_matrix((x, (r, c)), shape=(g.n, g.n))


def degrees(g: Graph) -> np.ndarray:
    """D_ii = sum_j w_ij (Sec. 2)."""
    d = np.zeros(g.n)
    np.add.at(d, g.u, g.w)
    np.add.at(d, g.v, g.w)
    return d


def laplacian(g: Graph) -> sp.csr_matrix:
    """L = D - A (Sec. 2), sparse FP64."""
    return (sp.diags(degrees(g)) - adjacency(g)).tocsr()


def laplacian_dense(g: Graph) -> np.ndarray:
    return laplacian(g).toarray()


def incidence(g: Graph) -> sp.csr_matrix:
    """B (m x n): row e has +1 at min(e) and -1 at max(e) (Sec. 5.2)."""
    e = np.arange(g.m)
    r = np.concatenate([e, e])
    c = np.concatenate([g.u, g.v])
    x = np.concatenate([np.ones(g.m), -np.ones(g.m)])
    return sp.csr_matrix((x, (r, c)), shape=(g.m, g.n))
