"""The pivot-sampling estimator, Sec. 5.1.

* Pivots: a uniform k-subset S of V, drawn without replacement from all of V
  (the proof of Proposition 1 averages over the k-combinations V_k of V, so
  v itself may be a pivot and then contributes d_ER(v, v) = 0).  Drawn with
  Floyd's algorithm (Bentley & Floyd, CACM 1987): for j = n-k .. n-1 draw
  t uniform in [0, j]; insert t unless already present, else insert j.
  Uniform integer in [0, j]: floor(u * (j + 1) / 2^64) for a 64-bit Philox
  word u (multiply-shift; bias below (j+1)/2^64).  Floyd step s = j - (n-k)
  uses counter (s, 0, 0, 0), key (seed, TAG_SAMPLE).
* d_ER(v, s) = p_vs(v) - p_vs(s) with L p_vs = e_v - e_s (Eq. system, Sec. 4).
* Estimate of the electrical farness of v: (n / k) sum_{s in S} d_ER(v, s).
  Reading: the proof of Proposition 1 shows that this scaled sum (not the
  bare f~(v, S)) is the unbiased estimator of sum_w d_ER(v, w).  The
  closeness estimate c~(v) = (k/n)(n-1)/f~(v, S) (Sec. 5.1) equals
  (n - 1) / [(n/k) f~(v, S)].
"""
from __future__ import annotations

import numpy as np

from .cg import cg_solve
from .dense import pinv
from .graph import Graph, laplacian
from .philox import TAG_SAMPLE, philox4x64_10_int


def uniform_below(u64: int, bound: int) -> int:
    """floor(u64 * bound / 2^64)."""
    return (int(u64) * int(bound)) >> 64


def floyd_pivots(n: int, k: int, seed: int) -> np.ndarray:
    """Uniform k-subset of {0..n-1} by Floyd's algorithm; returned sorted."""
    if not 0 < k <= n:
        raise ValueError("need 0 < k <= n")
    chosen: set[int] = set()
    for s, j in enumerate(range(n - k, n)):
        word = philox4x64_10_int((s, 0, 0, 0), (seed, TAG_SAMPLE))[0]
        t = uniform_below(word, j + 1)
        chosen.add(j if t in chosen else t)
    return np.array(sorted(chosen), dtype=np.int64)


def pair_resistance_solves(g: Graph, v: int, pivots, solver: str = "dense", tol: float = 1e-12):
    """d_ER(v, s) for each pivot s, one pair system L p = e_v - e_s each."""
    pivots = np.asarray(pivots)
    B = np.zeros((g.n, pivots.size))
    for j, s in enumerate(pivots):
        B[v, j] += 1.0
        B[s, j] -= 1.0
    if solver == "dense":
        P = pinv(g) @ B
    else:
        P, _, _ = cg_solve(laplacian(g), B, tol=tol)
    return np.array([P[v, j] - P[s, j] for j, s in enumerate(pivots)])


def sampled_farness(g: Graph, k: int, seed: int, nodes, solver: str = "dense", tol: float = 1e-12,
                    pivots=None):
    """(n/k) sum_{s in S} d_ER(v, s) for each query node v (one pivot set S
    shared by all query nodes)."""
    S = floyd_pivots(g.n, k, seed) if pivots is None else np.asarray(pivots)
    out = np.empty(len(nodes))
    for t, v in enumerate(nodes):
        d = pair_resistance_solves(g, int(v), S, solver, tol)
        out[t] = (g.n / S.size) * d.sum()
    return out
