"""Exact current-flow closeness by dense linear algebra (Sec. 4).

* ``pinv``: the Moore-Penrose pseudoinverse L^+ of a connected graph's
  Laplacian as (L + J/n)^{-1} - J/n, J the all-ones matrix.  On range(L)
  (vectors orthogonal to 1) L + J/n acts as L, and on 1 as the identity, so
  this equals L^+.  The inverse is a library routine (numpy.linalg.inv).
* ``grounded_resistance``: the paper's own exact form (Sec. 4): delete the row
  and column of one node g to get the regular matrix L~, then
  d_ER(v, w) = L~^{-1}_vv - 2 L~^{-1}_vw + L~^{-1}_ww with the deleted node's
  entries read as 0.
* ``resistance_matrix``: d_ER(u, v) = (e_u - e_v)^T L^+ (e_u - e_v), i.e. the
  potential difference p_uv(u) - p_uv(v) of Eq. system with b = e_u - e_v
  (Sec. 4).
* ``farness`` / ``closeness``: electrical farness sum_{w != v} d_ER(v, w) and
  c_ER(v) = (n - 1) / farness (Eq. closeness2).
"""
from __future__ import annotations

import numpy as np

from .graph import Graph, laplacian_dense


def pinv(g: Graph) -> np.ndarray:
    L = laplacian_dense(g)
    n = g.n
    return np.linalg.inv(L + np.full((n, n), 1.0 / n)) - 1.0 / n


def resistance_matrix(g: Graph, Lp: np.ndarray | None = None) -> np.ndarray:
    """R[u, v] = L^+_uu - 2 L^+_uv + L^+_vv, the quadratic form
    (e_u - e_v)^T L^+ (e_u - e_v)."""
    if Lp is None:
        Lp = pinv(g)
    dg = np.diag(Lp)
    R = dg[:, None] + dg[None, :] - 2.0 * Lp
    np.fill_diagonal(R, 0.0)  # d_ER(v, v) := 0 by convention (Sec. 4)
    return R


def grounded_resistance(g: Graph, ground: int = 0) -> np.ndarray:
    """Sec. 4: invert L with row/column ``ground`` removed."""
    L = laplacian_dense(g)
    keep = np.array([i for i in range(g.n) if i != ground])
    Lt = L[np.ix_(keep, keep)]
    Gi = np.zeros((g.n, g.n))
    Gi[np.ix_(keep, keep)] = np.linalg.inv(Lt)
    dg = np.diag(Gi)
    R = dg[:, None] + dg[None, :] - 2.0 * Gi
    np.fill_diagonal(R, 0.0)
    return R


def farness(g: Graph, R: np.ndarray | None = None) -> np.ndarray:
    """f(v) = sum_{w != v} d_ER(v, w) for every node v (Eq. closeness2)."""
    if R is None:
        R = resistance_matrix(g)
    off = R.copy()
    np.fill_diagonal(off, 0.0)  # the sum skips w = v
    return off.sum(axis=1)


def closeness(g: Graph, f: np.ndarray | None = None) -> np.ndarray:
    """c_ER(v) = (n - 1) / f(v) (Eq. closeness2)."""
    if f is None:
        f = farness(g)
    return (g.n - 1) / f
