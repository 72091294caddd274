"""The projection (Johnson-Lindenstrauss) estimator, Sec. 5.2, Algorithm 1.

Steps, in the paper's order and notation:

1. Construct the random k x m matrix Q.  Reading: entries +-1/sqrt(k) with
   equal probability and no zeros (Sec. 5.2 lists {0, +-1/sqrt(k)} without
   probabilities; zeros would need a rescaling the paper does not give).
   Signs come from Philox4x64-10, see ``oracle.philox``.
2. Y = Q W^{1/2} B (k x n).
3. For i = 1..k solve L z_i = Y_{i,.}.  Reading: the right-hand side is row i
   of Y, a length-n vector (the paper writes Y_{.,i}, but Y is k x n).
   Z is the k x n matrix with rows z_i^T.
4. d~(u, v) = ||Z_{.,u} - Z_{.,v}||_2^2, and the closeness estimate is
   c~(v) = (n - 1) / sum_{w != v} d~(v, w) (end of Sec. 5.2).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .cg import cg_solve
from .dense import pinv
from .graph import Graph, incidence, laplacian
from .philox import TAG_JL, philox4x64_10


def k_from_eps(n: int, eps: float) -> int:
    """k = ceil(log n / eps^2) (Sec. 6.4); reading: natural logarithm."""
    return int(math.ceil(math.log(n) / (eps * eps)))


def jl_sign_bits(seed: int, k: int, edge_ids: np.ndarray) -> np.ndarray:
    """(len(edge_ids), k) array of sign bits: 0 -> +1/sqrt(k), 1 -> -1/sqrt(k).
    Bit for JL row i of edge e: counter (e, i // 256, 0, 0), key (seed, TAG_JL),
    output word (i % 256) // 64, bit i % 64."""
    e = np.asarray(edge_ids, dtype=np.uint64)
    bits = np.empty((e.size, k), dtype=np.uint8)
    for blk in range((k + 255) // 256):
        words = philox4x64_10(e, np.uint64(blk), np.uint64(0), np.uint64(0), seed, TAG_JL)
        for i in range(blk * 256, min(k, blk * 256 + 256)):
            j = i % 256
            bits[:, i] = ((words[j // 64] >> np.uint64(j % 64)) & np.uint64(1)).astype(np.uint8)
    return bits


def projection_matrix(g: Graph, k: int, seed: int) -> np.ndarray:
    """Q (k x m) with entries +-1/sqrt(k) (Algorithm 1, step 1).  Dense:
    for small graphs only."""
    bits = jl_sign_bits(seed, k, np.arange(g.m))
    return (1.0 - 2.0 * bits.T.astype(np.float64)) / math.sqrt(k)


def jl_rhs(g: Graph, k: int, seed: int, chunk: int = 1 << 18) -> np.ndarray:
    """Y = Q W^{1/2} B as a k x n array (Algorithm 1, step 2).  Built in
    chunks of edges so Q is never held whole: Y = sum_e Q_{.,e} sqrt(w_e) B_{e,.}."""
    Y = np.zeros((k, g.n))
    B = incidence(g)
    sw = np.sqrt(g.w)
    for lo in range(0, g.m, chunk):
        hi = min(g.m, lo + chunk)
        bits = jl_sign_bits(seed, k, np.arange(lo, hi))
        Qc = (1.0 - 2.0 * bits.T.astype(np.float64)) / math.sqrt(k)  # k x chunk
        QW = Qc * sw[lo:hi][None, :]  # Q W^{1/2} restricted to the chunk
        Y += np.asarray(B[lo:hi].T @ QW.T).T
    return Y


def jl_solve(g: Graph, Y: np.ndarray, solver: str = "dense", tol: float = 1e-12):
    """Algorithm 1, step 3: rows z_i of Z solve L z_i = Y_i."""
    if solver == "dense":
        return (pinv(g) @ Y.T).T
    Z, _, _ = cg_solve(laplacian(g), Y.T, tol=tol)
    return Z.T


def pair_distance(Z: np.ndarray, u: int, v: int) -> float:
    """d~(u, v) = ||Z_{.,u} - Z_{.,v}||^2 (Algorithm 1, step 4)."""
    d = Z[:, u] - Z[:, v]
    return float(d @ d)


def jl_farness(g: Graph, k: int, seed: int, nodes, solver: str = "dense", tol: float = 1e-12,
               return_Z: bool = False):
    """Estimated electrical farness sum_{w != v} d~(v, w) of each query node,
    summed literally over w (end of Sec. 5.2)."""
    Y = jl_rhs(g, k, seed)
    Z = jl_solve(g, Y, solver, tol)
    out = farness_from_Z(Z, nodes)
    return (out, Z) if return_Z else out


def farness_from_Z(Z: np.ndarray, nodes) -> np.ndarray:
    """sum_{w != v} ||Z_{.,v} - Z_{.,w}||^2 for each query node v, summed
    literally over w (Algorithm 1, step 4; Z is k x n)."""
    out = np.empty(len(nodes))
    for t, v in enumerate(nodes):
        D = Z - Z[:, [v]]
        col = np.einsum("ij,ij->j", D, D)  # d~(v, w) for every w; w = v gives 0
        out[t] = col.sum()
    return out


def jl_rhs_at(g: Graph, k: int, seed: int, nodes) -> np.ndarray:
    """Columns ``nodes`` of Y = Q W^{1/2} B (a k x len(nodes) array), each
    summed over the node's incident edges only (Algorithm 1, step 2): for a
    node u, Y[i, u] = sum over edges e containing u of Q[i, e] sqrt(w_e)
    B[e, u], with B[e, u] = +1 when u is the smaller endpoint and -1 when it
    is the larger.  For spot checks of very large graphs, where the whole Y
    is too costly."""
    out = np.zeros((k, len(nodes)))
    for t, u in enumerate(nodes):
        e_lo = np.nonzero(g.u == u)[0]  # u = min(e): B[e, u] = +1
        e_hi = np.nonzero(g.v == u)[0]  # u = max(e): B[e, u] = -1
        for edges, sign in ((e_lo, 1.0), (e_hi, -1.0)):
            if edges.size == 0:
                continue
            q = (1.0 - 2.0 * jl_sign_bits(seed, k, edges).astype(np.float64)) / math.sqrt(k)  # edges x k
            out[:, t] += sign * (q * np.sqrt(g.w[edges])[:, None]).sum(axis=0)
    return out
