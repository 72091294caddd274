"""Conjugate gradient for the Laplacian system L x = b (Sec. 2, Eq. system;
Sec. 3.1: CG, stopping on the relative residual).

L is singular with null space span{1} (rank n - 1 for a connected G, Sec. 2),
so b is first projected onto range(L) = 1-perp and every iterate is kept
there: the solution returned is the one with zero mean, x = L^+ b.

Each column of B is an independent system with its own step lengths; the
columns are only stored side by side.  Stopping rule per column:
||b - L x||_2 <= tol * ||b||_2 (the relative residual of Sec. 3.1).
Optionally the diagonal (Jacobi) preconditioner D^{-1} is applied.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def project_mean(X: np.ndarray) -> np.ndarray:
    """Remove each column's mean: the orthogonal projection onto 1-perp."""
    return X - X.mean(axis=0, keepdims=True)


def cg_solve(L: sp.spmatrix, B: np.ndarray, tol: float = 1e-12, maxiter: int = 100000,
             jacobi: bool = True):
    """Solve L X = B column by column.  Returns (X, iterations, relres) where
    relres[j] is the final ||b_j - L x_j|| / ||b_j|| (computed afresh)."""
    B = np.asarray(B, dtype=np.float64)
    squeeze = B.ndim == 1
    if squeeze:
        B = B[:, None]
    n, k = B.shape
    b = project_mean(B)
    bnorm = np.linalg.norm(b, axis=0)
    dinv = 1.0 / L.diagonal() if jacobi else np.ones(n)
    x = np.zeros((n, k))
    r = b.copy()
    z = project_mean(dinv[:, None] * r)
    p = z.copy()
    rz = np.einsum("ij,ij->j", r, z)
    active = bnorm > 0
    it = 0
    while it < maxiter:
        rnorm = np.linalg.norm(r, axis=0)
        active &= rnorm > tol * bnorm
        if not active.any():
            break
        q = L @ p
        pq = np.einsum("ij,ij->j", p, q)
        alpha = np.where(active, rz / np.where(pq == 0, 1, pq), 0.0)
        x += alpha * p
        r -= alpha * q
        z = project_mean(dinv[:, None] * r)
        rz_new = np.einsum("ij,ij->j", r, z)
        beta = np.where(active, rz_new / np.where(rz == 0, 1, rz), 0.0)
        p = z + beta * p
        rz = rz_new
        it += 1
    x = project_mean(x)
    res = np.linalg.norm(b - L @ x, axis=0)
    relres = np.where(bnorm > 0, res / np.where(bnorm > 0, bnorm, 1), 0.0)
    if squeeze:
        return x[:, 0], it, relres
    return x, it, relres
