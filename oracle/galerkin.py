"""Brute-force block-CG iterate straight from Def. BCG (Sec. 3). Test infrastructure only.

bcg_t^(i)(mu) minimises the A_mu-norm error over K_t(A_mu, B) (Def. BCG), and
K_t(A_mu, B) = K_t(A, B) (Eq. shift_invariance). For a basis V of K_t the minimiser
is the Galerkin solution x = V (V^T A_mu V)^{-1} V^T b. The basis here is the
explicit block Krylov matrix [B, A B, ..., A^{t-1} B] (Eq. block_krylov_def),
orthonormalised by an SVD that drops numerically dependent directions. For tiny d
only: the monomial basis is ill-conditioned by construction.
"""
from __future__ import annotations

import numpy as np

from .operators import as_operator


def krylov_basis(a, B, t, rtol=1e-12):
    op = as_operator(a)
    blocks = [np.asarray(B, dtype=np.float64)]
    for _ in range(1, t):
        blocks.append(op.apply(blocks[-1], 0.0))
    K = np.column_stack(blocks)
    # scale columns so the SVD rank decision is not dominated by growth of A^k B
    K = K / np.maximum(np.linalg.norm(K, axis=0), 1e-300)
    u, s, _ = np.linalg.svd(K, full_matrices=False)
    keep = s > rtol * s[0]
    return u[:, keep]


def bcg_iterate(a, mu, B, t, col=0):
    """The t-th block-CG iterate for column `col` of B (t-1 ... t loads; see Q2 reading)."""
    op = as_operator(a)
    V = krylov_basis(op, B, t)
    AV = op.apply(V, mu)
    H = V.T @ AV
    rhs = V.T @ np.asarray(B, dtype=np.float64)[:, col]
    return V @ np.linalg.solve(0.5 * (H + H.T), rhs)
