"""O5: block-CG whose block shrinks to one column after s steps (Outlook; Sec. CG_pro).
Test infrastructure only.

The outlook asks for a block-CG that drops to a smaller block once the large block no
longer pays, and Sec. CG_pro runs full reorthogonalisation until s blocks are held,
then orthogonalises later vectors only against those. This module writes that out as:

* locked basis: W = an orthonormal basis of K_s(A, [b Omega]) (the first s block-Krylov
  blocks, full reorthogonalisation; nystrom.krylov_orthobasis).
* deflated CG on W (Def-CG of Saad, Yeung, Erhel & Guyomarc'h, SIAM J. Sci. Comput. 21,
  2000): from x_{-1} = 0,
      x_0 = W (W^T A_mu W)^{-1} W^T b,          r_0 = b - A_mu x_0  (r_0 orthogonal to W),
      mu_j = (W^T A_mu W)^{-1} (A_mu W)^T r_j,  p_0 = r_0 - W mu_0,
      alpha_j = r_j^T r_j / p_j^T A_mu p_j,     x_{j+1} = x_j + alpha_j p_j,
      r_{j+1} = r_j - alpha_j A_mu p_j,         beta_j = r_{j+1}^T r_{j+1} / r_j^T r_j,
      p_{j+1} = beta_j p_j + r_{j+1} - W mu_{j+1}.
  Every direction is A_mu-orthogonal to W and every residual orthogonal to it, so each
  iteration is a one-column CG step that keeps orthogonalising against the locked
  blocks. x_0 is the block-CG iterate after s loads (the Galerkin solution on K_s), and
  x_j minimises the A_mu-norm error over span(W) + K_j(P A_mu, r_0) with the projector
  P = I - A_mu W (W^T A_mu W)^{-1} W^T (A_mu p_0 = P A_mu r_0, and so on by induction).

Pinned by: the brute-force Galerkin solution over that space, SciPy's CG when W spans
an invariant subspace (the projection is then inert), finite termination after
d - dim W iterations, the block-CG iterate at j = 0, and the space inclusion
span(W) + K_j(P A_mu, r_0) in K_{s+j}(A, [b Omega]) (block-CG after s + j loads is never
less accurate).
"""
from __future__ import annotations

import numpy as np

from .nystrom import krylov_orthobasis
from .operators import as_operator


def locked_basis(a, b, omega, s):
    """Orthonormal basis of K_s(A, [b Omega]) (s - 1 block products)."""
    B = np.column_stack([np.asarray(b, np.float64), np.asarray(omega, np.float64)])
    return krylov_orthobasis(a, B, s)


def deflated_cg(a, mu, b, W, t):
    """Iterates [x_0, x_1, .., x_t] of Def-CG on A_mu = A + mu I with deflation space W."""
    op = as_operator(a)
    b = np.asarray(b, np.float64)
    W = np.asarray(W, np.float64).reshape(b.shape[0], -1)
    AW = op.apply(W, mu) if W.shape[1] else W
    WAW = W.T @ AW
    WAW = 0.5 * (WAW + WAW.T)

    def coarse(v):  # (W^T A_mu W)^{-1} v
        return np.linalg.solve(WAW, v) if W.shape[1] else np.zeros(0)

    x = W @ coarse(W.T @ b)
    r = b - op.apply(x, mu)
    p = r - W @ coarse(AW.T @ r)
    rr = r @ r
    out = [x.copy()]
    for _ in range(t):
        q = op.apply(p, mu)
        alpha = rr / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        out.append(x.copy())
        rr_new = r @ r
        beta = rr_new / rr
        rr = rr_new
        p = beta * p + r - W @ coarse(AW.T @ r)
    return out


def shrink_solve(a, mu, b, omega, s, t):
    """Iterates after s block steps on [b Omega] and then t deflated one-column steps."""
    return deflated_cg(a, mu, b, locked_basis(a, b, omega, s), t)
