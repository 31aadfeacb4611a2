"""O1: block-CG on the augmented start block [b Omega] (Def. BCG, Thm. main, Sec. 3).

Test infrastructure only. The paper defines the t-th block-CG iterate by its
optimality over the block Krylov space K_t(A_mu, B) (Def. BCG) and cites O'Leary's
recurrence for computing it (Sec. 3). This module writes that recurrence out with
X_0 = 0, R_0 = P_0 = B, one block product ("matrix-load") per step:

    Y     = A_mu P                      (the load)
    alpha = (P^T Y)^{-1} (R^T R)
    X    += P alpha                     (only column 0 is kept: bcg^(1))
    R    -= Y alpha
    beta  = (R_old^T R_old)^{-1} (R^T R)
    P     = R + P beta

The stopping rule is the a-posteriori residual of column 0 (Sec. 4, remark on
a-posteriori estimates): stop once ||R[:,0]|| <= tol * ||b||.

Rank deficiency. The block Krylov space can grow by fewer than m directions in one
step even in exact arithmetic (Sec. 3.2 notes blocks becoming rank deficient); then
P^T Y is singular. The small systems are solved by a Cholesky factorisation of the
unit-diagonal scaled matrix D^{-1/2} G D^{-1/2} with diagonal pivoting (LAPACK
dpstrf), which stops at the first pivot below `rank_tol`. alpha is the solution on
the kept columns (zero rows for the dependent ones), so X += P alpha is still the
Galerkin update over span(P). The step that detects a dependent column applies that
update and ends the run with status "deflated"; `refined_solve` restarts from the
new residual (the remedy the paper's outlook suggests, deflating the block).

Pinned by: brute-force Galerkin iterates (Def. BCG), CG for a one-column block
(Def. CG, Hestenes-Stiefel), finite termination at ceil(d/m) loads (proof of
Thm. cost), exact recovery for k <= l outliers over a flat spectrum (Thm. nested).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .operators import as_operator


class Breakdown(Exception):
    pass


def pivoted_solve(g, rhs, rank_tol):
    """X with G X = RHS on the numerically independent columns of G (see module doc).

    Returns (X, rank). Raises Breakdown if G has a non-positive diagonal entry.
    """
    g = 0.5 * (g + g.T)
    dg = np.diag(g).copy()
    if not np.all(np.isfinite(g)) or np.any(dg <= 0):
        raise Breakdown("non-positive diagonal")
    s = np.sqrt(dg)
    gs = g / np.outer(s, s)
    c, piv, rank, info = sla.lapack.dpstrf(gs, lower=1, tol=rank_tol)
    if rank == 0:
        raise Breakdown("rank 0")
    p = piv[:rank] - 1
    L = np.tril(c[:rank, :rank])
    y = sla.solve_triangular(L, rhs[p, :] / s[p, None], lower=True)
    y = sla.solve_triangular(L.T, y, lower=False)
    x = np.zeros((g.shape[0], rhs.shape[1]))
    x[p, :] = y / s[p, None]
    return x, int(rank)


def block_cg(a, mu, b, omega, tol=1e-10, max_loads=10000, keep_all=False, history=False, rank_tol=1e-12):
    """Run block-CG on B = [b Omega]; return dict(x, loads, converged, ...).

    a      operator (see operators) or dense matrix
    mu     shift (A_mu = A + mu I)
    b      right-hand side, shape (d,)
    omega  sketch, shape (d, l); l = 0 gives CG
    tol    stop when ||R[:,0]|| <= tol ||b||
    max_loads  cap on block products
    keep_all   also return the full block iterate X (d x m)
    history    record x after every load (list of arrays)
    """
    op = as_operator(a)
    b = np.asarray(b, dtype=np.float64)
    B = np.column_stack([b, np.asarray(omega, dtype=np.float64)]) if omega is not None and np.size(omega) else b[:, None].copy()
    d, m = B.shape
    X = np.zeros((d, m))
    R = B.copy()
    P = R.copy()
    S = R.T @ R
    bnorm = np.linalg.norm(b)
    xs, res = [], [np.sqrt(S[0, 0]) / bnorm]
    loads = 0
    status = "max_loads"
    if res[-1] <= tol:
        status = "converged"
    while status != "converged" and loads < max_loads:
        Y = op.apply(P, mu)
        loads += 1
        G = P.T @ Y
        try:
            alpha, rank = pivoted_solve(G, S, rank_tol)
        except Breakdown:
            status = "breakdown"
            break
        X += P @ alpha
        if history:
            xs.append(X[:, 0].copy())
        if rank < m:
            status = "deflated"
            res.append(np.nan)
            break
        R -= Y @ alpha
        S_new = R.T @ R
        res.append(np.sqrt(max(S_new[0, 0], 0.0)) / bnorm)
        if res[-1] <= tol:
            status = "converged"
            break
        try:
            beta, rank = pivoted_solve(S, S_new, rank_tol)
        except Breakdown:
            status = "breakdown"
            break
        if rank < m:
            status = "deflated"
            break
        P = R + P @ beta
        S = S_new
    out = dict(x=X[:, 0].copy(), loads=loads, status=status, converged=status == "converged",
               residuals=np.array(res))
    if keep_all:
        out["X"] = X
    if history:
        out["history"] = xs
    return out


def refined_solve(a, mu, b, omega, tol=1e-10, inner_tol=1e-10, max_refine=10, max_loads=10000,
                  adaptive_inner=False):
    """Block-CG with FP64 residual refinement (Sec. 4 remark on a-posteriori checks).

    Each outer step computes r = b - A_mu x, restarts block-CG on [r/||r|| Omega] and
    adds the column-0 iterate scaled back by ||r||. Stops when ||r|| <= tol ||b||.

    The inner solve stops at relative residual `inner_tol`. With adaptive_inner it
    stops instead at min(0.5, max(inner_tol, tol ||b|| / (2 ||r||))): a pass asks for
    no more reduction than the outer target still needs (with a factor 2 of margin),
    so the last pass does not solve far below tol. The paper gives no inner rule; this
    is the reading the solver library takes for its refinement loop.

    Returns x, loads (inner block products plus one residual product per pass),
    inner_loads (block products alone), refinements and the final relative residual.
    """
    op = as_operator(a)
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    total, inner, steps = 0, 0, 0
    r = b.copy()
    while True:
        rn = np.linalg.norm(r)
        if rn <= tol * bnorm or steps >= max_refine:
            break
        target = inner_tol
        if adaptive_inner:
            target = min(0.5, max(inner_tol, 0.5 * tol * bnorm / rn))
        out = block_cg(op, mu, r / rn, omega, tol=target, max_loads=max_loads - total)
        total += out["loads"]
        inner += out["loads"]
        x += rn * out["x"]
        steps += 1
        r = b - op.apply(x, mu)
        total += 1
        if total >= max_loads:
            break
    return dict(x=x, loads=total, inner_loads=inner, refinements=steps, rel_residual=np.linalg.norm(r) / bnorm)
