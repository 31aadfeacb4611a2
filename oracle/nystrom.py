"""O3: Nystrom-preconditioned CG, the comparator of Thm. main. Test infrastructure only.

* nystrom(a, Omega, s): the block-Krylov Nystrom approximation of Eq. nystromBKI_def,
  A<K_s> = (A K)(K^T A K)^+ (K^T A) with K_s = [Omega, A Omega, ..., A^{s-1} Omega],
  computed from an orthonormal basis V of range(K_s) (the monomial basis is avoided,
  Sec. 2.2.2): with Y = A V and C = V^T Y = L L^T, A<K_s> = F F^T for F = Y L^{-T},
  so U and D come from the SVD of F (D = singular values squared). Uses s loads.
* preconditioner_inverse(U, D, theta, mu): P_mu^{-1} of Eq. precond_def,
  (theta + mu) U (D + mu I)^{-1} U^T + (I - U U^T).
* pcg(a, mu, b, Pinv, t): t iterations of textbook preconditioned CG from x_0 = 0;
  the iterate lies in K_t(P^{-1} A_mu, P^{-1} b) and minimises the A_mu-norm error
  there (Def. PCG). With Pinv = identity it is CG (Def. CG, Hestenes-Stiefel).
* theta follows Sec. 7: the smallest eigenvalue of the Nystrom approximation.

Pinned by: Prop. condno_perturb (condition-number bound), brute-force Galerkin over
the preconditioned Krylov space, scipy's CG for the unpreconditioned case.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .operators import as_operator


def krylov_orthobasis(a, Omega, s):
    """Orthonormal basis of range([Omega, A Omega, ..., A^{s-1} Omega]) by block
    Gram-Schmidt (twice) on successive products; (s - 1) loads for the basis."""
    op = as_operator(a)
    V = np.linalg.qr(np.asarray(Omega, np.float64))[0]
    blocks = [V]
    for _ in range(1, s):
        W = op.apply(blocks[-1], 0.0)
        Vall = np.column_stack(blocks)
        for _ in range(2):
            W = W - Vall @ (Vall.T @ W)
        u, sv, _ = np.linalg.svd(W, full_matrices=False)
        keep = sv > 1e-12 * max(sv[0], 1e-300) if sv.size else sv > 0
        blocks.append(u[:, keep])
    return np.column_stack(blocks)


def nystrom(a, Omega, s):
    """(U, D) with A<K_s> = U diag(D) U^T; U orthonormal (d x r), D > 0 descending."""
    op = as_operator(a)
    V = krylov_orthobasis(op, Omega, s)
    Y = op.apply(V, 0.0)
    C = V.T @ Y
    C = 0.5 * (C + C.T)
    lam, W = np.linalg.eigh(C)
    keep = lam > 1e-13 * lam[-1]
    # pseudo-inverse square root on the numerically nonzero part of C
    F = Y @ (W[:, keep] / np.sqrt(lam[keep])[None, :])
    U, sig, _ = np.linalg.svd(F, full_matrices=False)
    return U, sig ** 2


def preconditioner_inverse(U, D, theta, mu):
    """Dense P_mu^{-1} = (theta + mu) U (D + mu)^{-1} U^T + (I - U U^T) (Eq. precond_def)."""
    d = U.shape[0]
    return (theta + mu) * (U / (D + mu)[None, :]) @ U.T + (np.eye(d) - U @ U.T)


def pcg(a, mu, b, Pinv, t):
    """Iterates x_1..x_t of preconditioned CG from x_0 = 0 (Def. PCG); Pinv=None is CG."""
    op = as_operator(a)
    b = np.asarray(b, np.float64)
    M = (lambda v: v) if Pinv is None else (lambda v: Pinv @ v)
    x = np.zeros_like(b)
    r = b.copy()
    z = M(r)
    p = z.copy()
    rz = r @ z
    out = []
    for _ in range(t):
        q = op.apply(p, mu)
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        out.append(x.copy())
        z = M(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return out


def preconditioned_condition_number(a, mu, Pinv):
    """kappa(P^{-1/2} A_mu P^{-1/2}) from the generalized eigenvalues of (A_mu, P)."""
    A = as_operator(a).matrix()
    d = A.shape[0]
    Am = A + mu * np.eye(d)
    Pi = 0.5 * (Pinv + Pinv.T)
    w, V = np.linalg.eigh(Pi)
    Ph = V @ (np.sqrt(w)[:, None] * V.T)
    M = Ph @ Am @ Ph
    ev = np.linalg.eigvalsh(0.5 * (M + M.T))
    return ev[-1] / ev[0]
