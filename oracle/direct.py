"""O0: the plain result definitions the method converges to. Test infrastructure only.

* solve:      x = A_mu^{-1} b by Cholesky of A_mu (Eq. 1.1).
* ridge_path: x(mu_j) = (A + mu_j I)^{-1} b for every shift via one
              eigendecomposition of A (Sec. 1, ridge regression).
* sqrtm_apply: A^{1/2} B via the eigendecomposition (Sec. 1, sampling Gaussians).
* isqrtm_apply: A^{-1/2} B via the eigendecomposition (the inverse square root that
              Sec. 5 computes with the same basis and shifts, other weights).

Pinned by tests against closed forms (diagonal matrices, known eigenpairs) and
residuals.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def solve(a, mu, b):
    """x = (A + mu I)^{-1} b by Cholesky (float64)."""
    a = np.asarray(a, dtype=np.float64)
    am = a + mu * np.eye(a.shape[0])
    c = sla.cho_factor(am, lower=True)
    return sla.cho_solve(c, np.asarray(b, dtype=np.float64))


def ridge_path(a, mus, b):
    """Columns x(mu_j) = (A + mu_j I)^{-1} b from one eigendecomposition of A."""
    lam, v = np.linalg.eigh(np.asarray(a, dtype=np.float64))
    c = v.T @ np.asarray(b, dtype=np.float64)
    return np.stack([v @ (c / (lam + mu)) for mu in mus], axis=1)


def sqrtm_apply(a, b, shift=0.0):
    """(A + shift I)^{1/2} B from the eigendecomposition of A."""
    lam, v = np.linalg.eigh(np.asarray(a, dtype=np.float64))
    return v @ (np.sqrt(lam + shift)[:, None] * (v.T @ np.asarray(b, dtype=np.float64)))


def isqrtm_apply(a, b, shift=0.0):
    """(A + shift I)^{-1/2} B from the eigendecomposition of A."""
    lam, v = np.linalg.eigh(np.asarray(a, dtype=np.float64))
    return v @ ((1.0 / np.sqrt(lam + shift))[:, None] * (v.T @ np.asarray(b, dtype=np.float64)))


def rel_residual(op, mu, x, b):
    """||b - A_mu x|| / ||b|| with the operator's stored values promoted to float64."""
    r = np.asarray(b, np.float64) - op.apply(np.asarray(x, np.float64), mu)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


def a_norm_error(a, mu, x, xstar):
    """||x* - x||_{A_mu} / ||x*||_{A_mu}, the error measure of the paper's figures."""
    a = np.asarray(a, np.float64)
    e = xstar - x
    am = lambda v: a @ v + mu * v
    return float(np.sqrt(e @ am(e)) / np.sqrt(xstar @ am(xstar)))
