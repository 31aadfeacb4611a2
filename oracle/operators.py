"""Block products with A_mu = A + mu I (Eq. 1.1; access model of Sec. 1.2).

The stored values, promoted to float64, define A. Test infrastructure only.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class Dense:
    """A stored as a dense d x d matrix."""

    def __init__(self, a):
        self.a = np.asarray(a, dtype=np.float64)
        self.d = self.a.shape[0]

    def apply(self, p, mu=0.0):
        return self.a @ p + mu * p

    def matrix(self):
        return self.a


class CSR:
    """A stored in compressed sparse row form (rowptr, colidx, vals)."""

    def __init__(self, rowptr, colidx, vals, d=None):
        d = len(rowptr) - 1 if d is None else d
        self.m = sp.csr_matrix((np.asarray(vals, dtype=np.float64), np.asarray(colidx), np.asarray(rowptr)), shape=(d, d))
        self.d = d

    def apply(self, p, mu=0.0):
        return self.m @ p + mu * p

    def matrix(self):
        return self.m.toarray()


class Gram:
    """A = Z^T Z applied matrix-free as Z^T (Z P) (ridge regression, Sec. 1)."""

    def __init__(self, z):
        self.z = np.asarray(z, dtype=np.float64)
        self.d = self.z.shape[1]

    def apply(self, p, mu=0.0):
        return self.z.T @ (self.z @ p) + mu * p

    def matrix(self):
        return self.z.T @ self.z


def as_operator(a):
    if hasattr(a, "apply"):
        return a
    return Dense(a)
