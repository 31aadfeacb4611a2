"""FP64-accurate dense products A X of FP32-stored A and FP64 X, to check products
whose error is far below an FP64 GEMM's (a BLAS GEMM carries up to about d u of
sum |a_ik x_k|). The sampling driver needs its matrix-loads (Sec. 1.2) accurate well
beyond FP32 (Sec. 5: the nugget sits far below u ||K||). Test infrastructure only.

Method (plain definitions, no blocking): each x_k is split into a 26-bit head and the
rest with Veltkamp's splitting (Dekker 1971), so both products a_ik x_k^head and
a_ik x_k^tail are exact in FP64 (24 + 26 and 24 + 27 significant bits); the exact
products of a row are added by pairwise summation (NumPy's reduction along a
contiguous axis), whose error is at most about log2(d) u sum |a_ik x_k|.
"""
from __future__ import annotations

import numpy as np

_SPLITTER = 2.0 ** 27 + 1.0  # Veltkamp's constant for a 26-bit head of an FP64 value


def split_head_tail(x):
    """x = head + tail exactly, head with at most 26 significant bits (Veltkamp)."""
    x = np.asarray(x, dtype=np.float64)
    t = _SPLITTER * x
    head = t - (t - x)
    return head, x - head


def matvec(a32, x):
    """sum_k a_ik x_k for FP32-stored a (d x d) and FP64 x, to about log2(d) u sum |a x|."""
    a = np.asarray(a32, dtype=np.float32).astype(np.float64)
    head, tail = split_head_tail(x)
    return (a * head[None, :]).sum(axis=1) + (a * tail[None, :]).sum(axis=1)


def matmul(a32, X, mu=0.0):
    """A X + mu X column by column (X: d x L FP64)."""
    X = np.asarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    out = np.empty_like(X)
    for j in range(X.shape[1]):
        out[:, j] = matvec(a32, X[:, j]) + mu * X[:, j]
    return out


def abs_products(a32, X):
    """sum_k |a_ik| |x_kj| (the scale of the rounding bounds)."""
    return np.abs(np.asarray(a32, dtype=np.float64)) @ np.abs(np.asarray(X, dtype=np.float64))
