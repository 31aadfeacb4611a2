"""O2: block-Lanczos with full reorthogonalisation and projected shifted solves.

Test infrastructure only. Follows Sec. 3.2 (Thm. cost and Eq. bcg_alg): block-Lanczos
on (A, B) for t steps gives Q_t with orthonormal columns spanning K_t(A, B) and the
block-tridiagonal T_t = Q_t^T A Q_t; then for any shift mu

    bcg_t(mu) = Q_t (T_t + mu I)^{-1} E_1 R_0,        B = Q_1 R_0,

whose first column is ||b|| Q_t (T_t + mu I)^{-1} e_1 (Eq. bcg_alg). One basis serves
every shift (Eq. shift_invariance). The square-root iterate of Def. blansq
integrates A bcg_t(z^2) over z; with the Lanczos relation
A Q_t = Q_t T_t + Q_{t+1} B_t E_t^T and (2/pi) int_0^inf (T + z^2)^{-1} dz = T^{-1/2}
that integral is, exactly,

    bsq_t = Q_t T_t^{1/2} E_1 R_0 + Q_{t+1} B_t E_t^T T_t^{-1/2} E_1 R_0.

Orthogonalisation: each new block is orthogonalised against all previous blocks
twice (classical Gram-Schmidt, twice) and factorised by an SVD-based QR that drops
directions below rtol, so the block width may shrink once K_t fills R^d.

The inverse square root on the same basis is Q_t T_t^{-1/2} E_1 R_0: the integral of
bcg_t(z^2) itself, without the factor A.

Pinned by: shift invariance against separate direct solves, brute-force Galerkin
iterates, finite termination, closed-form A^{1/2} and A^{-1/2} on known spectra, and
adaptive quadrature of both integrals on a partial basis.
"""
from __future__ import annotations

import numpy as np

from .operators import as_operator


def _orth_block(W, rtol):
    """Orthonormal basis Q and coefficients C with W ~= Q C, dropping tiny directions."""
    if W.shape[1] == 0:
        return W, np.zeros((0, 0))
    u, s, vt = np.linalg.svd(W, full_matrices=False)
    keep = s > rtol
    return u[:, keep], s[keep, None] * vt[keep]


def block_lanczos(a, B, t, rtol=1e-12):
    """Run t steps; returns dict(Q=list of blocks, A=diag blocks, Bs=subdiag blocks, R0, loads)."""
    op = as_operator(a)
    B = np.asarray(B, dtype=np.float64)
    scale = np.linalg.norm(B)
    Q1, R0 = _orth_block(B, rtol * scale)
    Qs, As, Bs = [Q1], [], []
    loads = 0
    Qprev, Bprev = None, None
    for k in range(t):
        Qk = Qs[-1]
        W = op.apply(Qk, 0.0)
        loads += 1
        Ak = Qk.T @ W
        Ak = 0.5 * (Ak + Ak.T)
        As.append(Ak)
        W = W - Qk @ Ak
        if Qprev is not None:
            W = W - Qprev @ Bprev.T
        Qall = np.column_stack(Qs)
        for _ in range(2):
            W = W - Qall @ (Qall.T @ W)
        Qn, Bk = _orth_block(W, rtol * max(np.linalg.norm(op.apply(Qk, 0.0), 2), 1e-300))
        Bs.append(Bk)
        Qprev, Bprev = Qk, Bk
        Qs.append(Qn)
        if Qn.shape[1] == 0:
            break
    return dict(Q=Qs, A=As, B=Bs, R0=R0, loads=loads)


def tridiag(lz):
    """Assemble T_t (n x n) from the diagonal blocks A_k and subdiagonal blocks B_k."""
    As, Bs = lz["A"], lz["B"]
    sizes = [a.shape[0] for a in As]
    n = sum(sizes)
    T = np.zeros((n, n))
    off = np.concatenate([[0], np.cumsum(sizes)])
    for k, Ak in enumerate(As):
        T[off[k]:off[k + 1], off[k]:off[k + 1]] = Ak
        if k + 1 < len(As):
            Bk = Bs[k]  # rows: block k+1, cols: block k
            T[off[k + 1]:off[k + 2], off[k]:off[k + 1]] = Bk
            T[off[k]:off[k + 1], off[k + 1]:off[k + 2]] = Bk.T
    return T


def basis(lz):
    nblk = len(lz["A"])
    return np.column_stack(lz["Q"][:nblk])


def shifted_iterates(lz, mus, col=0):
    """Columns bcg_t^(col)(mu_j) = Q_t (T_t + mu_j I)^{-1} E_1 R_0 e_col for every shift."""
    Q = basis(lz)
    T = tridiag(lz)
    n = T.shape[0]
    rhs = np.zeros(n)
    rhs[:lz["R0"].shape[0]] = lz["R0"][:, col]
    Z = np.stack([np.linalg.solve(T + mu * np.eye(n), rhs) for mu in mus], axis=1)
    return Q @ Z


def isqrt_iterate(lz):
    """The inverse square root on the basis: (2/pi) int_0^inf bcg_t(z^2) dz for every
    column of B, which is exactly Q_t T_t^{-1/2} E_1 R_0 (Sec. 5: the same shifted
    iterates as bsq_t without the factor A, so no Lanczos-relation term)."""
    Q = basis(lz)
    T = tridiag(lz)
    n = T.shape[0]
    lam, V = np.linalg.eigh(T)
    E1R0 = np.zeros((n, lz["R0"].shape[1]))
    E1R0[:lz["R0"].shape[0]] = lz["R0"]
    return Q @ (V @ ((1.0 / np.sqrt(lam))[:, None] * (V.T @ E1R0)))


def sqrt_iterate(lz):
    """bsq_t for every column of B: the exact integral of Def. blansq on the basis."""
    Q = basis(lz)
    T = tridiag(lz)
    n = T.shape[0]
    lam, V = np.linalg.eigh(T)
    E1R0 = np.zeros((n, lz["R0"].shape[1]))
    E1R0[:lz["R0"].shape[0]] = lz["R0"]
    half = V @ (np.sqrt(lam)[:, None] * (V.T @ E1R0))
    mhalf = V @ ((1.0 / np.sqrt(lam))[:, None] * (V.T @ E1R0))
    out = Q @ half
    Qn, Bt = lz["Q"][len(lz["A"])], lz["B"][len(lz["A"]) - 1]
    if Qn.shape[1]:
        last = lz["A"][-1].shape[0]
        out += Qn @ (Bt @ mhalf[n - last:])
    return out
