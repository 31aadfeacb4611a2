"""Seeded synthetic inputs for the randomized block-CG solver.

This module draws random numbers and assembles test matrices. It holds none of
the solver's arithmetic, so both the CUDA path (through its Python binding) and
the FP64 CPU oracle can read the same buffers.

Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11), written here from its published
definition, followed by the Box-Muller transform. The CUDA library implements the
same generator independently to draw the Gaussian sketch Omega on the device; the
definition below is the contract both sides follow:

  key     = (seed mod 2^32, floor(seed / 2^32) mod 2^32)
  counter = (c mod 2^32, floor(c / 2^32), stream, 0)      for block index c
  normal k of a stream uses block c = floor(k / 2); with the block's words
  (x0, x1, x2, x3):
     u1 = ((x0 >> 5) * 2^26 + (x1 >> 6) + 0.5) * 2^-53
     u2 = ((x2 >> 5) * 2^26 + (x3 >> 6) + 0.5) * 2^-53
     r  = sqrt(-2 ln u1);  normal k = r cos(2 pi u2) if k even, else r sin(2 pi u2)

Streams: 0 matrix factors, 1 spectrum / coefficients, 2 right-hand side, 3 Omega,
4 noise. The sketch Omega (d x l, column-major) is entry k = j*d + i of stream 3.
"""
from __future__ import annotations

import numpy as np

PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint32(0x9E3779B9)
PHILOX_W1 = np.uint32(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)

STREAM_FACTORS, STREAM_SPECTRUM, STREAM_RHS, STREAM_OMEGA, STREAM_NOISE = 0, 1, 2, 3, 4
BASE_SEED = 2501187170


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on uint32 counter arrays with a scalar 2x32 key."""
    c0 = np.asarray(c0, dtype=np.uint32).astype(np.uint64)
    c1 = np.asarray(c1, dtype=np.uint32).astype(np.uint64)
    c2 = np.asarray(c2, dtype=np.uint32).astype(np.uint64)
    c3 = np.asarray(c3, dtype=np.uint32).astype(np.uint64)
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    for r in range(10):
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        n0 = hi1 ^ c1 ^ np.uint64(k0)
        n1 = lo1
        n2 = hi0 ^ c3 ^ np.uint64(k1)
        n3 = lo0
        c0, c1, c2, c3 = n0, n1, n2, n3
        k0 = np.uint32((int(k0) + int(PHILOX_W0)) & 0xFFFFFFFF)
        k1 = np.uint32((int(k1) + int(PHILOX_W1)) & 0xFFFFFFFF)
    return (c0.astype(np.uint32), c1.astype(np.uint32), c2.astype(np.uint32), c3.astype(np.uint32))


def _key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF


def normals(seed: int, stream: int, n: int, offset: int = 0, chunk: int = 1 << 22) -> np.ndarray:
    """Entries offset .. offset+n-1 of the standard-normal stream (float64)."""
    out = np.empty(n, dtype=np.float64)
    k0, k1 = _key(seed)
    two53 = 2.0 ** -53
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        idx = np.arange(offset + s, offset + e, dtype=np.uint64)
        blk = idx >> np.uint64(1)
        x0, x1, x2, x3 = philox4x32_10(blk & MASK32, blk >> np.uint64(32), np.uint32(stream), np.uint32(0), k0, k1)
        u1 = ((x0 >> np.uint32(5)).astype(np.float64) * 67108864.0 + (x1 >> np.uint32(6)).astype(np.float64) + 0.5) * two53
        u2 = ((x2 >> np.uint32(5)).astype(np.float64) * 67108864.0 + (x3 >> np.uint32(6)).astype(np.float64) + 0.5) * two53
        r = np.sqrt(-2.0 * np.log(u1))
        ang = 2.0 * np.pi * u2
        odd = (idx & np.uint64(1)).astype(bool)
        out[s:e] = np.where(odd, r * np.sin(ang), r * np.cos(ang))
    return out


def uniforms(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform (0,1) doubles: entry k uses words (x0, x1) of block k."""
    k0, k1 = _key(seed)
    idx = np.arange(offset, offset + n, dtype=np.uint64)
    x0, x1, _, _ = philox4x32_10(idx & MASK32, idx >> np.uint64(32), np.uint32(stream), np.uint32(0), k0, k1)
    return ((x0 >> np.uint32(5)).astype(np.float64) * 67108864.0 + (x1 >> np.uint32(6)).astype(np.float64) + 0.5) * 2.0 ** -53


def omega(seed: int, d: int, l: int) -> np.ndarray:
    """The Gaussian sketch Omega (d x l, float64, Fortran order) drawn from stream 3."""
    return normals(seed, STREAM_OMEGA, d * l).reshape(l, d).T.copy(order="F") if l > 0 else np.zeros((d, 0), order="F")


# --------------------------------------------------------------------------------------
# Dense SPD: A = Q diag(lambda) Q^T, Q from the QR factorisation of a Gaussian matrix.
# --------------------------------------------------------------------------------------
def orthogonal_from_gaussian(seed: int, d: int) -> np.ndarray:
    g = normals(seed, STREAM_FACTORS, d * d).reshape(d, d)
    q, r = np.linalg.qr(g)
    q *= np.sign(np.diag(r))[None, :]
    return q


def dense_spd(seed: int, lam: np.ndarray) -> np.ndarray:
    """Row-major float64 A = Q diag(lam) Q^T, symmetrised."""
    d = lam.shape[0]
    q = orthogonal_from_gaussian(seed, d)
    a = (q * lam[None, :]) @ q.T
    return np.ascontiguousarray(0.5 * (a + a.T))


def decay_spectrum(d: int, scale: float = 1e4, floor: float = 1e-2) -> np.ndarray:
    """lambda_i = scale * i^-2 + floor, i = 1..d (the dense d=2000 workload)."""
    i = np.arange(1, d + 1, dtype=np.float64)
    return scale * i ** -2 + floor


def outlier_spectrum(d: int, k: int, out_lo: float, out_hi: float, bulk: float, seed: int) -> np.ndarray:
    """k log-uniform outliers in [out_lo, out_hi] over a flat bulk at `bulk`."""
    lam = np.full(d, bulk, dtype=np.float64)
    u = uniforms(seed, STREAM_SPECTRUM, k)
    lam[:k] = np.exp(np.log(out_lo) + u * (np.log(out_hi) - np.log(out_lo)))
    return np.sort(lam)[::-1].copy()


def dense_workload(seed: int = BASE_SEED + 1, d: int = 2000):
    """Dense FP64 system: decaying spectrum, b ~ N(0, I)."""
    lam = decay_spectrum(d)
    a = dense_spd(seed, lam)
    b = normals(seed, STREAM_RHS, d)
    return a, b, lam


# --------------------------------------------------------------------------------------
# Sparse SPD: variable-coefficient 7-point diffusion on an n^3 grid (CSR, int32 indices).
# --------------------------------------------------------------------------------------
def diffusion_csr(seed: int, n: int, dtype=np.float64):
    """Unscaled 7-point operator with log-normal face coefficients exp(N(0,1)).

    Cell (x, y, z) has index x + n*y + n*n*z. Every cell face carries a coefficient,
    including the faces on the domain boundary (homogeneous Dirichlet), so the
    diagonal is the sum of the six face coefficients and the matrix is SPD.
    Returns (rowptr int32, colidx int32, vals dtype, d).
    """
    d = n ** 3
    # faces normal to x: (n+1) x n x n, ordered (fx, y, z) with fx fastest; then y faces, then z faces.
    nf = (n + 1) * n * n
    g = normals(seed, STREAM_SPECTRUM, 3 * nf)
    cx = np.exp(g[:nf]).reshape(n, n, n + 1)          # [z, y, fx]
    cy = np.exp(g[nf:2 * nf]).reshape(n, n + 1, n)    # [z, fy, x]
    cz = np.exp(g[2 * nf:]).reshape(n + 1, n, n)      # [fz, y, x]
    # per-cell coefficients of the six faces, arrays shaped [z, y, x]
    w_xm, w_xp = cx[:, :, :-1], cx[:, :, 1:]
    w_ym, w_yp = cy[:, :-1, :], cy[:, 1:, :]
    w_zm, w_zp = cz[:-1, :, :], cz[1:, :, :]
    diag = (w_xm + w_xp + w_ym + w_yp + w_zm + w_zp).reshape(-1)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    x = x.reshape(-1); y = y.reshape(-1); z = z.reshape(-1)
    idx = np.arange(d, dtype=np.int64)
    # neighbours in increasing column order: z-1, y-1, x-1, self, x+1, y+1, z+1
    nb = [(idx - n * n, z > 0, w_zm.reshape(-1)),
          (idx - n, y > 0, w_ym.reshape(-1)),
          (idx - 1, x > 0, w_xm.reshape(-1)),
          (idx, np.ones(d, bool), None),
          (idx + 1, x < n - 1, w_xp.reshape(-1)),
          (idx + n, y < n - 1, w_yp.reshape(-1)),
          (idx + n * n, z < n - 1, w_zp.reshape(-1))]
    counts = np.zeros(d, dtype=np.int64)
    for _, m, _ in nb:
        counts += m
    rowptr = np.zeros(d + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    nnz = int(rowptr[-1])
    colidx = np.empty(nnz, dtype=np.int32)
    vals = np.empty(nnz, dtype=np.float64)
    pos = rowptr[:-1].copy()
    for col, m, w in nb:
        r = idx[m]
        p = pos[m]
        colidx[p] = col[m].astype(np.int32)
        vals[p] = diag[m] if w is None else -w[m]
        pos[m] += 1
    return rowptr.astype(np.int32), colidx, vals.astype(dtype), d


def diffusion_workload(seed: int = BASE_SEED + 2, n: int = 128):
    rowptr, colidx, vals, d = diffusion_csr(seed, n)
    b = normals(seed, STREAM_RHS, d)
    return rowptr, colidx, vals, b


def inner_start_block(r: np.ndarray, omega_unscaled: np.ndarray) -> np.ndarray:
    """The start block the solver uses for an inner solve on residual r:
    [r / ||r||, Omega / sqrt(d)] (column scaling leaves the column-0 iterate unchanged)."""
    d = r.shape[0]
    return np.column_stack([r / np.linalg.norm(r), omega_unscaled / np.sqrt(d)])


# --------------------------------------------------------------------------------------
# Ridge regression: Z = U diag(sigma) V^T + noise, f ~ N(0, I), b = Z^T f.
# --------------------------------------------------------------------------------------
def householder_orthonormal(seed: int, n: int, d: int, reflectors: int = 16, stream: int = STREAM_FACTORS,
                            offset: int = 0) -> np.ndarray:
    """First d columns of H_1 ... H_k (k Householder reflectors with Gaussian vectors),
    an n x d matrix with orthonormal columns."""
    Q = np.zeros((n, d))
    Q[np.arange(d), np.arange(d)] = 1.0
    for r in range(reflectors):
        v = normals(seed, stream, n, offset=offset + r * n)
        v /= np.linalg.norm(v)
        Q -= 2.0 * np.outer(v, v @ Q)
    return Q


def ridge_workload(seed: int, n: int, d: int, noise_std: float, dtype=np.float32):
    """Z (n x d, row-major, dtype) with singular values 1/i plus N(0, noise_std^2) noise,
    f ~ N(0, I_n) and b = Z^T f computed from the stored Z in float64."""
    U = householder_orthonormal(seed, n, d)
    V = householder_orthonormal(seed, d, d, offset=16 * n)
    sig = 1.0 / np.arange(1, d + 1)
    Z = (U * sig[None, :]) @ V.T
    if noise_std > 0:
        Z += noise_std * normals(seed, STREAM_NOISE, n * d).reshape(n, d)
    Z = np.ascontiguousarray(Z.astype(dtype))
    f = normals(seed, STREAM_RHS, n)
    b = Z.astype(np.float64).T @ f
    return Z, f, b


def ridge_workload_torch(seed: int, n: int, d: int, noise_std: float, device, chunk: int = 1 << 14):
    """ridge_workload's construction on a CUDA device, for sizes the host cannot build
    quickly: Z = H_16 ... H_1 [diag(1/i) V^T; 0] with the same reflector vectors (with
    noise_std = 0 it is ridge_workload's Z up to the FP32 rounding of the construction),
    stored in FP32 row-major. The noise N(0, noise_std^2) and f ~ N(0, I_n) come from
    torch's CUDA generator seeded with `seed` (the host Philox stream would take
    minutes at 8e8 entries). b = Z^T f in FP64 from the stored Z.
    Returns (Z, f, b) as device tensors."""
    import torch
    V = torch.eye(d, dtype=torch.float64, device=device)
    for r in range(16):
        v = torch.from_numpy(normals(seed, STREAM_FACTORS, d, offset=16 * n + r * d)).to(device)
        v /= torch.linalg.norm(v)
        V -= 2.0 * torch.outer(v, v @ V)
    sig = 1.0 / torch.arange(1, d + 1, dtype=torch.float64, device=device)
    Z = torch.zeros((n, d), dtype=torch.float32, device=device)
    Z[:d] = (sig[:, None] * V.T).to(torch.float32)
    del V
    for r in range(16):
        u = torch.from_numpy(normals(seed, STREAM_FACTORS, n, offset=r * n)).to(device)
        u = (u / torch.linalg.norm(u)).to(torch.float32)
        w = u @ Z
        Z.addr_(u, w, alpha=-2.0)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    if noise_std > 0:
        for s in range(0, n, chunk):
            e = min(n, s + chunk)
            Z[s:e] += noise_std * torch.randn((e - s, d), generator=g, device=device, dtype=torch.float32)
    f = torch.randn(n, generator=g, device=device, dtype=torch.float64)
    b = torch.zeros(d, dtype=torch.float64, device=device)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        b += Z[s:e].to(torch.float64).T @ f[s:e]
    return Z, f, b


# --------------------------------------------------------------------------------------
# Gaussian sampling: RBF kernel on uniform points in [0, 1]^3.
# --------------------------------------------------------------------------------------
def rbf_points(seed: int, n: int) -> np.ndarray:
    return uniforms(seed, STREAM_FACTORS, 3 * n).reshape(n, 3)


def rbf_kernel(points: np.ndarray, lengthscale: float = 0.2, dtype=np.float64, chunk: int = 2048) -> np.ndarray:
    """K_ij = exp(-||x_i - x_j||^2 / (2 lengthscale^2)), row-major, built in row chunks."""
    n = points.shape[0]
    K = np.empty((n, n), dtype=dtype)
    sq = (points ** 2).sum(1)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        d2 = sq[s:e, None] + sq[None, :] - 2.0 * points[s:e] @ points.T
        np.maximum(d2, 0.0, out=d2)
        K[s:e] = np.exp(-d2 / (2.0 * lengthscale ** 2)).astype(dtype)
    return K


def rbf_kernel_torch(points: np.ndarray, device, lengthscale: float = 0.2, chunk: int = 4096):
    """rbf_kernel on a CUDA device: FP64 arithmetic in row chunks, stored in FP32."""
    import torch
    x = torch.from_numpy(np.asarray(points, dtype=np.float64)).to(device)
    n = x.shape[0]
    K = torch.empty((n, n), dtype=torch.float32, device=device)
    sq = (x * x).sum(1)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        d2 = sq[s:e, None] + sq[None, :] - 2.0 * (x[s:e] @ x.T)
        d2.clamp_(min=0.0)
        K[s:e] = torch.exp(-d2 / (2.0 * lengthscale ** 2)).to(torch.float32)
    return K


def sample_block(seed: int, d: int, m: int) -> np.ndarray:
    """B (d x m, Fortran order) of standard normals from the right-hand-side stream."""
    return normals(seed, STREAM_RHS, d * m).reshape(m, d).T.copy(order="F")


# --------------------------------------------------------------------------------------
# Batched uneven systems: A_i = Q_i diag(lambda_i) Q_i^T, Q_i a product of Householder
# reflectors; k_i ~ U{1..64} outliers log-uniform in [1e2, 1e5] over a bulk U[1, 10].
# --------------------------------------------------------------------------------------
def batch_sizes(seed: int, n: int, dmin: int = 500, dmax: int = 16000) -> np.ndarray:
    u = uniforms(seed, STREAM_SPECTRUM, n)
    return np.rint(np.exp(np.log(dmin) + u * (np.log(dmax) - np.log(dmin)))).astype(np.int64)


def batch_spectrum(seed: int, i: int, d: int) -> np.ndarray:
    """Spectrum of system i: outliers first (descending), then the bulk."""
    u = uniforms(seed + 1 + i, STREAM_SPECTRUM, d + 70)
    k = min(d, 1 + int(u[0] * 64))
    out = np.exp(np.log(1e2) + u[1:1 + k] * (np.log(1e5) - np.log(1e2)))
    bulk = 1.0 + 9.0 * u[70:70 + d - k]
    return np.concatenate([np.sort(out)[::-1], bulk])


def batch_reflectors(seed: int, i: int, d: int, r: int = 16) -> np.ndarray:
    v = normals(seed + 1 + i, STREAM_FACTORS, r * d).reshape(r, d)
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def batch_system(seed: int, i: int, d: int, dtype=np.float32):
    """A_i (d x d row-major, dtype) and b_i ~ N(0, I). The reflectors H = I - 2 v v^T are
    applied to diag(lambda) from both sides in float64: A <- A - 2 v w^T - 2 w v^T +
    4 (v.w) v v^T with w = A v."""
    lam = batch_spectrum(seed, i, d)
    A = np.diag(lam)
    for v in batch_reflectors(seed, i, d):
        w = A @ v
        A -= 2.0 * np.outer(v, w) + 2.0 * np.outer(w, v) - 4.0 * (v @ w) * np.outer(v, v)
    A = np.ascontiguousarray(0.5 * (A + A.T)).astype(dtype)
    b = normals(seed + 1 + i, STREAM_RHS, d)
    return A, b


def batch_system_torch(seed: int, i: int, d: int, device, dtype=None, pitch: int = 32):
    """The same A_i as batch_system, formed on a CUDA device with torch (float64, then
    rounded); for batches too large to build on the host. Rows are stored with a pitch
    rounded up to a multiple of `pitch` elements (a strided view), so every row starts
    on a 16-byte boundary."""
    import torch
    dtype = torch.float32 if dtype is None else dtype
    lam = torch.from_numpy(batch_spectrum(seed, i, d)).to(device)
    A = torch.diag(lam)
    for v in torch.from_numpy(batch_reflectors(seed, i, d)).to(device):
        w = A @ v
        A -= 2.0 * torch.outer(v, w) + 2.0 * torch.outer(w, v) - 4.0 * torch.dot(v, w) * torch.outer(v, v)
    A = (0.5 * (A + A.T)).to(dtype)
    ldp = (d + pitch - 1) // pitch * pitch
    buf = torch.zeros((d, ldp), dtype=dtype, device=device)
    buf[:, :d] = A
    del A
    b = torch.from_numpy(normals(seed + 1 + i, STREAM_RHS, d)).to(device)
    return buf[:, :d], b
