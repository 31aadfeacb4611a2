"""GPU parity of the individual hot-path steps against the FP64 oracle / definitions.

Every call goes through the C ABI (libbk.so) via the ctypes binding.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2501_18717_gb300 import workloads as W  # noqa: E402
from oracle import operators  # noqa: E402


@pytest.fixture(scope="module")
def bk():
    from paper_2501_18717_gb300 import bk as _bk
    return _bk


@pytest.fixture(scope="module")
def ctx(bk):
    c = bk.Context(0)
    yield c
    c.close()


def dev():
    return torch.device("cuda:0")


def test_gaussian_matches_generator(bk, ctx):
    for seed, stream, n, off in [(1, 3, 10001, 0), (W.BASE_SEED, 3, 777, 13), (2**40 + 5, 7, 4096, 2**33 + 1)]:
        out = torch.empty(n, dtype=torch.float64, device=dev())
        bk.gaussian(ctx, seed, stream, out, offset=off)
        ref = W.normals(seed, stream, n, offset=off)
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("m", [1, 3, 8, 21, 33, 37, 65])
def test_gram(bk, ctx, dtype, m):
    d = 1000  # several 256/128-row tiles and a ragged tail
    ld = 1024
    rng = np.random.default_rng(m)
    npdt = np.float64 if dtype == "f64" else np.float32
    X = rng.standard_normal((d, m)).astype(npdt)
    Y = rng.standard_normal((d, m)).astype(npdt)
    Xt = torch.from_numpy(bk.to_panels(X, ld)).to(dev())
    Yt = torch.from_numpy(bk.to_panels(Y, ld)).to(dev())
    G = torch.zeros(m, m, dtype=torch.float64, device=dev())
    bk.gram(ctx, Xt, Yt, G, d, m, ld)
    Xr = X.astype(np.float64).T
    Yr = Y.astype(np.float64).T
    ref = Xr @ Yr.T
    ref = np.triu(ref) + np.triu(ref, 1).T  # the library returns the upper triangle mirrored
    tol = 1e-12 if dtype == "f64" else 2e-6
    scale = np.sqrt(np.outer(np.sum(Xr ** 2, 1), np.sum(Yr ** 2, 1)))
    assert np.max(np.abs(G.cpu().numpy() - ref) / scale) < tol


def test_chol_solve(bk, ctx):
    rng = np.random.default_rng(5)
    for m in [1, 2, 7, 21, 33, 36, 64, 65]:
        M = rng.standard_normal((m, m))
        G = M @ M.T + m * np.eye(m)
        S = rng.standard_normal((m, m))
        X = np.zeros((m, m))
        st = bk.chol_solve(ctx, G, S, X, m)
        assert st == bk.BK_OK
        np.testing.assert_allclose(X, np.linalg.solve(G, S), rtol=1e-10, atol=1e-12)
    G = np.ones((4, 4))  # rank one: breakdown
    assert bk.chol_solve(ctx, G, np.eye(4), np.zeros((4, 4)), 4) == bk.BK_BREAKDOWN


def _block(d, m, seed, npdt):
    """A random d x m block (NumPy, d x m)."""
    return np.random.default_rng(seed).standard_normal((d, m)).astype(npdt)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("m", [1, 5, 21, 33, 40, 65])
def test_block_apply_csr(bk, ctx, dtype, m):
    n = 11  # d = 1331: ragged against the row tiles
    rp, ci, va, d = W.diffusion_csr(W.BASE_SEED + 50, n)
    npdt = np.float64 if dtype == "f64" else np.float32
    ld = d + 5
    P = _block(d, m, m, npdt)
    mu = 1e-2
    A = bk.csr_operator(torch.from_numpy(rp).to(dev()), torch.from_numpy(ci).to(dev()),
                        torch.from_numpy(va.astype(npdt)).to(dev()))
    Pt = torch.from_numpy(bk.to_panels(P, ld)).to(dev())
    Yt = torch.zeros_like(Pt)
    G = torch.zeros(m, m, dtype=torch.float64, device=dev())
    bk.block_apply(ctx, A, mu, Pt, Yt, G, m, ld)
    op = operators.CSR(rp, ci, va.astype(npdt))
    P64 = P.astype(np.float64)
    Yref = op.apply(P64, mu)
    Y = bk.from_panels(Yt.cpu().numpy(), d, m).astype(np.float64)
    # padding columns come back as zeros
    assert np.all(Yt.cpu().numpy()[:, :d][(m - 1) // 4, :, (m - 1) % 4 + 1:] == 0)
    tol = 1e-13 if dtype == "f64" else 3e-6
    assert np.max(np.abs(Y - Yref)) / np.max(np.abs(Yref)) < tol
    Gref = P64.T @ Y
    Gref = np.triu(Gref) + np.triu(Gref, 1).T
    assert np.max(np.abs(G.cpu().numpy() - Gref)) / np.max(np.abs(Gref)) < (1e-12 if dtype == "f64" else 2e-6)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("m", [1, 9, 21, 33, 65])
def test_block_apply_dense(bk, ctx, dtype, m):
    d = 333
    npdt = np.float64 if dtype == "f64" else np.float32
    a = W.dense_spd(W.BASE_SEED + 51, W.decay_spectrum(d, 1e2, 1e-1)).astype(npdt)
    ld = d + 3
    P = _block(d, m, 100 + m, npdt)
    mu = 0.5
    A = bk.dense_operator(torch.from_numpy(a).to(dev()))
    Pt = torch.from_numpy(bk.to_panels(P, ld)).to(dev())
    Yt = torch.zeros_like(Pt)
    G = torch.zeros(m, m, dtype=torch.float64, device=dev())
    bk.block_apply(ctx, A, mu, Pt, Yt, G, m, ld)
    P64 = P.astype(np.float64)
    Yref = operators.Dense(a).apply(P64, mu)
    Y = bk.from_panels(Yt.cpu().numpy(), d, m).astype(np.float64)
    tol = 1e-13 if dtype == "f64" else 5e-6
    assert np.max(np.abs(Y - Yref)) / np.max(np.abs(Yref)) < tol


def test_chol_solve_scaling_range(bk, ctx):
    """Diagonal scaling spans many orders of magnitude (Grams of nearly converged
    residuals): the solve stays accurate."""
    rng = np.random.default_rng(9)
    m = 33
    M = rng.standard_normal((m, m))
    base = M @ M.T + m * np.eye(m)
    for lo, hi in [(-30, 30), (-150, -100), (100, 150)]:
        dsc = 10.0 ** rng.uniform(lo, hi, m)
        G = base * np.outer(dsc, dsc)
        S = rng.standard_normal((m, m)) * dsc[:, None]
        X = np.zeros((m, m))
        assert bk.chol_solve(ctx, G, S, X, m) == bk.BK_OK
        Xr = np.linalg.solve(base, S / dsc[:, None]) / dsc[:, None]
        np.testing.assert_allclose(X, Xr, rtol=1e-9, atol=0)


def test_chol_solve_dependent_columns(bk, ctx):
    """A column in the span of earlier ones is dropped: bk_chol_solve reports it."""
    rng = np.random.default_rng(10)
    B = rng.standard_normal((50, 6))
    B = np.column_stack([B, B[:, 1] + 2 * B[:, 4]])
    G = B.T @ B
    assert bk.chol_solve(ctx, G, np.eye(7), np.zeros((7, 7)), 7) == bk.BK_BREAKDOWN
