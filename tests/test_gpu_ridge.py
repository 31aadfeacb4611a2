"""bk_ridge_path against the FP64 oracle: one block-Lanczos basis for every shift."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2501_18717_gb300 import workloads as W  # noqa: E402
from oracle import direct, lanczos, operators  # noqa: E402


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


def shift_residuals(op, mus, X, b):
    return np.array([direct.rel_residual(op, mu, X[:, j], b) for j, mu in enumerate(mus)])


def test_ridge_iterates_match_oracle_lanczos(bk, ctx):
    """With a fixed number of loads and no refinement, the GPU combine equals the oracle's
    block-Lanczos shifted iterates on the same start block (Eq. bcg_alg)."""
    d, l, seed = 240, 7, 77
    a = W.dense_spd(W.BASE_SEED + 20, np.logspace(0, 2, d))
    b = W.normals(W.BASE_SEED + 20, W.STREAM_RHS, d)
    mus = np.logspace(-3, 0, 6)
    B = W.inner_start_block(b, W.omega(seed, d, l))
    for t in [1, 2, 4]:
        X = np.zeros((d, len(mus)), order="F")
        bk.ridge_path(ctx, bk.dense_operator(a), mus, b, X,
                      bk.default_opts(tol=1e-14, inner_tol=1e-15, sketch=l, seed=seed, max_loads=t, max_refine=1,
                                      check_every=1), check=False)
        lz = lanczos.block_lanczos(a, B, t)
        ref = lanczos.shifted_iterates(lz, mus) * np.linalg.norm(b)
        assert np.max(np.abs(X - ref)) / np.max(np.abs(ref)) < 1e-9, t


@pytest.mark.parametrize("inner", ["fp64", "fp32"])
def test_ridge_dense_path(bk, ctx, inner):
    d, l = 500, 12
    a = W.dense_spd(W.BASE_SEED + 21, np.concatenate([np.logspace(4, 2, 10), np.linspace(1.0, 0.01, d - 10)]))
    b = W.normals(W.BASE_SEED + 21, W.STREAM_RHS, d)
    mus = np.logspace(-4, 0, 16)
    tol = 1e-10 if inner == "fp64" else 1e-8
    A = bk.dense_operator(torch.from_numpy(a if inner == "fp64" else a.astype(np.float32)).to(dev()))
    X = np.zeros((d, len(mus)), order="F")
    info = bk.ridge_path(ctx, A, mus, b, X, bk.default_opts(tol=tol, sketch=l, seed=5, inner=inner,
                                                            inner_tol=1e-6 if inner == "fp64" else 1e-5))
    aa = a if inner == "fp64" else a.astype(np.float32).astype(np.float64)
    res = shift_residuals(operators.Dense(aa), mus, X, b)
    assert res.max() <= tol, (res.max(), info.as_dict())
    np.testing.assert_allclose(X, direct.ridge_path(aa, mus, b), rtol=0, atol=1e-4 * np.abs(X).max())


@pytest.mark.parametrize("inner", ["fp64", "fp32"])
def test_ridge_gram_path(bk, ctx, inner):
    """A = Z^T Z matrix-free (two products over Z per load), FP32 Z."""
    n, d, l = 3000, 256, 16
    Z, f, b = W.ridge_workload(W.BASE_SEED + 22, n, d, noise_std=1e-3)
    mus = np.logspace(-6, 0, 20)
    tol = 1e-10 if inner == "fp64" else 1e-8
    X = np.zeros((d, len(mus)), order="F")
    info = bk.ridge_path(ctx, bk.gram_operator(torch.from_numpy(Z).to(dev())), mus, b, X,
                         bk.default_opts(tol=tol, sketch=l, seed=6, inner=inner,
                                         inner_tol=1e-6 if inner == "fp64" else 1e-5))
    op = operators.Gram(Z.astype(np.float64))
    res = shift_residuals(op, mus, X, b)
    assert res.max() <= tol, (res.max(), info.as_dict())
    assert info.loads <= 40 * info.refinements
