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


@pytest.mark.parametrize("inner", ["fp64", "fp32", "f32x2", "bf16"])
def test_ridge_gram_path(bk, ctx, inner):
    """A = Z^T Z matrix-free (two products over Z per load), FP32 Z. bf16: the loads on
    the BF16 tensor cores (head/tail splits), FP64-accurate refinement residuals."""
    n, d, l = 3000, 256, 16
    Z, f, b = W.ridge_workload(W.BASE_SEED + 22, n, d, noise_std=1e-3)
    mus = np.logspace(-6, 0, 20)
    tol = 1e-8 if inner in ("fp32", "bf16") else 1e-10
    X = np.zeros((d, len(mus)), order="F")
    info = bk.ridge_path(ctx, bk.gram_operator(torch.from_numpy(Z).to(dev())), mus, b, X,
                         bk.default_opts(tol=tol, sketch=l, seed=6, inner=inner,
                                         inner_tol=1e-5 if inner in ("fp32", "bf16") else 1e-6))
    op = operators.Gram(Z.astype(np.float64))
    res = shift_residuals(op, mus, X, b)
    assert res.max() <= tol, (res.max(), info.as_dict())
    assert info.loads <= 40 * info.refinements


@pytest.mark.parametrize("d,inner", [(300, "fp32"), (257, "fp32"), (300, "bf16"), (257, "bf16")])
def test_ridge_gram_tiles_and_ragged_edges(bk, ctx, d, inner):
    """Block width 65 (sketch 64) over ragged row and column tiles. d = 300 runs the
    tall-skinny product kernels (FP32 loads, compensated FP64-accurate residuals) with a
    partial last tile in both dimensions; d = 257 has rows that are not 16-byte aligned
    and takes the general GEMM. bf16: the BF16 tensor-core loads, whose TMA boxes run
    past the last 64-wide K slice and the last 128-row tile (zero fill) in both products.
    All must meet 1e-8 in the oracle's FP64 residual."""
    n = 5003
    Z, f, b = W.ridge_workload(W.BASE_SEED + 23, n, d, noise_std=1e-3)
    mus = np.logspace(-6, 0, 20)
    X = np.zeros((d, len(mus)), order="F")
    info = bk.ridge_path(ctx, bk.gram_operator(torch.from_numpy(Z).to(dev())), mus, b, X,
                         bk.default_opts(tol=1e-8, sketch=64, seed=7, inner=inner, inner_tol=1e-5, check_every=2))
    op = operators.Gram(Z.astype(np.float64))
    res = shift_residuals(op, mus, X, b)
    assert res.max() <= 1e-8, (res.max(), info.as_dict())
    ref = direct.ridge_path(op.matrix(), mus, b)
    np.testing.assert_allclose(X, ref, rtol=0, atol=1e-6 * np.abs(ref).max())


def test_ridge_generator_matches_host_construction():
    """The device generator of the full-size ridge inputs builds the same Z as the
    host generator (noise off): same reflectors, same singular values."""
    n, d = 3000, 96
    Zh, _, _ = W.ridge_workload(W.BASE_SEED + 24, n, d, noise_std=0.0)
    Zd, f, b = W.ridge_workload_torch(W.BASE_SEED + 24, n, d, 0.0, dev())
    Zd = Zd.cpu().numpy()
    assert np.max(np.abs(Zd - Zh)) <= 1e-6 * np.max(np.abs(Zh))
    np.testing.assert_allclose(b.cpu().numpy(), Zd.astype(np.float64).T @ f.cpu().numpy(), rtol=1e-12,
                               atol=1e-12 * np.abs(b.cpu().numpy()).max())
