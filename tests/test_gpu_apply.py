"""bk_apply, the FP64-accurate block product Y = A X + mu X (one matrix-load, Sec. 1.2),
against the oracle's FP64 product of the stored values; and the entries of the
on-the-fly RBF kernel (double-float exp) against NumPy's FP64 exp."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2501_18717_gb300 import workloads as W  # noqa: E402
from oracle import operators  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def bk():
    from paper_2501_18717_gb300 import bk as _bk
    return _bk


@pytest.fixture(scope="module")
def ctx(bk):
    c = bk.Context(0)
    yield c
    c.close()


def _cols(d, L, seed):
    return np.asfortranarray(np.random.default_rng(seed).standard_normal((d, L)))


def test_rbf_entries_match_fp64_exp(bk, ctx):
    """Columns e_j of the identity give columns of K exactly as the products carry them
    (one nonzero term), so Y holds the kernel's entries. Lengthscale 0.07 puts the
    exponents t = -|x_i - x_j|^2 / (2 l^2) over [-240, 0]: relative error <= 1e-13 for
    t >= -70 (the pair arithmetic's 2^-46 plus the exponent's FP64 rounding), absolute
    error <= 2^-126 for -100 <= t < -70 (the tail below the FP32 normal range), and 0
    below t = -100."""
    d, ell = 700, 0.07
    pts = W.rbf_points(W.BASE_SEED + 71, d)
    js = np.linspace(0, d - 1, 16).astype(int)
    X = np.zeros((d, len(js)), order="F")
    X[js, np.arange(len(js))] = 1.0
    Y = np.zeros_like(X)
    bk.apply(ctx, bk.rbf_operator(torch.from_numpy(pts).to(DEV), ell), 0.0, X, Y)
    diff = pts[:, None, :] - pts[None, js, :]
    t = -np.sum(diff * diff, axis=2) / (2.0 * ell * ell)
    ref = np.exp(t)
    hi = t >= -70.0
    mid = (t >= -100.0) & ~hi
    lo = t < -100.0
    assert hi.sum() > 1000 and mid.sum() > 100 and lo.sum() > 100  # the ranges are covered
    assert np.all(t[hi] >= -70.0) and t.min() < -100.0
    assert np.max(np.abs(Y[hi] - ref[hi]) / ref[hi]) <= 1e-13
    assert np.max(np.abs(Y[mid] - ref[mid])) <= 2.0 ** -126
    assert np.all(Y[lo] == 0.0)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_apply_dense_matches_oracle(bk, ctx, dtype):
    d, L, mu = 520, 7, 0.3
    A = W.dense_spd(W.BASE_SEED + 72, W.decay_spectrum(d, 1e3, 1e-1)).astype(dtype)
    X = _cols(d, L, 1)
    # device blocks, column-major d x L (transposed views of contiguous L x d tensors)
    Xd = torch.from_numpy(X.T.copy()).to(DEV).T
    Yd = torch.zeros((L, d), dtype=torch.float64, device=DEV).T
    bk.apply(ctx, bk.dense_operator(torch.from_numpy(A).to(DEV)), mu, Xd, Yd)
    got = Yd.cpu().numpy()
    A64 = A.astype(np.float64)
    ref = operators.Dense(A64).apply(X, mu)
    scale = np.abs(A64) @ np.abs(X) + abs(mu) * np.abs(X)
    # FP64 values: FP64 products, within (d + 1) u of sum |a||x|; FP32 values,
    # promoted: compensated pairs, about 2^-44
    tol = (d + 1) * 2.0 ** -53 if dtype == np.float64 else 1e-12
    assert np.max(np.abs(got - ref) / scale) <= tol


def test_apply_csr_host_arrays_and_leading_dimensions(bk, ctx):
    """Host X and Y (staged through the workspace) with ldy != ldx."""
    rp, ci, va, d = W.diffusion_csr(W.BASE_SEED + 73, 11)
    L, mu = 5, 1e-4
    ldx, ldy = d + 3, d + 9
    X = np.zeros((ldx, L), order="F")
    X[:d] = _cols(d, L, 2)
    Y = np.full((ldy, L), 7.0, order="F")
    bk.apply(ctx, bk.csr_operator(rp, ci, va), mu, X, Y, ldx=ldx, ldy=ldy)
    ref = operators.CSR(rp, ci, va).apply(X[:d], mu)
    scale = np.abs(operators.CSR(rp, ci, np.abs(va)).apply(np.abs(X[:d]), abs(mu)))
    assert np.max(np.abs(Y[:d] - ref) / scale) <= 8 * 2.0 ** -53  # eight terms a row
    assert np.all(Y[d:] == 7.0)  # rows beyond d untouched


def test_apply_gram_form_matches_oracle(bk, ctx):
    Z, _, _ = W.ridge_workload(W.BASE_SEED + 74, 1500, 132, noise_std=1e-3)
    d, L, mu = 132, 6, 1e-3
    X = _cols(d, L, 3)
    Y = np.zeros((d, L), order="F")
    bk.apply(ctx, bk.gram_operator(torch.from_numpy(Z).to(DEV)), mu, X, Y)
    Z64 = Z.astype(np.float64)
    ref = operators.Gram(Z64).apply(X, mu)
    scale = np.abs(Z64).T @ (np.abs(Z64) @ np.abs(X)) + abs(mu) * np.abs(X)
    assert np.max(np.abs(Y - ref) / scale) <= 1e-12


def test_apply_rejects_bad_arguments(bk, ctx):
    d = 64
    A = np.eye(d)
    X = np.zeros((d, 2), order="F")
    Y = np.zeros_like(X)
    op = bk.dense_operator(A)
    with pytest.raises(bk.BKError):
        bk.apply(ctx, op, float("nan"), X, Y)
    with pytest.raises(bk.BKError):
        bk.apply(ctx, op, 0.0, X, Y, ldx=d - 1)
