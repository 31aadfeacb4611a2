"""bk_apply_ozaki (dense FP32 A times FP64 X on the BF16 tensor cores, error-free
digit splitting) against the oracle's FP64-accurate product, element by element, and
the sampling drivers in the BK_PREC_OZAKI mode against the oracle's
eigendecomposition."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2501_18717_gb300 import workloads as W  # noqa: E402
from oracle import accurate, direct  # noqa: E402

KB = 512  # the K block of the splitting (one scale per row / column and block)


@pytest.fixture(scope="module")
def bk():
    from paper_2501_18717_gb300 import bk as _bk
    return _bk


@pytest.fixture(scope="module")
def ctx(bk):
    c = bk.Context(0)
    yield c
    c.close()


def block_bound(A32, X):
    """sum_k 2^eA(i,k) 2^eX(k,j): 2^e bounds the magnitudes of the 512-element block
    (of row i of A, of column j of X) that k falls in; the documented error scale."""
    A = np.abs(np.asarray(A32, dtype=np.float64))
    X = np.abs(np.asarray(X, dtype=np.float64))
    d = A.shape[0]
    out = np.zeros((d, X.shape[1]))
    for k0 in range(0, d, KB):
        k1 = min(d, k0 + KB)
        ma = A[:, k0:k1].max(axis=1)
        mx = X[k0:k1].max(axis=0)
        ba = np.where(ma > 0, np.exp2(np.frexp(ma)[1].astype(np.float64)), 0.0)
        bx = np.where(mx > 0, np.exp2(np.frexp(mx)[1].astype(np.float64)), 0.0)
        out += (k1 - k0) * np.outer(ba, bx)
    return out


def run(bk, ctx, A32, X, mu=0.0, device=True):
    d, L = X.shape
    if device:
        Xt = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()  # column-major d x L
        Yt = torch.zeros((L, d), dtype=torch.float64, device="cuda")
        bk.apply(ctx, bk.dense_operator(torch.from_numpy(A32).cuda()), mu, Xt.T, Yt.T, ozaki=True)
        return Yt.cpu().numpy().T
    Y = np.zeros((d, L), order="F")
    bk.apply(ctx, bk.dense_operator(A32), mu, np.asfortranarray(X), Y, ozaki=True)
    return Y


@pytest.mark.parametrize("kind,d,L,mu", [("gaussian", 1537, 3, 0.25), ("gaussian", 700, 65, 0.0),
                                         ("rbf", 2000, 8, 1e-6), ("tiny", 5, 2, 0.0)])
def test_ozaki_matches_accurate_product(bk, ctx, kind, d, L, mu):
    """Every entry within 2^-44 of the block-bound scale (the documented bound; ragged
    row tiles, K blocks and column tiles, two column tiles at L = 65). For the RBF
    kernel matrix of the sampling configuration the error is also within 2^-40 of
    sum |a_ik x_k|."""
    rng = np.random.default_rng(d + L)
    if kind == "rbf":
        A = W.rbf_kernel(W.rbf_points(W.BASE_SEED + 4, 40000)[:d], dtype=np.float32)
    else:
        A = rng.standard_normal((d, d)).astype(np.float32)
    X = rng.standard_normal((d, L))
    Y = run(bk, ctx, A, X, mu)
    ref = accurate.matmul(A, X, mu)
    err = np.abs(Y - ref)
    assert np.all(err <= 2.0 ** -44 * block_bound(A, X) + 1e-300), np.max(err / block_bound(A, X))
    if kind == "rbf":
        assert np.all(err <= 2.0 ** -40 * accurate.abs_products(A, X)), np.max(err / accurate.abs_products(A, X))


def test_ozaki_is_exact_on_integers(bk, ctx):
    """Integer A and X whose digit expansions are short: every digit product and every
    tensor-core partial sum is an exact integer, so Y equals the exact product bit for
    bit (it would not if the tensor core's FP32 accumulation lost bits of the sums)."""
    rng = np.random.default_rng(11)
    d, L = 3000, 4
    A = rng.integers(-2000, 2001, (d, d)).astype(np.float32)
    X = rng.integers(-2000, 2001, (d, L)).astype(np.float64)
    Y = run(bk, ctx, A, X)
    ref = A.astype(np.float64) @ X  # exact: every partial sum is an integer below 2^53
    np.testing.assert_array_equal(Y, ref)


def test_ozaki_exponent_range_and_zero_blocks(bk, ctx):
    """Rows of A scaled by 2^-120 and 2^100, a zero row, a zero 512-block of a row, X
    columns scaled by 2^-600 and 2^500 (beyond FP32 range, the exponents are carried
    apart from the digits); host arrays with leading dimensions above d."""
    rng = np.random.default_rng(12)
    d, L = 1200, 4
    A = rng.standard_normal((d, d)).astype(np.float32)
    A[3] *= np.float32(2.0 ** -120)
    A[4] *= np.float32(2.0 ** 100)
    A[5] = 0
    A[6, 512:1024] = 0
    X = rng.standard_normal((d, L))
    X[:, 1] *= 2.0 ** -600
    X[:, 2] *= 2.0 ** 500
    ref = accurate.matmul(A, X)
    Xh = np.zeros((d + 7, L), order="F")
    Xh[:d] = X
    Yh = np.zeros((d + 3, L), order="F")
    bk.apply(ctx, bk.dense_operator(A), 0.0, Xh, Yh, ldx=d + 7, ldy=d + 3, ozaki=True)
    Y = Yh[:d]
    assert np.all(Y[5] == 0)
    assert np.all(np.abs(Y - ref) <= 2.0 ** -44 * block_bound(A, X) + 1e-300)
    np.testing.assert_array_equal(Y, run(bk, ctx, A, X))  # device arrays: same result


def test_ozaki_rejects_other_operators(bk, ctx):
    X = np.ones((4, 1), order="F")
    Y = np.zeros((4, 1), order="F")
    with pytest.raises(bk.BKError) as e:
        bk.apply(ctx, bk.dense_operator(np.eye(4)), 0.0, X, Y, ozaki=True)  # FP64 values
    assert e.value.status == bk.BK_ERR_UNSUPPORTED
    rp, ci, va, d = W.diffusion_csr(W.BASE_SEED, 3)
    with pytest.raises(bk.BKError) as e:
        bk.apply(ctx, bk.csr_operator(rp, ci, va.astype(np.float32)), 0.0, np.ones((d, 1), order="F"),
                 np.zeros((d, 1), order="F"), ozaki=True)
    assert e.value.status == bk.BK_ERR_UNSUPPORTED


@pytest.mark.parametrize("fn", ["sqrt", "isqrt"])
def test_sampling_ozaki_mode(bk, ctx, fn):
    """The sampling configuration's 2000-point validation problem (K stored in FP32,
    nugget 1e-6, 256 samples, 32 nodes) with the loads on the tensor cores, against the
    oracle's eigendecomposition of the stored K promoted to FP64, at the bounds of the
    compensated-pair mode."""
    d, m = 2000, 256
    K = W.rbf_kernel(W.rbf_points(W.BASE_SEED + 4, 40000)[:d], dtype=np.float32)
    B = W.sample_block(W.BASE_SEED + 4, 40000, m)[:d].copy(order="F")
    S = np.zeros((d, m), order="F")
    call = bk.sample if fn == "sqrt" else bk.sample_isqrt
    info = call(ctx, bk.dense_operator(torch.from_numpy(K).to("cuda:0")), 1e-6, B, S, 32,
                bk.default_opts(tol=1e-10, inner="ozaki", check_every=2, max_loads=64), check=False)
    assert info.status == bk.BK_OK, info.as_dict()
    if fn == "sqrt":
        ref = direct.sqrtm_apply(K.astype(np.float64), B, shift=1e-6)
        tol = 1e-7
    else:
        ref = direct.isqrtm_apply(K.astype(np.float64), B, shift=1e-6)
        lam = np.linalg.eigvalsh(K.astype(np.float64)) + 1e-6
        tol = 1e-13 * lam[-1] / lam[0]
    err = np.linalg.norm(S - ref) / np.linalg.norm(ref)
    assert err <= tol, (err, tol, info.as_dict())


def test_ozaki_gram_form_matches_accurate_product(bk, ctx):
    """Z^T (Z X) for the ridge configuration's Z shape (here 5003 x 300: ragged row
    tiles of Z^T and K blocks of both products), 4 columns, mu 0.5, against the
    oracle's accurate products (V = Z X, then Z^T V): within 2^-40 of
    sum_i |z_ik| (|Z| |X|)_i, the scale of the two rounded products."""
    n, d, L = 5003, 300, 4
    rng = np.random.default_rng(21)
    Z = W.ridge_workload(W.BASE_SEED + 22, n, d, 1e-3)[0].astype(np.float32)
    X = rng.standard_normal((d, L))
    Y = np.zeros((d, L), order="F")
    bk.apply(ctx, bk.gram_operator(Z), 0.5, np.asfortranarray(X), Y, ozaki=True)
    V = np.stack([accurate.matvec(Z, X[:, j]) for j in range(L)], axis=1)
    ref = np.stack([accurate.matvec(np.ascontiguousarray(Z.T), V[:, j]) for j in range(L)], axis=1) + 0.5 * X
    scale = np.abs(Z.astype(np.float64)).T @ (np.abs(Z.astype(np.float64)) @ np.abs(X))
    assert np.all(np.abs(Y - ref) <= 2.0 ** -40 * scale), np.max(np.abs(Y - ref) / scale)
