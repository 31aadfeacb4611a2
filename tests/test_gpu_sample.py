"""bk_sample (block-Lanczos square root, Def. blansq) against the FP64 oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2501_18717_gb300 import workloads as W  # noqa: E402
from oracle import direct, lanczos  # noqa: E402


@pytest.fixture(scope="module")
def bk():
    from paper_2501_18717_gb300 import bk as _bk
    return _bk


@pytest.fixture(scope="module")
def ctx(bk):
    c = bk.Context(0)
    yield c
    c.close()


def test_sample_matches_exact_integral_on_same_basis(bk, ctx):
    """At a fixed number of loads the quadrature result equals the oracle's exact
    integral of Def. blansq on the same basis up to the quadrature error."""
    d, m = 300, 12
    pts = W.rbf_points(W.BASE_SEED + 30, d)
    K = W.rbf_kernel(pts)
    nug = 1e-2
    B = W.sample_block(W.BASE_SEED + 30, d, m)
    for t in [2, 4]:
        S = np.zeros((d, m), order="F")
        bk.sample(ctx, bk.dense_operator(K), nug, B, S, 32,
                  bk.default_opts(tol=1e-14, max_loads=t, check_every=100), check=False)
        lz = lanczos.block_lanczos(K + nug * np.eye(d), B, t)
        ref = lanczos.sqrt_iterate(lz)
        assert np.linalg.norm(S - ref) / np.linalg.norm(ref) < 1e-9, t


@pytest.mark.parametrize("inner", ["fp64", "fp32"])
def test_sample_converges_to_sqrt(bk, ctx, inner):
    d, m = 600, 32
    pts = W.rbf_points(W.BASE_SEED + 31, d)
    K = W.rbf_kernel(pts, dtype=np.float64 if inner == "fp64" else np.float32)
    nug = 1e-3
    B = W.sample_block(W.BASE_SEED + 31, d, m)
    S = np.zeros((d, m), order="F")
    info = bk.sample(ctx, bk.dense_operator(torch.from_numpy(K).to("cuda:0")), nug, B, S, 32,
                     bk.default_opts(tol=1e-10, inner=inner, check_every=4))
    ref = direct.sqrtm_apply(K.astype(np.float64), B, shift=nug)
    err = np.max(np.linalg.norm(S - ref, axis=0) / np.linalg.norm(ref, axis=0))
    # FP64 basis: 1e-8. FP32 basis: the basis and its products carry FP32 rounding
    # u = 2^-24, amplified by at most sqrt(kappa(A)) in the square root; allow 20 u sqrt(kappa).
    lam = np.linalg.eigvalsh(K.astype(np.float64)) + nug
    tol = 1e-8 if inner == "fp64" else 20 * 2.0 ** -24 * np.sqrt(lam[-1] / lam[0])
    assert err <= tol, (err, tol, info.as_dict())


@pytest.mark.parametrize("inner", ["fp64", "f32x2"])
def test_sample_rbf_subset_validation(bk, ctx, inner):
    """The sampling configuration's validation problem: the first 2000 of the seeded
    uniform points, K stored in FP32 (lengthscale 0.2), nugget 1e-6 as the shift, 256
    samples, 32 nodes; against the oracle's eigendecomposition of the stored K
    promoted to FP64. At this size the FP32 rounding of K (norm 4e-7) stays below the
    nugget, so K32 + 1e-6 I is positive definite (smallest eigenvalue 6.6e-7)."""
    d, m = 2000, 256
    pts = W.rbf_points(W.BASE_SEED + 4, 40000)[:d]
    K = W.rbf_kernel(pts, dtype=np.float32)
    B = W.sample_block(W.BASE_SEED + 4, 40000, m)[:d].copy(order="F")
    S = np.zeros((d, m), order="F")
    info = bk.sample(ctx, bk.dense_operator(torch.from_numpy(K).to("cuda:0")), 1e-6, B, S, 32,
                     bk.default_opts(tol=1e-10, inner=inner, check_every=2, max_loads=64), check=False)
    ref = direct.sqrtm_apply(K.astype(np.float64), B, shift=1e-6)
    err = np.linalg.norm(S - ref) / np.linalg.norm(ref)
    # K_t spans R^2000 after 8 loads, so only quadrature and rounding remain. An FP32
    # basis cannot resolve this spectrum (u ||K|| = 1e-5 exceeds the nugget: the shifted
    # projected systems become indefinite), hence FP64 blocks with FP64 or compensated
    # FP32-pair products (about 2^-44 relative, 1e-11 absolute here).
    assert info.status == bk.BK_OK, info.as_dict()
    tol = 1e-8 if inner == "fp64" else 1e-7
    assert err <= tol, (err, tol, info.as_dict())


def test_isqrt_matches_exact_integral_on_same_basis(bk, ctx):
    """The inverse square root at a fixed number of loads equals the oracle's exact
    integral on the same basis, Q_t T_t^{-1/2} E_1 R_0, up to the quadrature error."""
    d, m = 300, 12
    pts = W.rbf_points(W.BASE_SEED + 32, d)
    K = W.rbf_kernel(pts)
    nug = 1e-2
    B = W.sample_block(W.BASE_SEED + 32, d, m)
    for t in [2, 4]:
        S = np.zeros((d, m), order="F")
        bk.sample_isqrt(ctx, bk.dense_operator(K), nug, B, S, 32,
                        bk.default_opts(tol=1e-14, max_loads=t, check_every=100), check=False)
        lz = lanczos.block_lanczos(K + nug * np.eye(d), B, t)
        ref = lanczos.isqrt_iterate(lz)
        assert np.linalg.norm(S - ref) / np.linalg.norm(ref) < 1e-9, t


@pytest.mark.parametrize("d, m, nug, inner, tol", [(600, 32, 1e-3, "fp64", 1e-8), (2000, 256, 1e-6, "fp64", 1e-7),
                                                  (2000, 256, 1e-6, "f32x2", None)])
def test_isqrt_converges(bk, ctx, d, m, nug, inner, tol):
    """(K + nugget I)^{-1/2} B against the oracle's eigendecomposition of the stored K;
    the 2000-point case is the sampling configuration's validation problem (K in FP32).
    Compensated FP32-pair products carry about 1e-13 ||K|| absolute error; the inverse
    square root amplifies a perturbation of A by up to 1 / lambda_min relative, so the
    bound is 1e-13 ||K|| / lambda_min(K + nugget) (2.6e-5 here)."""
    pts = W.rbf_points(W.BASE_SEED + 4 if d == 2000 else W.BASE_SEED + 33, 40000 if d == 2000 else d)[:d]
    K = W.rbf_kernel(pts, dtype=np.float32 if d == 2000 else np.float64)
    B = (W.sample_block(W.BASE_SEED + 4, 40000, m)[:d].copy(order="F") if d == 2000
         else W.sample_block(W.BASE_SEED + 33, d, m))
    S = np.zeros((d, m), order="F")
    info = bk.sample_isqrt(ctx, bk.dense_operator(torch.from_numpy(K).to("cuda:0")), nug, B, S, 32,
                           bk.default_opts(tol=1e-10, inner=inner, check_every=2, max_loads=64), check=False)
    assert info.status == bk.BK_OK, info.as_dict()
    ref = direct.isqrtm_apply(K.astype(np.float64), B, shift=nug)
    err = np.linalg.norm(S - ref) / np.linalg.norm(ref)
    if tol is None:
        lam = np.linalg.eigvalsh(K.astype(np.float64)) + nug
        tol = 1e-13 * lam[-1] / lam[0]
    assert err <= tol, (err, tol, info.as_dict())


def test_rbf_operator_exact_integral_on_same_basis(bk, ctx):
    """The on-the-fly RBF operator (K never stored, entries in FP64): at a fixed number
    of loads the sample equals the oracle's exact integral on the basis built from the
    FP64 kernel matrix, so the operator matches K to the pair arithmetic's accuracy."""
    d, m = 333, 12
    pts = W.rbf_points(W.BASE_SEED + 34, d)
    K = W.rbf_kernel(pts)
    nug = 1e-2
    B = W.sample_block(W.BASE_SEED + 34, d, m)
    op = bk.rbf_operator(torch.from_numpy(pts).to("cuda:0"), 0.2)
    for t in [2, 4]:
        S = np.zeros((d, m), order="F")
        bk.sample(ctx, op, nug, B, S, 32, bk.default_opts(tol=1e-14, inner="f32x2", max_loads=t, check_every=100),
                  check=False)
        ref = lanczos.sqrt_iterate(lanczos.block_lanczos(K + nug * np.eye(d), B, t))
        assert np.linalg.norm(S - ref) / np.linalg.norm(ref) < 1e-9, t


@pytest.mark.parametrize("fn", ["sqrt", "isqrt"])
def test_rbf_operator_subset_literal_nugget(bk, ctx, fn):
    """The sampling validation problem with the kernel formed on the fly instead of
    stored in FP32: the first 2000 points, 256 samples, the configuration's nugget 1e-6,
    against the oracle's eigendecomposition of the FP64 kernel. An F32X2 basis is built
    with compensated-pair products (2^-44 each); over the steps and the two CholQR
    passes its relative accuracy is about 1e-12 ||K||, amplified by at most sqrt(kappa)
    (square root) or kappa (inverse square root) relative."""
    d, m, nug = 2000, 256, 1e-6
    pts = W.rbf_points(W.BASE_SEED + 4, 40000)[:d].copy()
    K = W.rbf_kernel(pts)
    B = W.sample_block(W.BASE_SEED + 4, 40000, m)[:d].copy(order="F")
    S = np.zeros((d, m), order="F")
    call = bk.sample if fn == "sqrt" else bk.sample_isqrt
    info = call(ctx, bk.rbf_operator(torch.from_numpy(pts).to("cuda:0"), 0.2), nug, B, S, 32,
                bk.default_opts(tol=1e-10, inner="f32x2", check_every=2, max_loads=64), check=False)
    assert info.status == bk.BK_OK, info.as_dict()
    ref = (direct.sqrtm_apply if fn == "sqrt" else direct.isqrtm_apply)(K, B, shift=nug)
    lam = np.linalg.eigvalsh(K) + nug
    kap = lam[-1] / lam[0]
    tol = 1e-12 * (np.sqrt(kap) if fn == "sqrt" else kap)
    err = np.linalg.norm(S - ref) / np.linalg.norm(ref)
    assert err <= max(tol, 1e-9), (err, tol, info.as_dict())
