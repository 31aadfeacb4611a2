"""bk_solve_shrink (block-CG whose block shrinks to one column after s_lock steps: the
outlook's deflation to a smaller block, Sec. CG_pro's locked reorthogonalisation)
against the FP64 oracle's Def-CG on the locked basis."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2501_18717_gb300 import workloads as W  # noqa: E402
from oracle import deflated, direct, operators  # noqa: E402


@pytest.fixture(scope="module")
def bk():
    from paper_2501_18717_gb300 import bk as _bk
    return _bk


@pytest.fixture(scope="module")
def ctx(bk):
    c = bk.Context(0)
    yield c
    c.close()


def _problem(d=300, seed=W.BASE_SEED + 60):
    lam = np.concatenate([1e3 * np.arange(1, 31, dtype=float) ** -2.0, np.linspace(0.5, 0.05, d - 30)])
    a = W.dense_spd(seed, lam)
    b = W.normals(seed, W.STREAM_RHS, d)
    return a, b


@pytest.mark.parametrize("s_lock,l", [(1, 10), (3, 10), (2, 0)])
def test_iterates_match_oracle(bk, ctx, s_lock, l):
    """After s_lock block loads, the load for r_0 and t one-column steps the GPU iterate
    equals the oracle's Def-CG iterate on the locked basis of K_s(A, [b Omega]) (same
    Omega). t = 0 is the block-CG iterate after s_lock loads. l = 0 is CG with s_lock
    locked Lanczos vectors. While the locked basis misses some of the 30 outliers
    (s_lock (l + 1) < 30), the one-column phase amplifies rounding differences about 20x
    per step once Ritz values of the missed outliers converge (a CPU restatement of this
    driver, with the 2^-44 error of its pair-arithmetic basis products, against the
    oracle: 7e-11 apart at t = 6, 5e-6 at t = 10), so those cases stop at t = 6;
    s_lock = 3, l = 10 locks 33 vectors and is compared up to t = 10 (1e-12 there)."""
    a, b = _problem()
    d, mu, seed = a.shape[0], 1e-3, 61
    om = W.omega(seed, d, l)
    ref = deflated.shrink_solve(a, mu, b, om, s_lock, 10)
    for t in [0, 1, 4, 6] + ([10] if s_lock * (l + 1) >= 30 else []):
        x = np.zeros(d)
        info = bk.solve_shrink(ctx, bk.dense_operator(a), mu, b, x, s_lock,
                               bk.default_opts(tol=1e-30, sketch=l, seed=seed, max_loads=s_lock + 1 + t,
                                               check_every=1), check=False)
        assert info.loads == s_lock + 1 + t and info.refinements == s_lock * (l + 1), info.as_dict()
        err = np.linalg.norm(x - ref[t]) / np.linalg.norm(ref[t])
        assert err <= 1e-9, (t, err)


def test_shrink_converges_csr(bk, ctx):
    """CSR diffusion 12^3 (FP64 values) to 1e-10 in the oracle's recomputed residual."""
    rp, ci, va, d = W.diffusion_csr(W.BASE_SEED + 62, 12)
    b = W.normals(W.BASE_SEED + 62, W.STREAM_RHS, d)
    mu = 1e-4
    op = bk.csr_operator(torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(), torch.from_numpy(va).cuda())
    x = np.zeros(d)
    info = bk.solve_shrink(ctx, op, mu, b, x, 2, bk.default_opts(tol=1e-10, sketch=16, seed=63, max_loads=5000,
                                                               check_every=4))
    res = direct.rel_residual(operators.CSR(rp, ci, va), mu, x, b)
    assert res <= 1e-10, (res, info.as_dict())
    assert info.loads < 400, info.as_dict()


def test_shrink_gram_fp32(bk, ctx):
    """A = Z^T Z matrix-free with FP32 Z (compensated one-column products): 1e-10 in the
    oracle's residual from the stored Z promoted to FP64."""
    Z, f, b = W.ridge_workload(W.BASE_SEED + 64, 2000, 128, noise_std=1e-3)
    mu = 1e-4
    x = np.zeros(128)
    info = bk.solve_shrink(ctx, bk.gram_operator(torch.from_numpy(Z).cuda()), mu, b, x, 2,
                           bk.default_opts(tol=1e-10, sketch=8, seed=65, max_loads=2000, check_every=2))
    res = direct.rel_residual(operators.Gram(Z.astype(np.float64)), mu, x, b)
    assert res <= 1e-10, (res, info.as_dict())


def test_shrink_edge_cases(bk, ctx):
    a, b = _problem(d=40)
    x = np.ones(40)
    info = bk.solve_shrink(ctx, bk.dense_operator(a), 0.1, np.zeros(40), x, 1, bk.default_opts(sketch=4))
    assert info.status == bk.BK_OK and np.all(x == 0.0)
    # a block as wide as d: the locked basis spans R^d and x_0 is the solution
    x = np.zeros(40)
    info = bk.solve_shrink(ctx, bk.dense_operator(a), 0.1, b, x, 1,
                           bk.default_opts(tol=1e-11, sketch=64, check_every=1, max_loads=50))
    assert direct.rel_residual(operators.Dense(a), 0.1, x, b) <= 1e-11 and info.loads <= 4, info.as_dict()
    with pytest.raises(bk.BKError):
        bk.solve_shrink(ctx, bk.dense_operator(a), 0.1, b, x, 0, bk.default_opts(sketch=4))
    # (s_lock + 1)(1 + sketch) > 768 columns of [V Q_s]: refused before any device work
    with pytest.raises(bk.BKError) as e:
        bk.solve_shrink(ctx, bk.dense_operator(np.eye(400)), 0.0, np.ones(400), np.zeros(400), 3,
                        bk.default_opts(sketch=200))
    assert e.value.status == bk.BK_ERR_UNSUPPORTED


def test_shrink_dense_fp32_values(bk, ctx):
    """Dense FP32 values (single-column products through the compensated FP32-pair
    kernels): 1e-10 in the oracle's residual of the stored matrix promoted to FP64."""
    a, b = _problem(d=320)
    a32 = np.ascontiguousarray(a.astype(np.float32))
    x = np.zeros(320)
    info = bk.solve_shrink(ctx, bk.dense_operator(torch.from_numpy(a32).cuda()), 1e-3, b, x, 2,
                           bk.default_opts(tol=1e-10, sketch=12, seed=66, max_loads=3000, check_every=4))
    res = direct.rel_residual(operators.Dense(a32.astype(np.float64)), 1e-3, x, b)
    assert res <= 1e-10, (res, info.as_dict())


def test_shrink_rbf_operator(bk, ctx):
    """The kernel matrix formed on the fly (BK_RBF, 500 points, lengthscale 0.2): 1e-9
    in the residual the oracle recomputes from its FP64 kernel matrix. The on-the-fly
    products carry about 2^-44 of sum |K_ij x_j|, so the reachable relative residual is
    about 6e-14 ||K|| ||x|| / ||b|| <= 6e-14 ||K|| / mu: 3e-11 at mu = 0.1 (||K|| = 44
    here), 3e-9 at mu = 1e-3."""
    d, mu = 500, 0.1
    pts = W.rbf_points(W.BASE_SEED + 67, d)
    K = W.rbf_kernel(pts)
    b = W.normals(W.BASE_SEED + 67, W.STREAM_RHS, d)
    x = np.zeros(d)
    info = bk.solve_shrink(ctx, bk.rbf_operator(torch.from_numpy(pts).cuda(), 0.2), mu, b, x, 2,
                           bk.default_opts(tol=1e-9, sketch=16, seed=68, max_loads=5000, check_every=4),
                           check=False)
    res = direct.rel_residual(operators.Dense(K), mu, x, b)
    assert info.status == bk.BK_OK and res <= 1e-9, (res, info.as_dict())
