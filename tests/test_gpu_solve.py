"""End-to-end parity of bk_solve against the FP64 oracle (C ABI through the binding)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2501_18717_gb300 import workloads as W  # noqa: E402
from oracle import bcg, direct, operators  # noqa: E402


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


def test_iterate_parity_dense(bk, ctx):
    """After k loads (one inner solve, no refinement) the GPU iterate equals the
    oracle's block-CG recurrence on the same start block [b/||b||, Omega/sqrt(d)]."""
    d, l, seed = 400, 9, 1234
    a = W.dense_spd(W.BASE_SEED + 60, W.decay_spectrum(d, 1e2, 1.0))
    b = W.normals(W.BASE_SEED + 60, W.STREAM_RHS, d)
    mu = 1e-2
    B = W.inner_start_block(b, W.omega(seed, d, l))
    A = bk.dense_operator(torch.from_numpy(a).to(dev()))
    bt = torch.from_numpy(b).to(dev())
    # The recurrence amplifies rounding differences between any two implementations;
    # measure that amplification on the oracle itself (start block perturbed by 1e-14
    # relative) and allow 100 times it.
    Bp = B * (1 + 1e-14 * np.random.default_rng(0).standard_normal(B.shape))
    for k in [1, 2, 3, 6, 10]:
        x = torch.zeros(d, dtype=torch.float64, device=dev())
        info = bk.solve(ctx, A, mu, bt, x, bk.default_opts(tol=1e-14, inner_tol=1e-15, sketch=l, seed=seed,
                                                            max_loads=k, max_refine=1), check=False)
        assert info.loads == k
        ref = bcg.block_cg(a, mu, B[:, 0], B[:, 1:], tol=0.0, max_loads=k)
        refp = bcg.block_cg(a, mu, Bp[:, 0], Bp[:, 1:], tol=0.0, max_loads=k)
        xr = ref["x"] * np.linalg.norm(b)
        sens = np.linalg.norm(refp["x"] - ref["x"]) / np.linalg.norm(ref["x"])
        err = np.linalg.norm(x.cpu().numpy() - xr) / np.linalg.norm(xr)
        assert err < max(1e-11, 100 * sens), (k, err, sens)


@pytest.mark.parametrize("inner", ["fp64", "fp32"])
def test_iterate_parity_width65(bk, ctx, inner):
    """The widest block (l = 64, m = 65, padded to 68): after k loads the GPU iterate
    equals the oracle's block-CG recurrence on the same start block, FP64 blocks to the
    recurrence's rounding sensitivity, FP32 blocks (FP32-stored values) to FP32 level."""
    d, l, seed = 700, 64, 4321
    a = W.dense_spd(W.BASE_SEED + 61, W.decay_spectrum(d, 1e2, 1.0))
    if inner == "fp32":
        a = a.astype(np.float32)
    b = W.normals(W.BASE_SEED + 61, W.STREAM_RHS, d)
    mu = 1e-2
    B = W.inner_start_block(b, W.omega(seed, d, l))
    A = bk.dense_operator(torch.from_numpy(a).to(dev()))
    bt = torch.from_numpy(b).to(dev())
    Bp = B * (1 + 1e-14 * np.random.default_rng(1).standard_normal(B.shape))
    for k in [1, 2, 4]:
        x = torch.zeros(d, dtype=torch.float64, device=dev())
        info = bk.solve(ctx, A, mu, bt, x, bk.default_opts(tol=1e-14, inner_tol=1e-15, sketch=l, seed=seed,
                                                            inner=inner, max_loads=k, max_refine=1), check=False)
        assert info.loads == k
        a64 = a.astype(np.float64)
        ref = bcg.block_cg(a64, mu, B[:, 0], B[:, 1:], tol=0.0, max_loads=k)
        refp = bcg.block_cg(a64, mu, Bp[:, 0], Bp[:, 1:], tol=0.0, max_loads=k)
        xr = ref["x"] * np.linalg.norm(b)
        sens = np.linalg.norm(refp["x"] - ref["x"]) / np.linalg.norm(ref["x"])
        err = np.linalg.norm(x.cpu().numpy() - xr) / np.linalg.norm(xr)
        # FP32 blocks: unit roundoff 6e-8 amplified like a 1e-14 perturbation is by sens
        bound = max(1e-11, 100 * sens) if inner == "fp64" else max(1e-5, 100 * sens * 6e-8 / 1e-14)
        assert err < bound, (k, err, sens)


def test_dense_fp64_workload(bk, ctx):
    """The dense FP64 workload (d = 2000, lambda_i = 1e4 i^-2 + 1e-2, mu = 1e-3, l = 20):
    relative residual <= 1e-10 recomputed by the oracle in FP64."""
    a, b, lam = W.dense_workload()
    mu = 1e-3
    A = bk.dense_operator(torch.from_numpy(a).to(dev()))
    x = torch.zeros(2000, dtype=torch.float64, device=dev())
    info = bk.solve(ctx, A, mu, torch.from_numpy(b).to(dev()), x,
                    bk.default_opts(tol=1e-10, sketch=20, seed=W.BASE_SEED + 1))
    xs = x.cpu().numpy()
    rel = direct.rel_residual(operators.Dense(a), mu, xs, b)
    assert rel <= 1e-10, info.as_dict()
    xstar = direct.solve(a, mu, b)
    # forward error bounded by kappa(A_mu) * residual, kappa ~ 7.4e5
    assert np.linalg.norm(xs - xstar) / np.linalg.norm(xstar) < 1e-10 * 7.5e5
    assert info.loads < 400


@pytest.mark.parametrize("inner,tol", [("fp64", 1e-10), ("fp32", 1e-8)])
@pytest.mark.parametrize("n,l", [(16, 32), (20, 8), (9, 0), (14, 64)])
def test_csr_solve_small(bk, ctx, inner, tol, n, l):
    rp, ci, va, b = W.diffusion_workload(W.BASE_SEED + 70 + n, n=n)
    mu = 1e-4
    A = bk.csr_operator(torch.from_numpy(rp).to(dev()), torch.from_numpy(ci).to(dev()), torch.from_numpy(va).to(dev()))
    x = torch.zeros(b.shape[0], dtype=torch.float64, device=dev())
    info = bk.solve(ctx, A, mu, torch.from_numpy(b).to(dev()), x,
                    bk.default_opts(tol=tol, sketch=l, seed=11, inner=inner,
                                    inner_tol=1e-6 if inner == "fp64" else 1e-5))
    rel = direct.rel_residual(operators.CSR(rp, ci, va), mu, x.cpu().numpy(), b)
    assert rel <= tol, info.as_dict()


def test_exact_recovery(bk, ctx):
    """A = I + U diag(outliers) U^T with 7 <= l outliers: the second step is rank deficient,
    its Galerkin update is already exact (deflation), and the solve stops at 2 loads."""
    d, l, k = 500, 10, 7
    rng = np.random.default_rng(5)
    U = np.linalg.qr(rng.standard_normal((d, k)))[0]
    a = np.eye(d) + (U * np.logspace(2, 5, k)) @ U.T
    b = W.normals(5, 2, d)
    x = np.zeros(d)
    info = bk.solve(ctx, bk.dense_operator(a), 0.0, b, x, bk.default_opts(tol=1e-10, sketch=l, seed=9))
    # two loads reach the kappa(A) = 1e5 rounding floor; one refinement load may follow
    assert info.loads <= 3, info.as_dict()
    # after one load the new residual directions span at most the k outlier directions:
    # the rank test drops the other l + 1 - k columns of the block (reported, Q1 reading)
    assert info.deflations >= l + 1 - k, info.as_dict()
    assert direct.rel_residual(operators.Dense(a), 0.0, x, b) <= 1e-10


def test_profile_counts(bk, ctx):
    rp, ci, va, b = W.diffusion_workload(W.BASE_SEED + 81, n=16)
    A = bk.csr_operator(rp, ci, va)
    x = np.zeros(b.shape[0])
    info = bk.solve(ctx, A, 1e-4, b, x, bk.default_opts(tol=1e-8, sketch=16, seed=5, inner="fp32", inner_tol=1e-5,
                                                        profile=1))
    n = list(info.launches)
    assert n[bk.KERNEL_CLASSES.index("operator")] == info.loads
    assert n[bk.KERNEL_CLASSES.index("reduce")] == 2 * info.loads
    assert all(t > 0 for t in list(info.ms_kernel)[:6])


def test_host_buffers(bk, ctx):
    """Host (NumPy) arrays go through the same C ABI and give the same x."""
    rp, ci, va, b = W.diffusion_workload(W.BASE_SEED + 80, n=10)
    mu = 1e-3
    o = bk.default_opts(tol=1e-10, sketch=12, seed=5)
    xh = np.zeros(b.shape[0])
    bk.solve(ctx, bk.csr_operator(rp, ci, va), mu, b, xh, o)
    A = bk.csr_operator(torch.from_numpy(rp).to(dev()), torch.from_numpy(ci).to(dev()), torch.from_numpy(va).to(dev()))
    xd = torch.zeros(b.shape[0], dtype=torch.float64, device=dev())
    bk.solve(ctx, A, mu, torch.from_numpy(b).to(dev()), xd, o)
    np.testing.assert_array_equal(xh, xd.cpu().numpy())


def test_edge_cases(bk, ctx):
    d = 7
    a = np.diag(np.arange(1.0, d + 1))
    A = bk.dense_operator(a)
    # b = 0 gives x = 0
    x = np.ones(d)
    info = bk.solve(ctx, A, 0.0, np.zeros(d), x, bk.default_opts(sketch=3))
    assert info.status == bk.BK_OK and np.all(x == 0)
    # block wider than d: clamped, still exact
    b = np.arange(1.0, d + 1)
    x = np.zeros(d)
    bk.solve(ctx, A, 0.5, b, x, bk.default_opts(sketch=20, tol=1e-12))
    np.testing.assert_allclose(x, b / (np.arange(1.0, d + 1) + 0.5), rtol=1e-11)
    # d = 1
    x1 = np.zeros(1)
    bk.solve(ctx, bk.dense_operator(np.array([[4.0]])), 1.0, np.array([10.0]), x1, bk.default_opts(sketch=2))
    assert abs(x1[0] - 2.0) < 1e-14
    # invalid arguments
    with pytest.raises(bk.BKError) as e:
        bk.solve(ctx, A, -1.0, b, x)
    assert e.value.status == bk.BK_ERR_ARG
    # blocks wider than the compiled widths (m <= 65) on a system large enough to use them
    big = np.diag(np.arange(1.0, 101.0))
    with pytest.raises(bk.BKError) as e:
        bk.solve(ctx, bk.dense_operator(big), 0.0, np.ones(100), np.zeros(100), bk.default_opts(sketch=65))
    assert e.value.status == bk.BK_ERR_UNSUPPORTED
