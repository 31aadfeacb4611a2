"""Full-size runs of the block-Lanczos drivers in the configuration bench.py times,
checked by the FP64 oracle on properties that hold at any size (sampled outputs the
oracle can compute one by one)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2501_18717_gb300 import workloads as W  # noqa: E402
from oracle import direct, operators  # noqa: E402


@pytest.fixture(scope="module")
def bk():
    from paper_2501_18717_gb300 import bk as _bk
    return _bk


@pytest.fixture(scope="module")
def ctx(bk):
    c = bk.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("inner", ["bf16", "fp32"])
def test_ridge_path_full_size(bk, ctx, inner):
    """Z 200,000 x 4096 FP32 (sigma_i = 1/i plus N(0, 1e-6) noise), 64 shifts in
    [1e-6, 1], sketch 64, BF16 tensor-core loads (the configuration's precision, as the
    bench leg runs them) or FP32 loads, with FP64-accurate refinement residuals: every
    sampled shift's residual, recomputed by the oracle in FP64 from the stored Z, is at
    most 1e-8."""
    dev = torch.device("cuda:0")
    n, d, L = 200000, 4096, 64
    Z, f, b = W.ridge_workload_torch(W.BASE_SEED + 3, n, d, 1e-3, dev)
    mus = np.logspace(-6, 0, L)
    X = torch.zeros((L, d), dtype=torch.float64, device=dev)
    info = bk.ridge_path(ctx, bk.gram_operator(Z), mus, b, X,
                         bk.default_opts(tol=1e-8, sketch=64, seed=W.BASE_SEED + 3, inner=inner, inner_tol=1e-5,
                                         check_every=2, max_loads=400), check=False)
    assert info.status == bk.BK_OK, info.as_dict()
    op = operators.Gram(Z.cpu().numpy())
    Xh = X.cpu().numpy().T
    bh = b.cpu().numpy()
    del Z
    for j in range(0, L, 9):
        res = direct.rel_residual(op, mus[j], Xh[:, j], bh)
        assert res <= 1e-8, (j, mus[j], res, info.as_dict())


def _rbf_full(dev, d=40000, m=256):
    seed = W.BASE_SEED + 4
    pts = W.rbf_points(seed, d)
    ld = (d + 31) // 32 * 32
    Kbuf = torch.zeros((d, ld), dtype=torch.float32, device=dev)
    Kbuf[:, :d] = W.rbf_kernel_torch(pts, dev)
    B = W.sample_block(seed, d, m)
    return Kbuf[:, :d], B


def test_sample_full_size(bk, ctx):
    """40,000 RBF points, K stored in FP32 (6.4 GB), 256 samples, 32 nodes, FP64
    blocks with compensated FP32-pair products. The oracle checks, from the stored K
    promoted to FP64, the identity S^T S = B^T (K + nugget I) B on 8 sampled columns
    (it holds for the exact square root and for the block-Lanczos approximation
    alike, so it pins scaling, column order and the operator, not convergence), and
    the driver must report convergence of S itself (relative change <= 1e-6).
    Nugget 1e-5: the FP32 rounding of K is a symmetric perturbation of norm about
    3e-6 at this size, so K32 + 1e-6 I is indefinite (next test)."""
    dev = torch.device("cuda:0")
    K, B = _rbf_full(dev)
    d, m = B.shape
    nug = 1e-5
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).to(dev)
    S = torch.zeros((m, d), dtype=torch.float64, device=dev)
    info = bk.sample(ctx, bk.dense_operator(K), nug, Bt.T, S.T, 32,
                     bk.default_opts(tol=1e-6, inner="f32x2", check_every=4, max_loads=24), check=False)
    assert info.status == bk.BK_OK, info.as_dict()
    cols = 8
    Sh = S[:cols].cpu().numpy().T
    Kh = K.cpu().numpy()
    del K
    op = operators.Dense(Kh[:, :d])  # stored FP32 values promoted to FP64
    Bc = B[:, :cols]
    G_ref = Bc.T @ op.apply(Bc, nug)
    G = Sh.T @ Sh
    scale = np.sqrt(np.outer(np.diag(G_ref), np.diag(G_ref)))
    assert np.max(np.abs(G - G_ref) / scale) <= 1e-8


def test_sample_full_size_fp32_floor(bk, ctx):
    """At the configuration's nugget 1e-6 the stored FP32 K + 1e-6 I is indefinite
    (rounding perturbation about 3e-6): the driver must stop with BK_BREAKDOWN rather
    than return a square root that does not exist."""
    dev = torch.device("cuda:0")
    K, B = _rbf_full(dev)
    d, m = B.shape
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).to(dev)
    S = torch.zeros((m, d), dtype=torch.float64, device=dev)
    info = bk.sample(ctx, bk.dense_operator(K), 1e-6, Bt.T, S.T, 32,
                     bk.default_opts(tol=1e-6, inner="f32x2", check_every=4, max_loads=16), check=False)
    assert info.status == bk.BK_BREAKDOWN, info.as_dict()


def test_shrink_full_size(bk, ctx):
    """The 128^3 diffusion system (d = 2,097,152, FP64 CSR values, mu 1e-4) as the
    shrink leg of bench.py runs it: one block step on [b Omega] (33 columns) locks V,
    then one-column deflated CG to 1e-8. The oracle recomputes b - A_mu x in FP64 from
    the stored CSR values; the iterate must also beat the block-CG iterate after the
    single locked step (x_0) by many orders."""
    seed, omega_seed, grid = W.BASE_SEED + 2, W.BASE_SEED + 3, 128  # the bench's seeds
    rp, ci, va, d = W.diffusion_csr(seed, grid)
    b = W.normals(seed, W.STREAM_RHS, d)
    mu = 1e-4
    op = bk.csr_operator(torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(), torch.from_numpy(va).cuda())
    x = torch.zeros(d, dtype=torch.float64, device="cuda")
    info = bk.solve_shrink(ctx, op, mu, torch.from_numpy(b).cuda(), x, 1,
                           bk.default_opts(tol=1e-8, sketch=32, seed=omega_seed, check_every=32, max_loads=20000))
    A = operators.CSR(rp, ci, va)
    res = direct.rel_residual(A, mu, x.cpu().numpy(), b)
    assert res <= 1e-8, (res, info.as_dict())
    assert info.refinements == 33 and info.loads < 4000, info.as_dict()
    x0 = torch.zeros(d, dtype=torch.float64, device="cuda")
    bk.solve_shrink(ctx, op, mu, torch.from_numpy(b).cuda(), x0, 1,
                    bk.default_opts(tol=1e-30, sketch=32, seed=omega_seed, max_loads=2), check=False)
    assert direct.rel_residual(A, mu, x0.cpu().numpy(), b) > 1e3 * res


@pytest.mark.parametrize("inner,tol", [("fp32", 1e-8), ("fp64", 1e-10)])
def test_headline_solve_full_size(bk, ctx, inner, tol):
    """The headline system as bench.py times it: 128^3 diffusion (d = 2,097,152, FP64 CSR
    values), mu 1e-4, Omega of 32 columns, FP32 blocks with FP64 refinement (tol 1e-8)
    or FP64 blocks (tol 1e-10). The oracle recomputes b - A_mu x in FP64 from the stored
    CSR values (a property that holds at any size)."""
    seed, omega_seed, grid = W.BASE_SEED + 2, W.BASE_SEED + 3, 128  # the bench's seeds
    rp, ci, va, d = W.diffusion_csr(seed, grid)
    b = W.normals(seed, W.STREAM_RHS, d)
    mu = 1e-4
    op = bk.csr_operator(torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(), torch.from_numpy(va).cuda())
    x = torch.zeros(d, dtype=torch.float64, device="cuda")
    info = bk.solve(ctx, op, mu, torch.from_numpy(b).cuda(), x,
                    bk.default_opts(tol=tol, sketch=32, seed=omega_seed, inner=inner,
                                    inner_tol=1e-5 if inner == "fp32" else 1e-6, check_every=16))
    res = direct.rel_residual(operators.CSR(rp, ci, va), mu, x.cpu().numpy(), b)
    assert res <= tol, (res, info.as_dict())
    assert info.loads < 2000, info.as_dict()


def test_batched_full_size(bk, ctx):
    """The batched workload at full size: 512 uneven FP32 systems (d log-uniform in
    [500, 16000], 75 GB of matrices) solved together in mixed precision to 1e-8 (block
    width 17 for every system instead of the autotuner's pick). The oracle recomputes
    the FP64 residual from the stored FP32 values of three sampled systems (the
    smallest, a median and the largest)."""
    seed = W.BASE_SEED + 5  # the bench's batch seed
    ds = [int(v) for v in W.batch_sizes(seed, 512)]
    dev = torch.device("cuda:0")
    mats, bs = [], []
    for i, d in enumerate(ds):
        A, b = W.batch_system_torch(seed, i, d, dev)
        mats.append(A)
        bs.append(b)
    xs = [torch.zeros(d, dtype=torch.float64, device=dev) for d in ds]
    infos = bk.solve_batched(ctx, bk.Batch(mats, np.zeros(len(ds)), bs, xs),
                             bk.default_opts(tol=1e-8, sketch=16, seed=W.BASE_SEED + 3, inner="fp32",
                                             inner_tol=1e-5, check_every=16))
    assert all(i.status == bk.BK_OK for i in infos)
    order = np.argsort(ds)
    for i in (int(order[0]), int(order[len(ds) // 2]), int(order[-1])):
        A = mats[i].cpu().numpy().astype(np.float64)
        res = direct.rel_residual(operators.Dense(A), 0.0, xs[i].cpu().numpy(), bs[i].cpu().numpy())
        assert res <= 1e-8, (i, ds[i], res, infos[i].as_dict())
