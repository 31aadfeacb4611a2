"""bk_nystrom_pcg (the comparator of Thm. main: Nystrom-preconditioned CG, Def. PCG,
Eq. precond_def, Eq. nystromBKI_def) against the FP64 oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2501_18717_gb300 import workloads as W  # noqa: E402
from oracle import direct, nystrom, operators  # noqa: E402


@pytest.fixture(scope="module")
def bk():
    from paper_2501_18717_gb300 import bk as _bk
    return _bk


@pytest.fixture(scope="module")
def ctx(bk):
    c = bk.Context(0)
    yield c
    c.close()


def _problem(d=300, seed=W.BASE_SEED + 40):
    lam = np.concatenate([1e3 * np.arange(1, 31, dtype=float) ** -2.0, np.linspace(0.5, 0.05, d - 30)])
    a = W.dense_spd(seed, lam)
    b = W.normals(seed, W.STREAM_RHS, d)
    return a, b


@pytest.mark.parametrize("s_ny", [1, 3])
def test_pcg_iterates_match_oracle(bk, ctx, s_ny):
    """After t iterations (loads = s_ny + t) the GPU iterate equals the oracle's PCG
    iterate with the oracle's Nystrom preconditioner built from the same Omega
    (theta = smallest eigenvalue of the approximation, Sec. 7)."""
    a, b = _problem()
    d, l, mu, seed = a.shape[0], 10, 1e-3, 41
    om = W.omega(seed, d, l)
    U, D = nystrom.nystrom(a, om, s_ny)
    Pinv = nystrom.preconditioner_inverse(U, D, D.min(), mu)
    ref = nystrom.pcg(a, mu, b, Pinv, 8)
    for t in [1, 3, 8]:
        x = np.zeros(d)
        info = bk.nystrom_pcg(ctx, bk.dense_operator(a), mu, b, x, s_ny,
                              bk.default_opts(tol=1e-30, sketch=l, seed=seed, max_loads=s_ny + t, check_every=1),
                              check=False)
        assert info.loads == s_ny + t and info.refinements == U.shape[1], info.as_dict()
        err = np.linalg.norm(x - ref[t - 1]) / np.linalg.norm(ref[t - 1])
        assert err <= 1e-9, (t, err)


def test_pcg_converges_csr(bk, ctx):
    """CSR diffusion 12^3 (FP64 values): PCG reaches 1e-10 in the oracle's recomputed
    FP64 residual, and needs fewer iterations than plain CG would (Prop.
    condno_perturb: the preconditioner removes the top of the spectrum)."""
    rp, ci, va, d = W.diffusion_csr(W.BASE_SEED + 42, 12)
    b = W.normals(W.BASE_SEED + 42, W.STREAM_RHS, d)
    mu = 1e-4
    op = bk.csr_operator(torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(), torch.from_numpy(va).cuda())
    x = np.zeros(d)
    info = bk.nystrom_pcg(ctx, op, mu, b, x, 2, bk.default_opts(tol=1e-10, sketch=16, seed=43, max_loads=5000,
                                                               check_every=4))
    res = direct.rel_residual(operators.CSR(rp, ci, va), mu, x, b)
    assert res <= 1e-10, (res, info.as_dict())
    # plain CG on the same system (the oracle's textbook CG) needs more iterations
    xs = nystrom.pcg(operators.CSR(rp, ci, va), mu, b, None, info.loads)
    assert direct.rel_residual(operators.CSR(rp, ci, va), mu, xs[info.loads - 2 - 1], b) > res


def test_pcg_gram_fp32(bk, ctx):
    """A = Z^T Z matrix-free with FP32 Z (compensated products): 1e-10 in the oracle's
    residual from the stored Z promoted to FP64."""
    Z, f, b = W.ridge_workload(W.BASE_SEED + 44, 2000, 128, noise_std=1e-3)
    mu = 1e-4
    x = np.zeros(128)
    info = bk.nystrom_pcg(ctx, bk.gram_operator(torch.from_numpy(Z).cuda()), mu, b, x, 1,
                          bk.default_opts(tol=1e-10, sketch=8, seed=45, max_loads=2000, check_every=2))
    res = direct.rel_residual(operators.Gram(Z.astype(np.float64)), mu, x, b)
    assert res <= 1e-10, (res, info.as_dict())


def test_pcg_edge_cases(bk, ctx):
    a, b = _problem(d=40)
    x = np.ones(40)
    info = bk.nystrom_pcg(ctx, bk.dense_operator(a), 0.1, np.zeros(40), x, 1, bk.default_opts(sketch=4))
    assert info.status == bk.BK_OK and np.all(x == 0.0)
    # a sketch wider than d: the approximation is A itself, PCG converges at once
    x = np.zeros(40)
    info = bk.nystrom_pcg(ctx, bk.dense_operator(a), 0.1, b, x, 1,
                          bk.default_opts(tol=1e-12, sketch=64, check_every=1, max_loads=50))
    assert direct.rel_residual(operators.Dense(a), 0.1, x, b) <= 1e-12 and info.loads <= 4, info.as_dict()
    with pytest.raises(bk.BKError):
        bk.nystrom_pcg(ctx, bk.dense_operator(a), 0.1, b, x, 0, bk.default_opts(sketch=4))
