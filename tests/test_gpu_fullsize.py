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


def test_ridge_path_full_size(bk, ctx):
    """Z 200,000 x 4096 FP32 (sigma_i = 1/i plus N(0, 1e-6) noise), 64 shifts in
    [1e-6, 1], sketch 64, FP32 inner products with FP64-accurate refinement residuals:
    every sampled shift's residual, recomputed by the oracle in FP64 from the stored Z,
    is at most 1e-8."""
    dev = torch.device("cuda:0")
    n, d, L = 200000, 4096, 64
    Z, f, b = W.ridge_workload_torch(W.BASE_SEED + 3, n, d, 1e-3, dev)
    mus = np.logspace(-6, 0, L)
    X = torch.zeros((L, d), dtype=torch.float64, device=dev)
    info = bk.ridge_path(ctx, bk.gram_operator(Z), mus, b, X,
                         bk.default_opts(tol=1e-8, sketch=64, seed=W.BASE_SEED + 3, inner="fp32", inner_tol=1e-5,
                                         check_every=2, max_loads=400), check=False)
    assert info.status == bk.BK_OK, info.as_dict()
    op = operators.Gram(Z.cpu().numpy())
    Xh = X.cpu().numpy().T
    bh = b.cpu().numpy()
    del Z
    for j in range(0, L, 9):
        res = direct.rel_residual(op, mus[j], Xh[:, j], bh)
        assert res <= 1e-8, (j, mus[j], res, info.as_dict())
