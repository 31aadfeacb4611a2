"""Tensor-core (tcgen05, 3xTF32) dense block product against FP64 references."""
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


def apply(bk, ctx, A, P, mu, lda=None):
    d, m = P.shape
    dev = torch.device("cuda:0")
    if lda is not None and lda != d:
        buf = torch.zeros((d, lda), dtype=torch.float32, device=dev)
        buf[:, :d] = torch.from_numpy(A)
        tA = buf[:, :d]
    else:
        tA = torch.from_numpy(A).to(dev)
    ld = (d + 31) // 32 * 32
    tP = torch.from_numpy(bk.to_panels(P, ld)).to(dev)
    tY = torch.zeros_like(tP)
    tG = torch.zeros((m, m), dtype=torch.float64, device=dev)
    bk.block_apply(ctx, bk.dense_operator(tA), mu, tP, tY, tG, m, ld)
    return bk.from_panels(tY.cpu().numpy(), d, m), tG.cpu().numpy()


@pytest.mark.parametrize("d,m", [(96, 5), (300, 17), (1000, 33), (2052, 9), (129, 36), (33, 2)])
def test_tc_product_matches_fp64(bk, ctx, d, m):
    """Y = A P + mu P and G = P^T Y within FP32 accuracy, flat in d (the FP32 sums of
    32-wide K slices keep the tensor core's accumulation error from growing with d)."""
    rng = np.random.default_rng(d + m)
    A = rng.standard_normal((d, d)).astype(np.float32)
    A = 0.5 * (A + A.T)
    P = rng.standard_normal((d, m)).astype(np.float32)
    Y, G = apply(bk, ctx, A, P, 0.25)
    Yr = A.astype(np.float64) @ P.astype(np.float64) + 0.25 * P
    Gr = P.astype(np.float64).T @ Yr
    assert np.abs(Y - Yr).max() <= 3e-6 * np.abs(Yr).max()
    assert np.abs(G - Gr).max() <= 3e-6 * np.abs(Gr).max()


def test_unaligned_rows_fall_back(bk, ctx):
    """A leading dimension that is not a multiple of 4 (rows not 16-byte aligned) cannot be
    read by TMA; the product falls back to the FFMA kernel and is just as accurate."""
    d, m = 301, 17
    rng = np.random.default_rng(3)
    A = rng.standard_normal((d, d)).astype(np.float32)
    P = rng.standard_normal((d, m)).astype(np.float32)
    Y, _ = apply(bk, ctx, A, P, 0.0, lda=303)
    Yr = A.astype(np.float64) @ P.astype(np.float64)
    assert np.abs(Y - Yr).max() <= 3e-6 * np.abs(Yr).max()


def test_tc_dense_solve(bk, ctx):
    """A dense FP32 system of the batched workload solved with FP32 blocks (tensor-core
    products) to 1e-8, checked by the oracle."""
    d = 1024
    A, b = W.batch_system(W.BASE_SEED + 44, 0, d, dtype=np.float32)
    x = np.zeros(d)
    dev = torch.device("cuda:0")
    info = bk.solve(ctx, bk.dense_operator(torch.from_numpy(A).to(dev)), 0.0, b, x,
                    bk.default_opts(tol=1e-8, sketch=16, seed=2, inner="fp32", inner_tol=1e-5))
    assert direct.rel_residual(operators.Dense(A.astype(np.float64)), 0.0, x, b) <= 1e-8, info.as_dict()
