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
