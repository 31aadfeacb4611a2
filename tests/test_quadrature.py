"""The square-root quadrature of the library (host code, no GPU): nodes against SciPy's
Jacobi elliptic functions and the integral identity of Eq. sqrt_rational."""
import numpy as np
import pytest
import scipy.special as ss


@pytest.fixture(scope="module")
def bk():
    from paper_2501_18717_gb300 import bk as _bk
    return _bk


@pytest.mark.parametrize("lo,hi", [(1.0, 1e2), (1e-6, 4e3), (0.3, 0.3 * 1e10), (2.0, 2.0)])
def test_nodes_match_elliptic_functions(bk, lo, hi):
    n = 24
    z2, w = bk.sqrt_quadrature(lo, hi, n)
    m = 1 - lo / hi
    K = ss.ellipk(m)
    u = (np.arange(n) + 0.5) * K / n
    sn, cn, dn, _ = ss.ellipj(u, m)
    # near u = K, cn is tiny and sc(u) is ill-conditioned (relative condition ~ 1/cn)
    np.testing.assert_allclose(z2, lo * (sn / cn) ** 2, rtol=1e-8)
    np.testing.assert_allclose(w, 2 / np.pi * K / n * np.sqrt(lo) * dn / cn ** 2, rtol=1e-8)


@pytest.mark.parametrize("kappa,n,err", [(1e2, 16, 1e-13), (1e4, 32, 1e-12), (1e8, 32, 1e-11), (1e10, 32, 1e-9)])
def test_sqrt_accuracy_on_interval(bk, kappa, n, err):
    lo = 0.7
    z2, w = bk.sqrt_quadrature(lo, lo * kappa, n)
    lam = lo * np.logspace(0, np.log10(kappa), 3000)
    approx = (w[None, :] * lam[:, None] / (lam[:, None] + z2[None, :])).sum(1)
    assert np.max(np.abs(approx - np.sqrt(lam)) / np.sqrt(lam)) < err


def test_invalid_interval(bk):
    with pytest.raises(bk.BKError):
        bk.sqrt_quadrature(0.0, 1.0, 8)
