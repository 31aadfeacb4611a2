"""Seeded input generators: Philox known answers, normal streams, test matrices."""
import os

import numpy as np
import scipy.sparse as sp

from paper_2501_18717_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = W.philox4x32_10(v[0], v[1], v[2], v[3], v[4], v[5])
        assert [int(o) for o in out] == v[6:10]


def test_normal_stream_properties():
    z = W.normals(7, W.STREAM_OMEGA, 400000)
    assert abs(z.mean()) < 5e-3 and abs(z.std() - 1) < 5e-3
    # offsets address the same stream
    np.testing.assert_array_equal(W.normals(7, 3, 100, offset=37), z[37:137])
    # streams and keys are independent draws
    assert not np.allclose(W.normals(7, 2, 100), z[:100])
    assert not np.allclose(W.normals(8, 3, 100), z[:100])
    # Omega is column-major over the stream
    om = W.omega(7, 50, 3)
    np.testing.assert_array_equal(om[:, 1], z[50:100])


def test_dense_spd_spectrum():
    lam = W.decay_spectrum(60, 1e2, 1e-1)
    a = W.dense_spd(3, lam)
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(a))[::-1], lam, rtol=1e-12, atol=1e-12)
    assert np.array_equal(a, a.T)


def test_diffusion_operator():
    n = 6
    rp, ci, va, d = W.diffusion_csr(5, n)
    assert d == n ** 3
    assert rp[-1] == 6 * n ** 2 * (n - 1) + n ** 3  # off-diagonals of interior faces + diagonal
    A = sp.csr_matrix((va, ci, rp), shape=(d, d))
    assert abs(A - A.T).max() == 0
    # columns sorted within rows
    for i in range(d):
        assert np.all(np.diff(ci[rp[i]:rp[i + 1]]) > 0)
    # boundary faces make the matrix strictly diagonally dominant on the boundary rows
    dense = A.toarray()
    off = np.abs(dense).sum(1) - 2 * np.abs(np.diag(dense))
    assert np.all(off <= 1e-12)
    assert np.linalg.eigvalsh(dense).min() > 0
    # the 128^3 workload has the stated nonzero count
    assert 6 * 128 ** 2 * 127 + 128 ** 3 == 14_581_760
