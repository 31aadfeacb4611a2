"""Pins of the FP64 oracle against the mathematics the paper fixes.

Each test checks the oracle against something other than itself: brute-force Galerkin
projections (Def. BCG as written), closed forms, library routines, finite termination
(proof of Thm. cost), exact recovery (Thm. nested), Thm. main and Prop. condno_perturb.
"""
import numpy as np
import pytest
import scipy.integrate as si
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import bcg, direct, galerkin, lanczos, nystrom, operators
from paper_2501_18717_gb300 import workloads as W


def spd(d, lam, seed):
    return W.dense_spd(seed, np.asarray(lam, dtype=np.float64))


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ---------------------------------------------------------------- O0
def test_direct_closed_forms():
    lam = np.array([5.0, 2.0, 1.0, 0.5])
    b = np.array([1.0, -2.0, 3.0, 4.0])
    np.testing.assert_allclose(direct.solve(np.diag(lam), 0.25, b), b / (lam + 0.25), rtol=1e-15)
    X = direct.ridge_path(np.diag(lam), [0.0, 1.0, 10.0], b)
    for j, mu in enumerate([0.0, 1.0, 10.0]):
        np.testing.assert_allclose(X[:, j], b / (lam + mu), rtol=1e-14)
    np.testing.assert_allclose(direct.sqrtm_apply(np.diag(lam), b[:, None])[:, 0], np.sqrt(lam) * b, rtol=1e-14)
    a = spd(30, np.linspace(1, 10, 30), 1)
    bb = np.arange(30.0)
    np.testing.assert_allclose(direct.solve(a, 0.1, bb), np.linalg.solve(a + 0.1 * np.eye(30), bb), rtol=1e-12)


def test_ridge_closed_form():
    """Noiseless Z = U diag(sigma) V^T: x_mu = V diag(sigma/(sigma^2+mu)) U^T f (Sec. 1, ridge regression)."""
    rng = np.random.default_rng(0)
    n, d = 50, 12
    U = np.linalg.qr(rng.standard_normal((n, d)))[0]
    V = np.linalg.qr(rng.standard_normal((d, d)))[0]
    sig = 1.0 / np.arange(1, d + 1)
    Z = (U * sig) @ V.T
    f = rng.standard_normal(n)
    mus = [1e-6, 1e-3, 1.0]
    X = direct.ridge_path(Z.T @ Z, mus, Z.T @ f)
    for j, mu in enumerate(mus):
        np.testing.assert_allclose(X[:, j], V @ (sig / (sig ** 2 + mu) * (U.T @ f)), rtol=1e-9)


# ---------------------------------------------------------------- O1 recurrence
def test_bcg_matches_brute_force_galerkin():
    """P1: the recurrence iterate after t loads is the A_mu-norm minimiser over K_t(A,[b Omega])."""
    d, l = 40, 3
    a = spd(d, np.linspace(1.0, 4.0, d), 2)
    b = W.normals(2, 2, d)
    om = W.omega(2, d, l)
    B = np.column_stack([b, om])
    for mu in [0.0, 0.3]:
        for t in range(1, 5):
            x = bcg.block_cg(a, mu, b, om, tol=0.0, max_loads=t)["x"]
            xg = galerkin.bcg_iterate(a, mu, B, t)
            assert rel(x, xg) < 1e-8, (mu, t)


def test_cg_special_case():
    """P6: a one-column block is CG (Def. CG); compare with SciPy's CG iterates."""
    d = 50
    a = spd(d, np.linspace(1.0, 20.0, d), 3)
    b = W.normals(3, 2, d)
    for t in [1, 3, 7]:
        x = bcg.block_cg(a, 0.1, b, None, tol=0.0, max_loads=t)["x"]
        xs, _ = spla.cg(a + 0.1 * np.eye(d), b, x0=np.zeros(d), maxiter=t, rtol=0.0, atol=0.0)
        assert rel(x, xs) < 1e-11, t
        xp = nystrom.pcg(a, 0.1, b, None, t)[-1]
        assert rel(x, xp) < 1e-11, t


def test_finite_termination():
    """P2: K_t(A, B) = R^d once t m >= d, so the iterate is exact at ceil(d/m) loads."""
    d, l = 60, 5
    a = spd(d, np.linspace(1.0, 3.0, d), 4)
    b = W.normals(4, 2, d)
    om = W.omega(4, d, l)
    mu = 0.05
    xs = direct.solve(a, mu, b)
    t = int(np.ceil(d / (l + 1)))
    out = bcg.block_cg(a, mu, b, om, tol=0.0, max_loads=t)
    assert rel(out["x"], xs) < 1e-9
    lz = lanczos.block_lanczos(a, np.column_stack([b, om]), t)
    assert rel(lanczos.shifted_iterates(lz, [mu])[:, 0], xs) < 1e-11
    # one load short is not exact
    short = bcg.block_cg(a, mu, b, om, tol=0.0, max_loads=t - 2)
    assert rel(short["x"], xs) > 1e-6


def test_exact_recovery_outliers():
    """P3: A = c I + U diag(out) U^T with k <= l outliers: range(U) lies in span(Omega, A Omega)
    (Thm. nested), so the iterate is exact after two loads."""
    d, l, k = 200, 10, 7
    rng = np.random.default_rng(5)
    U = np.linalg.qr(rng.standard_normal((d, k)))[0]
    out = np.logspace(2, 5, k)
    a = 1.0 * np.eye(d) + (U * out) @ U.T
    b = W.normals(5, 2, d)
    om = W.omega(5, d, l)
    for mu in [0.0, 1e-2]:
        xs = direct.solve(a, mu, b)
        out = bcg.block_cg(a, mu, b, om, tol=0.0, max_loads=2)
        # the second step's block adds only k new directions: it is rank deficient, and the
        # Galerkin update over its span is already exact
        assert out["loads"] == 2 and out["status"] == "deflated"
        assert rel(out["x"], xs) < 1e-10  # kappa(A) = 1e5 sets the rounding floor
        lz = lanczos.block_lanczos(a, np.column_stack([b, om]), 2)
        assert rel(lanczos.shifted_iterates(lz, [mu])[:, 0], xs) < 1e-10
    # with more outliers than sketch columns two loads do not suffice
    U2 = np.linalg.qr(rng.standard_normal((d, 3 * l)))[0]
    a2 = np.eye(d) + (U2 * np.logspace(2, 5, 3 * l)) @ U2.T
    assert rel(bcg.block_cg(a2, 0.0, b, om, tol=0.0, max_loads=2)["x"], direct.solve(a2, 0.0, b)) > 1e-6


def test_column_scaling_invariance():
    """The column-0 iterate depends on span(K_t) only: scaling b and Omega's columns
    (the solver's start block [b/||b||, Omega/sqrt(d)]) changes it by the factor ||b||."""
    d, l = 80, 4
    a = spd(d, np.linspace(1.0, 50.0, d), 6)
    b = W.normals(6, 2, d)
    om = W.omega(6, d, l)
    B = W.inner_start_block(b, om)
    for t in [1, 3, 5]:
        x1 = bcg.block_cg(a, 0.0, b, om, tol=0.0, max_loads=t)["x"]
        x2 = bcg.block_cg(a, 0.0, B[:, 0], B[:, 1:], tol=0.0, max_loads=t)["x"] * np.linalg.norm(b)
        assert rel(x2, x1) < 1e-10


def test_refined_solve_reaches_tolerance():
    d, l = 300, 8
    a = spd(d, W.decay_spectrum(d, 1e4, 1e-2), 7)
    b = W.normals(7, 2, d)
    om = W.omega(7, d, l)
    out = bcg.refined_solve(a, 1e-3, b, om, tol=1e-11, inner_tol=1e-6)
    assert out["rel_residual"] <= 1e-11
    assert direct.rel_residual(operators.Dense(a), 1e-3, out["x"], b) <= 1e-11
    assert out["loads"] == out["inner_loads"] + out["refinements"]


def test_refined_solve_adaptive_inner_target():
    """With the adaptive inner target the last pass stops once the outer target is met
    (with margin 2), so the solve still reaches tol, needs no more block products than
    with the fixed inner target, and does not overshoot tol by orders of magnitude."""
    d, l = 300, 8
    a = spd(d, W.decay_spectrum(d, 1e4, 1e-2), 7)
    b = W.normals(7, 2, d)
    om = W.omega(7, d, l)
    fixed = bcg.refined_solve(a, 1e-3, b, om, tol=1e-8, inner_tol=1e-6)
    adapt = bcg.refined_solve(a, 1e-3, b, om, tol=1e-8, inner_tol=1e-6, adaptive_inner=True)
    res = direct.rel_residual(operators.Dense(a), 1e-3, adapt["x"], b)
    assert res <= 1e-8
    assert adapt["inner_loads"] <= fixed["inner_loads"]
    # the fixed rule solves the last pass to 1e-6 of an already small residual
    assert fixed["rel_residual"] < 1e-3 * res


# ---------------------------------------------------------------- O2 Lanczos
def test_lanczos_equals_recurrence():
    d, l = 120, 5
    a = spd(d, np.linspace(1.0, 10.0, d), 8)
    b = W.normals(8, 2, d)
    om = W.omega(8, d, l)
    B = np.column_stack([b, om])
    for t in [1, 2, 4, 6]:
        lz = lanczos.block_lanczos(a, B, t)
        x = lanczos.shifted_iterates(lz, [0.2])[:, 0]
        xr = bcg.block_cg(a, 0.2, b, om, tol=0.0, max_loads=t)["x"]
        assert rel(x, xr) < 1e-9, t
        Q = lanczos.basis(lz)
        np.testing.assert_allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-12)
        np.testing.assert_allclose(lanczos.tridiag(lz), Q.T @ a @ Q, atol=1e-10)


def test_shift_invariance():
    """P7: one block-Lanczos basis gives the block-CG iterate for every shift (Eq. shift_invariance)."""
    d, l = 90, 6
    a = spd(d, np.logspace(0, 3, d), 9)
    b = W.normals(9, 2, d)
    om = W.omega(9, d, l)
    mus = np.logspace(-6, 0, 7)
    lz = lanczos.block_lanczos(a, np.column_stack([b, om]), 4)
    X = lanczos.shifted_iterates(lz, mus)
    for j, mu in enumerate(mus):
        xr = bcg.block_cg(a, mu, b, om, tol=0.0, max_loads=4)["x"]
        assert rel(X[:, j], xr) < 1e-8
    lzf = lanczos.block_lanczos(a, np.column_stack([b, om]), int(np.ceil(d / (l + 1))))
    Xf = lanczos.shifted_iterates(lzf, mus)
    np.testing.assert_allclose(Xf, direct.ridge_path(a, mus, b), rtol=1e-8, atol=1e-12)


def test_sqrt_iterate_closed_forms():
    """P9: bsq_t of Def. blansq; exact once K_t = R^d, and equal to the integral of
    A bcg_t(z^2) over z computed by adaptive quadrature for partial t."""
    d, l = 24, 3
    lam = np.logspace(-1, 2, d)
    a = spd(d, lam, 10)
    B = np.column_stack([W.normals(10, 2, d), W.omega(10, d, l)])
    lz = lanczos.block_lanczos(a, B, int(np.ceil(d / (l + 1))))
    np.testing.assert_allclose(lanczos.sqrt_iterate(lz), direct.sqrtm_apply(a, B), rtol=1e-9, atol=1e-10)
    # diagonal A: closed form sqrt(lambda) * b
    np.testing.assert_allclose(lanczos.sqrt_iterate(lanczos.block_lanczos(np.diag(lam), B, 8)),
                               np.sqrt(lam)[:, None] * B, rtol=1e-9, atol=1e-10)
    # partial space: compare with numerical integration of the definition, column 0
    t = 3
    lzp = lanczos.block_lanczos(a, B, t)
    bsq = lanczos.sqrt_iterate(lzp)[:, 0]

    def integrand(z, i):
        return (a @ lanczos.shifted_iterates(lzp, [z * z])[:, 0])[i]
    for i in [0, 5, 17]:
        val, _ = si.quad(integrand, 0, np.inf, args=(i,), epsabs=1e-12, epsrel=1e-11, limit=400)
        assert abs(2 / np.pi * val - bsq[i]) <= 1e-8 * np.linalg.norm(bsq)


def test_isqrt_closed_forms():
    """A^{-1/2}: diagonal closed form; SciPy's matrix square root, inverted; the Lanczos
    iterate is exact once K_t = R^d and equals the integral of bcg_t(z^2) over z for a
    partial basis (adaptive quadrature)."""
    import scipy.linalg as sla
    lam = np.logspace(-1, 2, 24)
    b = W.normals(11, 2, 24)
    np.testing.assert_allclose(direct.isqrtm_apply(np.diag(lam), b[:, None], shift=0.5)[:, 0],
                               b / np.sqrt(lam + 0.5), rtol=1e-14)
    a = spd(24, lam, 12)
    B = np.column_stack([b, W.omega(11, 24, 3)])
    ref = np.linalg.solve(np.real(sla.sqrtm(a + 0.1 * np.eye(24))), B)
    np.testing.assert_allclose(direct.isqrtm_apply(a, B, shift=0.1), ref, rtol=1e-9, atol=1e-12)
    lz = lanczos.block_lanczos(a, B, 6)
    np.testing.assert_allclose(lanczos.isqrt_iterate(lz), direct.isqrtm_apply(a, B), rtol=1e-9, atol=1e-10)
    lzp = lanczos.block_lanczos(a, B, 2)
    v = lanczos.isqrt_iterate(lzp)[:, 0]

    def integrand(z, i):
        return lanczos.shifted_iterates(lzp, [z * z])[i, 0]
    for i in [0, 7, 19]:
        val, _ = si.quad(integrand, 0, np.inf, args=(i,), epsabs=1e-12, epsrel=1e-11, limit=400)
        assert abs(2 / np.pi * val - v[i]) <= 1e-8 * np.linalg.norm(v)


def test_elliptic_identity():
    """Eq. ellipticK_eval: int_0^inf dz / sqrt((l1+z^2)(ld+z^2)) = K(1 - l1/ld)/sqrt(ld)
    (K with parameter m, ld < l1), and it equals pi / (2 AGM(sqrt l1, sqrt ld))."""
    import scipy.special as ss
    for l1, ld in [(10.0, 1.0), (1e4, 2.0), (3.0, 2.5)]:
        val, _ = si.quad(lambda z: 1.0 / np.sqrt((l1 + z * z) * (ld + z * z)), 0, np.inf, epsrel=1e-12)
        np.testing.assert_allclose(val, ss.ellipk(1 - l1 / ld) / np.sqrt(ld), rtol=1e-9)
        x, y = np.sqrt(l1), np.sqrt(ld)
        for _ in range(40):
            x, y = 0.5 * (x + y), np.sqrt(x * y)
        np.testing.assert_allclose(val, np.pi / (2 * x), rtol=1e-9)
        # the bound of Eq. ellipticK_bd with x = kappa
        kappa = l1 / ld
        assert 2 / np.pi * np.sqrt(kappa) * ss.ellipk(1 - kappa) <= 5 / (4 * np.pi) * np.log(16 * kappa)


# ---------------------------------------------------------------- O3 Nystrom / PCG
def _problem(seed=11, d=150):
    lam = np.concatenate([np.logspace(4, 2, 12), np.linspace(1.0, 0.1, d - 12)])
    a = spd(d, lam, seed)
    b = W.normals(seed, 2, d)
    return a, b, lam


def test_nystrom_approximation():
    """Eq. nystromBKI_def: A<K_s> equals (A K)(K^T A K)^+ (K^T A) for the monomial K_s."""
    a, b, lam = _problem()
    om = W.omega(11, a.shape[0], 6)
    for s in [1, 2, 3]:
        U, D = nystrom.nystrom(a, om, s)
        # A<K> depends on range(K) only: orthonormalise the column-normalised monomial
        # basis by Householder QR and apply the definition on it
        K = np.column_stack([np.linalg.matrix_power(a, j) @ om for j in range(s)])
        K = np.linalg.qr(K / np.linalg.norm(K, axis=0))[0]
        AK = a @ K
        ref = AK @ np.linalg.inv(K.T @ AK) @ AK.T
        assert np.linalg.norm((U * D) @ U.T - ref) <= 1e-7 * np.linalg.norm(ref)
        # best rank approximations are never beaten: A - A<K> is PSD
        assert np.linalg.eigvalsh(a - (U * D) @ U.T).min() > -1e-8 * lam[0]


def test_pcg_matches_brute_force():
    """Def. PCG: the PCG iterate minimises the A_mu-norm error over K_t(P^{-1}A_mu, P^{-1}b)."""
    a, b, lam = _problem(12, 80)
    om = W.omega(12, 80, 4)
    U, D = nystrom.nystrom(a, om, 2)
    mu = 0.01
    Pinv = nystrom.preconditioner_inverse(U, D, D.min(), mu)
    am = a + mu * np.eye(80)
    xs = nystrom.pcg(a, mu, b, Pinv, 5)
    for t in range(1, 6):
        V = np.column_stack([np.linalg.matrix_power(Pinv @ am, j) @ (Pinv @ b) for j in range(t)])
        V = np.linalg.qr(V)[0]
        xg = V @ np.linalg.solve(V.T @ am @ V, V.T @ b)
        assert rel(xs[t - 1], xg) < 1e-8, t


def test_prop_condno_perturb():
    """Prop. condno_perturb: kappa(P^{-1/2} A_mu P^{-1/2}) <= (theta+mu+||A - A<K>||)(1/(theta+mu)+1/(lambda_d+mu))."""
    a, b, lam = _problem(13, 120)
    om = W.omega(13, 120, 8)
    for s in [1, 3]:
        U, D = nystrom.nystrom(a, om, s)
        E = np.linalg.norm(a - (U * D) @ U.T, 2)
        for theta in [D.min(), lam[-1], 1.0]:
            for mu in [0.0, 1e-2, 1.0]:
                kap = nystrom.preconditioned_condition_number(a, mu, nystrom.preconditioner_inverse(U, D, theta, mu))
                bound = (theta + mu + E) * (1 / (theta + mu) + 1 / (lam[-1] + mu))
                assert kap <= bound * (1 + 1e-8)


@pytest.mark.parametrize("s", [1, 3])
def test_thm_main(s):
    """Thm. main: with the same Omega, block-CG after t loads is at least as accurate in the
    A_mu-norm as Nystrom PCG of depth s after t - s iterations (theta as in Sec. 7)."""
    a, b, lam = _problem(14, 150)
    d = a.shape[0]
    l = 6
    om = W.omega(14, d, l)
    U, D = nystrom.nystrom(a, om, s)
    for mu in [0.0, 1e-3]:
        Pinv = nystrom.preconditioner_inverse(U, D, D.min(), mu)
        xs = direct.solve(a, mu, b)
        am = a + mu * np.eye(d)
        anorm = lambda v: np.sqrt(v @ am @ v)
        pc = nystrom.pcg(a, mu, b, Pinv, 10)
        for t in range(s + 1, s + 11):
            lz = lanczos.block_lanczos(a, np.column_stack([b, om]), t)
            xb = lanczos.shifted_iterates(lz, [mu])[:, 0]
            eb = anorm(xs - xb)
            ep = anorm(xs - pc[t - s - 1])
            assert eb <= (1 + 1e-8) * ep + 1e-12 * anorm(xs), (mu, t)


# ---------------------------------------------------------------- O5 (f4)
from oracle import deflated  # noqa: E402


def _defl_problem(seed, d, k):
    lam = np.concatenate([np.geomspace(1e3, 20.0, 8), np.linspace(2.0, 0.1, d - 8)])
    a = spd(d, lam, seed)
    b = W.normals(seed, 2, d)
    Wb = np.linalg.qr(W.omega(seed, d, k))[0] if k else np.zeros((d, 0))
    return a, b, Wb


@pytest.mark.parametrize("k", [0, 4, 9])
def test_deflated_cg_brute_force_galerkin(k):
    """Def-CG: x_j minimises the A_mu-norm error over span(W) + K_j(P A_mu, r_0),
    P = I - A_mu W (W^T A_mu W)^{-1} W^T, r_0 = b - A_mu x_0."""
    d, mu = 70, 0.02
    a, b, Wb = _defl_problem(21, d, k)
    am = a + mu * np.eye(d)
    xs = deflated.deflated_cg(a, mu, b, Wb, 6)
    if k:
        P = np.eye(d) - am @ Wb @ np.linalg.solve(Wb.T @ am @ Wb, Wb.T)
        x0 = Wb @ np.linalg.solve(Wb.T @ am @ Wb, Wb.T @ b)
    else:
        P, x0 = np.eye(d), np.zeros(d)
    r0 = b - am @ x0
    for j in range(0, 7):
        K = [np.linalg.matrix_power(P @ am, i) @ r0 for i in range(j)]
        S = np.column_stack([Wb] + K) if (k or j) else np.zeros((d, 0))
        if S.shape[1] == 0:
            assert np.linalg.norm(xs[0]) == 0.0
            continue
        S = np.linalg.qr(S / np.linalg.norm(S, axis=0))[0]
        xg = S @ np.linalg.solve(S.T @ am @ S, S.T @ b)
        assert rel(xs[j], xg) < 1e-9, (k, j)


def test_deflated_cg_invariant_subspace_is_cg():
    """W spanning eigenvectors of A leaves the projection inert (A_mu W = W Lambda_mu and
    r_j orthogonal to W give mu_j = 0), so Def-CG runs SciPy's CG. Diagonal A with b zero
    on W's coordinates keeps that exact in rounding too (a rotated basis would leave
    rounding-level components along W that CG amplifies by the eigenvalue ratio)."""
    d, k, mu = 60, 5, 0.1
    lam = np.concatenate([np.geomspace(400.0, 50.0, k), np.linspace(10.0, 0.2, d - k)])
    a = np.diag(lam)
    b = W.normals(22, 2, d)
    b[:k] = 0.0
    Wb = np.eye(d)[:, :k]
    xs = deflated.deflated_cg(a, mu, b, Wb, 9)
    assert np.linalg.norm(xs[0]) == 0.0
    for t in [1, 3, 9]:
        ref, _ = spla.cg(a + mu * np.eye(d), b, x0=np.zeros(d), maxiter=t, rtol=0.0, atol=0.0)
        assert rel(xs[t], ref) < 1e-12, t
        ref0 = nystrom.pcg(a, mu, b, None, t)[-1]  # and the textbook CG of the comparator
        assert rel(xs[t], ref0) < 1e-12, t


def test_deflated_cg_finite_termination():
    """The iterate space reaches R^d after d - dim(W) iterations: exact there, not two
    iterations earlier (W random, so not an invariant subspace)."""
    d, k, mu = 40, 32, 0.05
    a = spd(d, np.geomspace(1e3, 1.0, d), 23)
    b = W.normals(23, 2, d)
    Wb = np.linalg.qr(W.omega(23, d, k))[0]
    xs = deflated.deflated_cg(a, mu, b, Wb, d - k)
    xstar = direct.solve(a, mu, b)
    assert rel(xs[d - k], xstar) < 1e-9
    assert rel(xs[d - k - 2], xstar) > 1e-6


@pytest.mark.parametrize("s", [1, 2, 3])
def test_shrink_start_and_inclusion(s):
    """j = 0 is the block-CG iterate after s loads on [b Omega] (Def. BCG, brute force);
    span(W) + K_j(P A_mu, r_0) lies in K_{s+j}(A, [b Omega]) (r_0 is in K_{s+1} and P A_mu
    maps K_{s+i} into K_{s+i+1}), so block-CG after s + j loads is at least as accurate in
    the A_mu-norm."""
    d, l, mu = 90, 5, 1e-3
    a, b, _ = _defl_problem(24, d, 0)
    om = W.omega(24, d, l)
    B = np.column_stack([b, om])
    xs = deflated.shrink_solve(a, mu, b, om, s, 8)
    assert rel(xs[0], galerkin.bcg_iterate(a, mu, B, s)) < 1e-9
    xstar = direct.solve(a, mu, b)
    am = a + mu * np.eye(d)
    anorm = lambda v: np.sqrt(v @ am @ v)
    for j in range(1, 9):
        xb = lanczos.shifted_iterates(lanczos.block_lanczos(a, B, s + j), [mu])[:, 0]
        assert anorm(xstar - xb) <= (1 + 1e-7) * anorm(xstar - xs[j]) + 1e-12 * anorm(xstar), (s, j)


@pytest.mark.parametrize("s", [1, 3, 5])
def test_shrink_one_column_block_is_cg(s):
    """Sec. CG_pro: with a one-column block (no Omega) the locked space is K_s(A, b),
    and span(W) + K_j(P A_mu, r_0) = K_{s+j}(A, b), so the shrunk iterate after j
    deflated steps is CG's iterate after s + j steps (SciPy's CG)."""
    d, mu = 60, 0.05
    a = spd(d, np.linspace(1.0, 8.0, d), 25)
    b = W.normals(25, 2, d)
    xs = deflated.shrink_solve(a, mu, b, np.zeros((d, 0)), s, 6)
    for j in [0, 2, 6]:
        ref, _ = spla.cg(a + mu * np.eye(d), b, x0=np.zeros(d), maxiter=s + j, rtol=0.0, atol=0.0)
        assert rel(xs[j], ref) < 1e-10, (s, j)


# ---- accurate dense products (oracle/accurate.py) against exact rational arithmetic
def _exact_rowsum(a_row, x):
    from fractions import Fraction
    return float(sum(Fraction(float(a)) * Fraction(float(v)) for a, v in zip(a_row, x)))


def test_accurate_split_is_exact_and_short():
    from oracle import accurate
    rng = np.random.default_rng(3)
    x = rng.standard_normal(1000) * np.exp2(rng.integers(-300, 300, 1000))
    h, t = accurate.split_head_tail(x)
    assert np.array_equal(h + t, x)
    # the head has at most 26 significant bits: scaled to [2^25, 2^26) it is an integer
    m, _ = np.frexp(h)
    assert np.all(m * 2.0 ** 26 == np.round(m * 2.0 ** 26))


@pytest.mark.parametrize("case", ["gaussian", "cancelling", "wide_range"])
def test_accurate_matvec_against_fractions(case):
    """Rows of 300 FP32 values times FP64 x: within 2e-15 sum |a x| of the exact
    rational sum; the cancelling case (sum near 0 with large terms) and exponents
    spread over 2^-60 .. 2^60 are where an ordinary dot product loses digits."""
    from oracle import accurate
    rng = np.random.default_rng({"gaussian": 1, "cancelling": 2, "wide_range": 3}[case])
    d = 300
    a = rng.standard_normal((6, d)).astype(np.float32)
    x = rng.standard_normal(d)
    if case == "cancelling":
        # x orthogonal to each row up to rounding, in FP64
        for i in range(6):
            a64 = a[i].astype(np.float64)
            x = x - (a64 @ x) / (a64 @ a64) * a64
    if case == "wide_range":
        x = x * np.exp2(rng.integers(-60, 60, d))
        a = (a * np.exp2(rng.integers(-30, 30, (6, d)))).astype(np.float32)
    A = np.zeros((d, d), dtype=np.float32)
    A[:6] = a
    y = accurate.matvec(A, x)[:6]
    scale = accurate.abs_products(A, x[:, None])[:6, 0]
    for i in range(6):
        exact = _exact_rowsum(a[i], x)
        assert abs(y[i] - exact) <= 2e-15 * scale[i], (i, y[i], exact)
