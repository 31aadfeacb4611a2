"""bk_solve_batched and bk_autotune against the FP64 oracle on small uneven batches
(systems shaped like the batched workload: outlier spectra rotated by Householder
reflectors, FP32 stored values, mu = 0)."""
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


def make_batch(seed, n, dmin, dmax, dtype=np.float32):
    ds = [int(d) for d in W.batch_sizes(seed, n, dmin, dmax)]
    mats, bs = [], []
    for i, d in enumerate(ds):
        A, b = W.batch_system(seed, i, d, dtype=dtype)
        mats.append(A)
        bs.append(b)
    return ds, mats, bs


def rel_res(A, x, b, mu=0.0):
    return direct.rel_residual(operators.Dense(A.astype(np.float64)), mu, x, b)


@pytest.mark.parametrize("inner,tol", [("fp32", 1e-8), ("fp64", 1e-10)])
def test_batched_matches_oracle(bk, ctx, inner, tol):
    seed = W.BASE_SEED + 40
    ds, mats, bs = make_batch(seed, 10, 300, 1200)
    dev = torch.device("cuda:0")
    tm = [torch.from_numpy(a).to(dev) for a in mats]
    tb = [torch.from_numpy(b).to(dev) for b in bs]
    tx = [torch.zeros(d, dtype=torch.float64, device=dev) for d in ds]
    infos = bk.solve_batched(ctx, bk.Batch(tm, np.zeros(len(ds)), tb, tx),
                             bk.default_opts(tol=tol, sketch=16, seed=3, inner=inner,
                                             inner_tol=1e-5 if inner == "fp32" else 1e-6))
    for i, d in enumerate(ds):
        x = tx[i].cpu().numpy()
        assert rel_res(mats[i], x, bs[i]) <= tol, (i, d, infos[i].as_dict())
        # forward error against the direct solve, bounded by kappa * residual (kappa <= 1e5)
        xstar = direct.solve(mats[i].astype(np.float64), 0.0, bs[i])
        assert np.linalg.norm(x - xstar) / np.linalg.norm(xstar) <= 1e5 * tol
        assert infos[i].status == bk.BK_OK


@pytest.mark.parametrize("loads,l", [(1, 8), (2, 8), (3, 8), (1, 64), (3, 64)])
def test_batched_iterates_match_oracle(bk, ctx, loads, l):
    """With one refinement pass and a load cap, each system's x is the column-0 block-CG
    iterate on [b/||b||, Omega_i/sqrt(d)] (Omega_i from the key seed + i) times ||b||;
    l = 64 is the widest block (m = 65, padded to 68)."""
    seed, oseed = W.BASE_SEED + 43, 17
    ds, mats, bs = make_batch(seed, 6, 200, 900, dtype=np.float64)
    xs = [np.zeros(d) for d in ds]
    bk.solve_batched(ctx, bk.Batch(mats, np.zeros(len(ds)), bs, xs),
                     bk.default_opts(tol=1e-15, sketch=l, seed=oseed, inner="fp64", inner_tol=1e-15,
                                     max_loads=loads, max_refine=1), check=False)
    for i, d in enumerate(ds):
        bn = np.linalg.norm(bs[i])
        om = W.omega(oseed + i, d, l) / np.sqrt(d)
        ref = bcg.block_cg(mats[i], 0.0, bs[i] / bn, om, tol=1e-15, max_loads=loads, history=True)
        xr = ref["history"][loads - 1] * bn
        # the recurrence's amplification of rounding, measured on the oracle itself
        # (start block perturbed by 1e-14 relative); wide blocks on small systems
        # (65 columns, d >= 200) amplify it most
        pert = 1 + 1e-14 * np.random.default_rng(i).standard_normal(om.shape)
        refp = bcg.block_cg(mats[i], 0.0, bs[i] / bn, om * pert, tol=1e-15, max_loads=loads, history=True)
        sens = np.linalg.norm(refp["history"][loads - 1] * bn - xr) / np.linalg.norm(xr)
        err = np.linalg.norm(xs[i] - xr) / np.linalg.norm(xr)
        assert err < max(1e-10, 100 * sens), (i, d, err, sens)


def test_batched_width65_matches_oracle(bk, ctx, tmp_path):
    """Block width 65 (sketch 64) in mixed precision: FP32 blocks, FP64 refinement to
    1e-8 on uneven FP32 systems, residuals recomputed by the oracle in FP64; then the
    same systems with the width chosen per size bucket from a loaded table, so that a
    width-65 group runs in one batch next to a group of width 9."""
    seed = W.BASE_SEED + 44
    ds, mats, bs = make_batch(seed, 8, 300, 2500)
    dev = torch.device("cuda:0")
    tm = [torch.from_numpy(a).to(dev) for a in mats]
    tb = [torch.from_numpy(b).to(dev) for b in bs]
    tx = [torch.zeros(d, dtype=torch.float64, device=dev) for d in ds]
    infos = bk.solve_batched(ctx, bk.Batch(tm, np.zeros(len(ds)), tb, tx),
                             bk.default_opts(tol=1e-8, sketch=64, seed=5, inner="fp32", inner_tol=1e-5))
    for i, d in enumerate(ds):
        assert infos[i].status == bk.BK_OK, infos[i].as_dict()
        assert rel_res(mats[i], tx[i].cpu().numpy(), bs[i]) <= 1e-8, (i, d, infos[i].as_dict())
    # buckets floor(log2 d): 8 and 10 -> sketch 64, 9 -> sketch 8
    (tmp_path / "mixed.txt").write_text("8 64 0\n9 8 0\n10 64 0\n")
    assert {int(np.log2(d)) for d in ds} & {8, 10} and {int(np.log2(d)) for d in ds} - {8, 10}
    with bk.Context(0) as c2:
        bk.autotune_load(c2, tmp_path / "mixed.txt")
        tx2 = [torch.zeros(d, dtype=torch.float64, device=dev) for d in ds]
        infos2 = bk.solve_batched(c2, bk.Batch(tm, np.zeros(len(ds)), tb, tx2),
                                  bk.default_opts(tol=1e-8, sketch=-1, seed=5, inner="fp32", inner_tol=1e-5))
    for i, d in enumerate(ds):
        assert infos2[i].status == bk.BK_OK, infos2[i].as_dict()
        assert rel_res(mats[i], tx2[i].cpu().numpy(), bs[i]) <= 1e-8, (i, d, infos2[i].as_dict())


def test_fp32_width65_falls_back_to_fp64_blocks(bk, ctx):
    """A system of 329 unknowns (kappa about 8e4) with 65-column FP32 blocks: five loads
    exhaust the space and the FP32 recurrence loses orthogonality (its residual estimate
    diverges or turns NaN; measured on this system for widths 49 to 65, in both the
    single-system and the batched kernels). The solve must not return that: the pass is
    rejected, the system is solved in FP64 blocks, and it converges to 1e-8 with the
    fallback reported. The other systems of the batch converge in FP32 blocks."""
    seed = W.BASE_SEED + 44
    ds, mats, bs = make_batch(seed, 8, 300, 2500)
    assert ds[6] == 329
    opts = bk.default_opts(tol=1e-8, sketch=64, seed=5, inner="fp32", inner_tol=1e-5)
    # single-system solve
    x = np.zeros(329)
    info = bk.solve(ctx, bk.dense_operator(mats[6]), 0.0, bs[6], x, opts)
    assert info.status == bk.BK_OK and info.fp64_fallback == 1, info.as_dict()
    assert rel_res(mats[6], x, bs[6]) <= 1e-8
    # batched: only that system falls back
    xs = [np.zeros(d) for d in ds]
    infos = bk.solve_batched(ctx, bk.Batch(mats, np.zeros(len(ds)), bs, xs), opts)
    for i, d in enumerate(ds):
        assert infos[i].status == bk.BK_OK, (i, infos[i].as_dict())
        assert rel_res(mats[i], xs[i], bs[i]) <= 1e-8, (i, d, infos[i].as_dict())
    assert [i for i in range(len(ds)) if infos[i].fp64_fallback] == [6]
    # the failed FP32 attempt stopped within a few hundred loads (no run to the load cap)
    assert infos[6].loads < 1000, infos[6].as_dict()


@pytest.mark.parametrize("inner,tol", [("fp32", 1e-8), ("fp64", 1e-10)])
def test_batched_product_tile_shapes(bk, ctx, tmp_path, inner, tol):
    """The three block-product choices of the autotune table (tensor cores, CUDA cores
    with 16-row and with 32-row tiles) loaded for one bucket each: every system meets
    tol in the oracle's FP64 residual, and the two CUDA-core tile shapes give the same
    solutions to the forward error that residual allows (kappa <= 1e5: 2 kappa tol)."""
    seed = W.BASE_SEED + 45
    ds, mats, bs = make_batch(seed, 6, 300, 1200)
    xs = {}
    for kern in (0, 1, 2):
        (tmp_path / "t.txt").write_text("".join(f"{b} 16 {kern}\n" for b in range(8, 12)))
        with bk.Context(0) as c2:
            bk.autotune_load(c2, tmp_path / "t.txt")
            x = [np.zeros(d) for d in ds]
            infos = bk.solve_batched(c2, bk.Batch(mats, np.zeros(len(ds)), bs, x),
                                     bk.default_opts(tol=tol, sketch=-1, seed=3, inner=inner,
                                                     inner_tol=1e-5 if inner == "fp32" else 1e-6))
        for i in range(len(ds)):
            assert infos[i].status == bk.BK_OK, (kern, i, infos[i].as_dict())
            assert rel_res(mats[i], x[i], bs[i]) <= tol, (kern, i)
        xs[kern] = x
    for i in range(len(ds)):
        assert np.linalg.norm(xs[0][i] - xs[2][i]) <= 2e5 * tol * np.linalg.norm(xs[0][i]), i


def test_batched_host_and_device_agree(bk, ctx):
    seed = W.BASE_SEED + 41
    ds, mats, bs = make_batch(seed, 4, 300, 600)
    o = bk.default_opts(tol=1e-8, sketch=8, seed=11, inner="fp32", inner_tol=1e-5)
    xh = [np.zeros(d) for d in ds]
    bk.solve_batched(ctx, bk.Batch(mats, np.zeros(4), bs, xh), o)
    dev = torch.device("cuda:0")
    xd = [torch.zeros(d, dtype=torch.float64, device=dev) for d in ds]
    bk.solve_batched(ctx, bk.Batch([torch.from_numpy(a).to(dev) for a in mats], np.zeros(4),
                                   [torch.from_numpy(b).to(dev) for b in bs], xd), o)
    for i in range(4):
        np.testing.assert_array_equal(xh[i], xd[i].cpu().numpy())


def test_batched_ragged_and_tiny(bk, ctx):
    """Sizes below the block width (m = d: one load is exact), a ragged tail of a
    128-row tile, and a shift mu > 0, in one batch of mixed widths."""
    rng = np.random.default_rng(7)
    ds = [3, 17, 129, 257]
    mats, bs, mus = [], [], [0.5, 1e-3, 0.0, 2.0]
    for d in ds:
        q = np.linalg.qr(rng.standard_normal((d, d)))[0]
        mats.append(np.ascontiguousarray((q * np.linspace(1, 50, d)) @ q.T))
        bs.append(rng.standard_normal(d))
    xs = [np.zeros(d) for d in ds]
    infos = bk.solve_batched(ctx, bk.Batch(mats, mus, bs, xs),
                             bk.default_opts(tol=1e-11, sketch=20, seed=1, inner="fp64"))
    for i, d in enumerate(ds):
        assert direct.rel_residual(operators.Dense(mats[i]), mus[i], xs[i], bs[i]) <= 1e-11
        if d <= 21:
            assert infos[i].loads <= 2, infos[i].as_dict()


def test_batched_rejects_bad_input(bk, ctx):
    a = np.eye(4, dtype=np.float64)
    b = np.ones(4)
    x = np.zeros(4)
    with pytest.raises(bk.BKError):  # FP32 blocks need FP32 values
        bk.solve_batched(ctx, bk.Batch([a], [0.0], [b], [x]), bk.default_opts(inner="fp32"))
    with pytest.raises(bk.BKError):  # negative shift
        bk.solve_batched(ctx, bk.Batch([a], [-1.0], [b], [x]), bk.default_opts())


def test_autotune_table(bk, ctx, tmp_path):
    """The configuration's candidates {8, 16, 32, 64} (block widths up to 65), and one
    the kernels are not built for (sketch 80, block width 81) that is skipped; each
    bucket also gets its product kernel; the table survives a save/load round trip
    into a fresh context."""
    seed = W.BASE_SEED + 42
    ds, mats, bs = make_batch(seed, 4, 300, 1200)
    xs = [np.zeros(d) for d in ds]
    cal = bk.Batch(mats, np.zeros(len(ds)), bs, xs)
    chosen = bk.autotune(ctx, cal, [8, 16, 32, 64, 80], bk.default_opts(tol=1e-8, inner="fp32", inner_tol=1e-5))
    assert set(chosen.tolist()) <= {8, 16, 32, 64}
    table = bk.autotune_table(ctx, tmp_path / "tune.txt")
    assert table and all(sk in (8, 16, 32, 64) and kern in ("tensor", "cuda", "cuda32") for sk, kern in table.values())
    # a fresh batch solved with sketch = -1 uses the table and converges
    ds2, mats2, bs2 = make_batch(seed + 100, 4, 300, 1200)
    xs2 = [np.zeros(d) for d in ds2]
    opts = bk.default_opts(tol=1e-8, sketch=-1, inner="fp32", inner_tol=1e-5)
    bk.solve_batched(ctx, bk.Batch(mats2, np.zeros(4), bs2, xs2), opts)
    for i in range(4):
        assert rel_res(mats2[i], xs2[i], bs2[i]) <= 1e-8
    # the saved table in a new context gives the same picks and solutions
    with bk.Context(0) as c2:
        bk.autotune_load(c2, tmp_path / "tune.txt")
        assert bk.autotune_table(c2, tmp_path / "tune2.txt") == table
        xs3 = [np.zeros(d) for d in ds2]
        bk.solve_batched(c2, bk.Batch(mats2, np.zeros(4), bs2, xs3), opts)
        for i in range(4):
            np.testing.assert_array_equal(xs3[i], xs2[i])
    # a malformed file is refused and leaves the table as it was
    (tmp_path / "bad.txt").write_text("9 sixteen 1\n")
    with pytest.raises(bk.BKError):
        bk.autotune_load(ctx, tmp_path / "bad.txt")
    assert bk.autotune_table(ctx, tmp_path / "tune3.txt") == table
