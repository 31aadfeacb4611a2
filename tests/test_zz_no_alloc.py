"""bk_block_apply_static, the allocation-free block product, against bk_block_apply
and against the oracle's operator.

Callers that cannot let a library allocate device memory (frameworks that own every
device allocation through their own pool, latency-sensitive callers that cannot take
the device synchronisation of cudaMalloc/cudaFree) use the static entry point; it must
give the block product and Gram matrix of the regular entry point, and both must match
the FP64 product of the stored values. This file is collected last on purpose, so that
a failure here stops a -x run only after every other test ran.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2501_18717_gb300 import workloads as W  # noqa: E402


def _case(kind, dtype, m, seed):
    npdt = np.float64 if dtype == "f64" else np.float32
    if kind == "csr":
        rp, ci, va, d = W.diffusion_csr(W.BASE_SEED + 90 + seed, 13)
        ops = (rp, ci, va.astype(npdt))
    else:
        # FP32 rows of 520 floats are 16-byte aligned, so the regular call takes the
        # tensor-core product there; FP64 at 517 rows covers a ragged tile
        d = 520 if dtype == "f32" else 517
        ops = (W.dense_spd(W.BASE_SEED + 90 + seed, W.decay_spectrum(d, 1e2, 1e-1)).astype(npdt),)
    ld = d + 7
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((d, m)).astype(npdt)
    from paper_2501_18717_gb300 import bk
    return ops, bk.to_panels(P, ld), d, ld


def _oracle(kind, ops, P, d, m, mu):
    """Y = A P + mu P and G = P^T Y in FP64 from the stored values (oracle operator)."""
    from oracle import operators
    from paper_2501_18717_gb300 import bk
    op = operators.CSR(*ops) if kind == "csr" else operators.Dense(ops[0])
    Pd = bk.from_panels(P, d, m).astype(np.float64)
    Y = op.apply(Pd, mu)
    return Y, Pd.T @ Y


@pytest.mark.parametrize("kind,dtype,m", [("csr", "f32", 33), ("dense", "f64", 21), ("dense", "f32", 33)])
def test_static_matches_regular(kind, dtype, m):
    from paper_2501_18717_gb300 import bk
    dev = torch.device("cuda:0")
    ops, P, d, ld = _case(kind, dtype, m, m)
    t = [torch.from_numpy(a).to(dev) for a in ops]
    A = bk.csr_operator(*t) if kind == "csr" else bk.dense_operator(t[0])
    mu = 1e-2
    Pt = torch.from_numpy(P).to(dev)
    Yref = torch.zeros_like(Pt)
    Gref = torch.zeros(m, m, dtype=torch.float64, device=dev)
    with bk.Context(0) as ctx:
        bk.block_apply(ctx, A, mu, Pt, Yref, Gref, m, ld)
    # FP64: only the summation order differs. FP32: an FP32 dot product of the row
    # length (and, for dense FP32, the regular call's split-TF32 tensor-core product).
    tol = 1e-13 if dtype == "f64" else 3e-6
    Yo, Go = _oracle(kind, ops, P, d, m, mu)
    Yr = bk.from_panels(Yref.cpu().numpy(), d, m).astype(np.float64)
    assert np.max(np.abs(Yr - Yo)) <= tol * np.max(np.abs(Yo))
    assert np.max(np.abs(Gref.cpu().numpy() - Go)) <= tol * np.max(np.abs(Go))
    for call in range(2):  # two calls in a row share (and overwrite) the static scratch
        Y = torch.zeros_like(Pt)
        G = torch.zeros(m, m, dtype=torch.float64, device=dev)
        st = bk.block_apply_static(A, mu, Pt, Y, G, m, ld)
        assert st == bk.BK_OK, bk.status_string(st)
        Yn = bk.from_panels(Y.cpu().numpy(), d, m).astype(np.float64)
        assert np.max(np.abs(Yn - Yr)) <= tol * np.max(np.abs(Yr)), call
        assert np.max(np.abs(Yn - Yo)) <= tol * np.max(np.abs(Yo)), call
        Gn, Gr = G.cpu().numpy(), Gref.cpu().numpy()
        assert np.max(np.abs(Gn - Gr)) <= tol * np.max(np.abs(Gr)), call
        assert np.max(np.abs(Gn - Go)) <= tol * np.max(np.abs(Go)), call


def test_static_rejects_what_it_cannot_do_without_allocating():
    from paper_2501_18717_gb300 import bk
    dev = torch.device("cuda:0")
    ops, P, d, ld = _case("csr", "f32", 9, 1)
    A = bk.csr_operator(*[torch.from_numpy(a).to(dev) for a in ops])
    Pt = torch.from_numpy(P).to(dev)
    Y = torch.zeros_like(Pt)
    G = torch.zeros(9, 9, dtype=torch.float64, device=dev)
    # host arrays would need a staging buffer
    assert bk.block_apply_static(A, 0.0, P, Y, G, 9, ld) == bk.BK_ERR_ARG
    # FP64 values with FP32 blocks would need a converted copy
    A64 = bk.csr_operator(*[torch.from_numpy(a).to(dev) for a in (ops[0], ops[1], ops[2].astype(np.float64))])
    assert bk.block_apply_static(A64, 0.0, Pt, Y, G, 9, ld) == bk.BK_ERR_UNSUPPORTED
    # the same argument rules as bk_block_apply: a non-finite shift is refused
    assert bk.block_apply_static(A, float("inf"), Pt, Y, G, 9, ld) == bk.BK_ERR_ARG
    assert bk.block_apply_static(A, float("nan"), Pt, Y, G, 9, ld) == bk.BK_ERR_ARG
    # blocks wider than 36 (the fixed scratch array's limit) are refused before any launch
    assert bk.block_apply_static(A, 0.0, Pt, Y, G, 40, ld) == bk.BK_ERR_UNSUPPORTED
