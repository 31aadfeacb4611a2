"""Failure detection on the GPU: the bounded pipeline waits of the tensor-core block
product give up after bk_opts.timeout_cycles SM clocks, the kernel drains the copies
and MMAs it has issued, frees its tensor memory and returns, and the call reports
BK_TIMEOUT. The context stays usable: the same system then solves to tolerance with
the default limit. A limit of one clock makes the first wait that is not already
complete give up, so no fault, trap or hang is involved."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2501_18717_gb300 import workloads as W  # noqa: E402
from oracle import direct, operators  # noqa: E402


def _system(i, d):
    # FP32 rows of d floats (d a multiple of 4): 16-byte aligned, so the FP32 block
    # product runs on the tensor cores
    return W.batch_system(W.BASE_SEED + 61, i, d, dtype=np.float32)


def test_solve_times_out_then_context_solves():
    from paper_2501_18717_gb300 import bk
    dev = torch.device("cuda:0")
    d = 1024
    A, b = _system(0, d)
    Ad = torch.from_numpy(A).to(dev)
    bd = torch.from_numpy(b).to(dev)
    with bk.Context(0) as ctx:
        x = torch.zeros(d, dtype=torch.float64, device=dev)
        o = bk.default_opts(tol=1e-8, sketch=16, seed=2, inner="fp32", inner_tol=1e-5, timeout_cycles=1)
        info = bk.solve(ctx, bk.dense_operator(Ad), 0.0, bd, x, o, check=False)
        assert info.status == bk.BK_TIMEOUT, info.as_dict()
        assert "timed out" in ctx.last_error()
        # a negative limit is an argument error
        o.timeout_cycles = -1
        with pytest.raises(bk.BKError) as exc:
            bk.solve(ctx, bk.dense_operator(Ad), 0.0, bd, x, o)
        assert exc.value.status == bk.BK_ERR_ARG
        # the same context and system with the default limit
        x.zero_()
        o = bk.default_opts(tol=1e-8, sketch=16, seed=2, inner="fp32", inner_tol=1e-5)
        info = bk.solve(ctx, bk.dense_operator(Ad), 0.0, bd, x, o)
        assert info.status == bk.BK_OK
        rel = direct.rel_residual(operators.Dense(A.astype(np.float64)), 0.0, x.cpu().numpy(), b)
        assert rel <= 1e-8, (rel, info.as_dict())


def test_batched_solve_times_out_then_context_solves():
    from paper_2501_18717_gb300 import bk
    dev = torch.device("cuda:0")
    ds = [512, 768, 1024]
    systems = [_system(i, d) for i, d in enumerate(ds)]
    mats = [torch.from_numpy(A).to(dev) for A, _ in systems]
    bs = [torch.from_numpy(b).to(dev) for _, b in systems]
    with bk.Context(0) as ctx:
        xs = [torch.zeros(d, dtype=torch.float64, device=dev) for d in ds]
        batch = bk.Batch(mats, np.zeros(len(ds)), bs, xs)
        o = bk.default_opts(tol=1e-8, sketch=16, seed=4, inner="fp32", inner_tol=1e-5, timeout_cycles=1)
        with pytest.raises(bk.BKError) as exc:
            bk.solve_batched(ctx, batch, o)
        assert exc.value.status == bk.BK_TIMEOUT
        for x in xs:
            x.zero_()
        o = bk.default_opts(tol=1e-8, sketch=16, seed=4, inner="fp32", inner_tol=1e-5)
        infos = bk.solve_batched(ctx, batch, o)
        for (A, b), x, inf in zip(systems, xs, infos):
            assert inf.status == bk.BK_OK
            rel = direct.rel_residual(operators.Dense(A.astype(np.float64)), 0.0, x.cpu().numpy(), b)
            assert rel <= 1e-8, (rel, inf.as_dict())
