"""Python binding of the block-CG C ABI (include/bk.h): argument marshalling only.

Every entry point passes raw pointers and sizes straight to libbk.so; all arithmetic
runs in the library's CUDA kernels. Arrays may be torch tensors (CUDA or CPU) or
NumPy arrays; CUDA tensors are passed as device pointers, everything else as host
pointers (the library copies host arrays through its workspace). PyTorch is used
only for device memory and the current CUDA stream.

The library is required: importing this module without a built libbk.so raises
ImportError (there is no CPU fallback). Build it with
``python -m paper_2501_18717_gb300.build``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbk.so")

BK_OK, BK_ERR_ARG, BK_ERR_CUDA, BK_ERR_OOM, BK_NOT_CONVERGED, BK_BREAKDOWN, BK_STAGNATED, BK_TIMEOUT, \
    BK_ERR_UNSUPPORTED, BK_ERR_TOO_LARGE = range(10)
BK_DENSE, BK_CSR, BK_GRAM, BK_RBF = 0, 1, 2, 3
BK_F64, BK_F32 = 0, 1
BK_PREC_FP64, BK_PREC_FP32, BK_PREC_F32X2, BK_PREC_BF16, BK_PREC_OZAKI = 0, 1, 2, 3, 4

EXPORTS = ("bk_default_opts", "bk_create", "bk_destroy", "bk_set_stream", "bk_status_string", "bk_last_error",
           "bk_solve",
           "bk_block_apply", "bk_gram", "bk_chol_solve", "bk_gaussian", "bk_block_apply_static", "bk_ridge_path",
           "bk_sqrt_quadrature", "bk_sample", "bk_solve_batched", "bk_autotune", "bk_nystrom_pcg", "bk_sample_isqrt",
           "bk_solve_shrink")


class Operator(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dtype", ctypes.c_int32), ("rows", ctypes.c_int64),
                ("cols", ctypes.c_int64), ("ld", ctypes.c_int64), ("vals", ctypes.c_void_p),
                ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p), ("nnz", ctypes.c_int64),
                ("param", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_loads", ctypes.c_int32), ("sketch", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("inner", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("max_refine", ctypes.c_int32), ("check_every", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("timeout_cycles", ctypes.c_int64)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("loads", ctypes.c_int32), ("refinements", ctypes.c_int32),
                ("residual_loads", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("ms_kernel", ctypes.c_double * 8), ("launches", ctypes.c_int32 * 8),
                ("kernel_launches", ctypes.c_int32), ("deflations", ctypes.c_int32),
                ("fp64_fallback", ctypes.c_int32)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if not isinstance(v, (int, float)) else v
        return out


KERNEL_CLASSES = ("operator", "reduce", "alpha", "update_r", "beta", "update_p", "residual", "orth")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libbk.so is not built ({LIB_PATH}); run python -m paper_2501_18717_gb300.build")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    sig = {
        "bk_default_opts": (None, [ctypes.POINTER(Opts)]),
        "bk_create": (i32, [ctypes.POINTER(vp), ctypes.c_int, vp]),
        "bk_destroy": (i32, [vp]),
        "bk_set_stream": (i32, [vp, vp]),
        "bk_status_string": (ctypes.c_char_p, [i32]),
        "bk_last_error": (ctypes.c_char_p, [vp]),
        "bk_solve": (i32, [vp, ctypes.POINTER(Operator), dbl, vp, vp, ctypes.POINTER(Opts), ctypes.POINTER(Info)]),
        "bk_block_apply": (i32, [vp, ctypes.POINTER(Operator), dbl, i32, i64, vp, vp, i64, vp]),
        "bk_gram": (i32, [vp, i32, i64, i64, vp, vp, i64, vp]),
        "bk_chol_solve": (i32, [vp, i64, vp, vp, vp]),
        "bk_gaussian": (i32, [vp, u64, ctypes.c_uint32, i64, i64, vp]),
        "bk_block_apply_static": (i32, [ctypes.POINTER(Operator), dbl, i32, i64, vp, vp, i64, vp, vp]),
        "bk_sqrt_quadrature": (i32, [dbl, dbl, i32, vp, vp]),
        "bk_solve_batched": (i32, [vp, i32, vp, vp, vp, vp, ctypes.POINTER(Opts), vp]),
        "bk_autotune": (i32, [vp, i32, vp, vp, vp, vp, i32, ctypes.POINTER(Opts), vp]),
        "bk_sample": (i32, [vp, ctypes.POINTER(Operator), dbl, i32, vp, vp, i32, ctypes.POINTER(Opts),
                            ctypes.POINTER(Info)]),
        "bk_ridge_path": (i32, [vp, ctypes.POINTER(Operator), i32, vp, vp, vp, ctypes.POINTER(Opts),
                                ctypes.POINTER(Info)]),
        "bk_nystrom_pcg": (i32, [vp, ctypes.POINTER(Operator), dbl, vp, vp, i32, ctypes.POINTER(Opts),
                                 ctypes.POINTER(Info)]),
        "bk_sample_isqrt": (i32, [vp, ctypes.POINTER(Operator), dbl, i32, vp, vp, i32, ctypes.POINTER(Opts),
                                  ctypes.POINTER(Info)]),
        "bk_solve_shrink": (i32, [vp, ctypes.POINTER(Operator), dbl, vp, vp, i32, ctypes.POINTER(Opts),
                                  ctypes.POINTER(Info)]),
        "bk_apply": (i32, [vp, ctypes.POINTER(Operator), dbl, i32, vp, i64, vp, i64]),
        "bk_apply_ozaki": (i32, [vp, ctypes.POINTER(Operator), dbl, i32, vp, i64, vp, i64]),
        "bk_autotune_save": (i32, [vp, ctypes.c_char_p]),
        "bk_autotune_load": (i32, [vp, ctypes.c_char_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


class BKError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status}) {detail}".rstrip())


def status_string(s: int) -> str:
    return _lib.bk_status_string(int(s)).decode()


def _ptr(a):
    """(pointer, keepalive) of a torch tensor or NumPy array (must be contiguous)."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if not (a.flags["C_CONTIGUOUS"] or a.flags["F_CONTIGUOUS"]):
            raise ValueError("array must be contiguous")
        return a.ctypes.data, a
    if hasattr(a, "data_ptr"):
        return a.data_ptr(), a
    raise TypeError(f"unsupported array type {type(a)}")


def _dtype_code(a):
    s = str(getattr(a, "dtype", ""))
    if s.endswith("float64"):
        return BK_F64
    if s.endswith("float32"):
        return BK_F32
    raise TypeError(f"unsupported dtype {s}")


def _current_stream(device):
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream(device).cuda_stream
    except Exception:  # noqa: BLE001 - torch is optional for host-only callers
        pass
    return None


class Context:
    """A bk_ctx bound to one CUDA device and stream."""

    def __init__(self, device: int = 0, stream=None):
        self.device = device
        h = ctypes.c_void_p()
        st = _current_stream(device) if stream is None else stream
        s = _lib.bk_create(ctypes.byref(h), int(device), st)
        if s != BK_OK:
            raise BKError(s, "bk_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def last_error(self) -> str:
        return _lib.bk_last_error(self._h).decode()

    def set_stream(self, stream):
        s = _lib.bk_set_stream(self._h, stream)
        if s != BK_OK:
            raise BKError(s, "bk_set_stream")

    def close(self):
        if getattr(self, "_h", None):
            _lib.bk_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class OperatorRef:
    """A bk_operator plus references that keep its arrays alive."""

    def __init__(self, op: Operator, keep):
        self.op = op
        self.keep = keep
        self.d = op.rows


def dense_operator(a) -> OperatorRef:
    """A dense row-major d x d matrix (float64 or float32)."""
    d = a.shape[0]
    ld = a.stride(0) if hasattr(a, "stride") and callable(a.stride) else a.strides[0] // a.itemsize
    p, k = _ptr(a)
    op = Operator(BK_DENSE, _dtype_code(a), d, a.shape[1], ld, p, None, None, 0)
    return OperatorRef(op, [k])


def csr_operator(rowptr, colidx, vals) -> OperatorRef:
    """A CSR matrix with int32 rowptr/colidx and float64/float32 values."""
    d = rowptr.shape[0] - 1
    pr, kr = _ptr(rowptr)
    pc, kc = _ptr(colidx)
    pv, kv = _ptr(vals)
    op = Operator(BK_CSR, _dtype_code(vals), d, d, 0, pv, pr, pc, vals.shape[0])
    return OperatorRef(op, [kr, kc, kv])


def rbf_operator(points, lengthscale: float) -> OperatorRef:
    """K_ij = exp(-||x_i - x_j||^2 / (2 lengthscale^2)) formed on the fly from d points
    (d x 3 float64, row-major); never stored."""
    d = points.shape[0]
    ld = points.stride(0) if hasattr(points, "stride") and callable(points.stride) else points.strides[0] // points.itemsize
    p, k = _ptr(points)
    op = Operator(BK_RBF, _dtype_code(points), d, d, ld, p, None, None, 0, float(lengthscale))
    return OperatorRef(op, [k])


def gram_operator(Z) -> OperatorRef:
    """A = Z^T Z applied matrix-free; Z is n x d row-major (float64 or float32)."""
    n, d = Z.shape
    ld = Z.stride(0) if hasattr(Z, "stride") and callable(Z.stride) else Z.strides[0] // Z.itemsize
    p, k = _ptr(Z)
    op = Operator(BK_GRAM, _dtype_code(Z), n, d, ld, p, None, None, 0)
    ref = OperatorRef(op, [k])
    ref.d = d
    return ref


def default_opts(**kw) -> Opts:
    o = Opts()
    _lib.bk_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "inner" and isinstance(v, str):
            v = {"fp64": BK_PREC_FP64, "fp32": BK_PREC_FP32, "f32x2": BK_PREC_F32X2, "bf16": BK_PREC_BF16,
                 "ozaki": BK_PREC_OZAKI}[v]
        setattr(o, k, v)
    return o


def solve(ctx: Context, A: OperatorRef, mu: float, b, x, opts: Opts | None = None, check=True) -> Info:
    """bk_solve: x <- (A + mu I)^{-1} b by randomized block-CG with FP64 refinement."""
    info = Info()
    pb, kb = _ptr(b)
    px, kx = _ptr(x)
    o = opts if opts is not None else default_opts()
    s = _lib.bk_solve(ctx.handle, ctypes.byref(A.op), float(mu), pb, px, ctypes.byref(o), ctypes.byref(info))
    if check and s not in (BK_OK,):
        raise BKError(s, "bk_solve", ctx.last_error())
    return info


def to_panels(B, ld=None):
    """A d x m NumPy block as the library's panel layout: array (ceil(m/4), ld, 4) with
    element (i, c) at [c // 4, i, c % 4] and zero padding rows/columns."""
    d, m = B.shape
    ld = d if ld is None else ld
    nq = (m + 3) // 4
    out = np.zeros((nq, ld, 4), dtype=B.dtype)
    for c in range(m):
        out[c // 4, :d, c % 4] = B[:, c]
    return out


def from_panels(Pn, d, m):
    """The d x m block held in a panel-layout array (inverse of to_panels)."""
    Pn = np.asarray(Pn)
    return np.stack([Pn[c // 4, :d, c % 4] for c in range(m)], axis=1)


def ridge_path(ctx: Context, A: OperatorRef, mus, b, X, opts: Opts | None = None, check=True) -> Info:
    """bk_ridge_path: X[:, j] = (A + mus[j] I)^{-1} b for every shift from one
    block-Lanczos basis (X is d x L column-major: a Fortran-ordered array or the
    transpose view of an L x d row-major array)."""
    info = Info()
    pm, km = _ptr(mus)
    pb, kb = _ptr(b)
    px, kx = _ptr(X)
    o = opts if opts is not None else default_opts()
    s = _lib.bk_ridge_path(ctx.handle, ctypes.byref(A.op), int(len(mus)), pm, pb, px, ctypes.byref(o),
                           ctypes.byref(info))
    if check and s != BK_OK:
        raise BKError(s, "bk_ridge_path", ctx.last_error())
    return info


def sample_isqrt(ctx: Context, K: OperatorRef, nugget: float, B, S, n_quad: int = 32, opts: Opts | None = None,
                 check=True) -> Info:
    """bk_sample_isqrt: S ~= (K + nugget I)^{-1/2} B (B, S d x m column-major)."""
    info = Info()
    pb, kb = _ptr(B)
    ps, ks = _ptr(S)
    m = B.shape[1]
    o = opts if opts is not None else default_opts()
    st = _lib.bk_sample_isqrt(ctx.handle, ctypes.byref(K.op), float(nugget), int(m), pb, ps, int(n_quad),
                              ctypes.byref(o), ctypes.byref(info))
    if check and st != BK_OK:
        raise BKError(st, "bk_sample_isqrt", ctx.last_error())
    return info


def nystrom_pcg(ctx: Context, A: OperatorRef, mu: float, b, x, s_ny: int = 1, opts: Opts | None = None,
                check=True) -> Info:
    """bk_nystrom_pcg: x ~= (A + mu I)^{-1} b by Nystrom-preconditioned CG (depth s_ny)."""
    info = Info()
    pb, kb = _ptr(b)
    px, kx = _ptr(x)
    o = opts if opts is not None else default_opts()
    s = _lib.bk_nystrom_pcg(ctx.handle, ctypes.byref(A.op), float(mu), pb, px, int(s_ny), ctypes.byref(o),
                            ctypes.byref(info))
    if check and s != BK_OK:
        raise BKError(s, "bk_nystrom_pcg", ctx.last_error())
    return info


def solve_shrink(ctx: Context, A: OperatorRef, mu: float, b, x, s_lock: int = 3, opts: Opts | None = None,
                 check=True) -> Info:
    """bk_solve_shrink: x ~= (A + mu I)^{-1} b by s_lock block steps on [b Omega], then
    one-column deflated CG against the locked basis."""
    info = Info()
    pb, kb = _ptr(b)
    px, kx = _ptr(x)
    o = opts if opts is not None else default_opts()
    s = _lib.bk_solve_shrink(ctx.handle, ctypes.byref(A.op), float(mu), pb, px, int(s_lock), ctypes.byref(o),
                             ctypes.byref(info))
    if check and s != BK_OK:
        raise BKError(s, "bk_solve_shrink", ctx.last_error())
    return info


def apply(ctx: Context, A: OperatorRef, mu: float, X, Y, ldx: int | None = None, ldy: int | None = None,
          ozaki: bool = False) -> None:
    """bk_apply: Y = A X + mu X in FP64. X and Y are column-major (a Fortran-ordered
    NumPy array or a transposed contiguous torch tensor) with the operator's d rows
    first in each column; the leading dimensions default to the column strides.
    ozaki=True calls bk_apply_ozaki (dense FP32 A on the BF16 tensor cores)."""
    def cols(a):
        if len(a.shape) == 1:
            return 1, int(a.shape[0])
        st = a.strides[1] // a.itemsize if isinstance(a, np.ndarray) else a.stride(1)
        return int(a.shape[1]), int(st)
    L, sx = cols(X)
    _, sy = cols(Y)
    px, kx = _ptr(X)
    py, ky = _ptr(Y)
    fn = _lib.bk_apply_ozaki if ozaki else _lib.bk_apply
    s = fn(ctx.handle, ctypes.byref(A.op), float(mu), L, px, int(ldx or sx), py, int(ldy or sy))
    if s != BK_OK:
        raise BKError(s, "bk_apply_ozaki" if ozaki else "bk_apply", ctx.last_error())


def block_apply(ctx: Context, A: OperatorRef, mu: float, P, Y, G, m: int, ld: int, dtype=None) -> None:
    """bk_block_apply: Y = A P + mu P and G = P^T Y (panel-layout blocks, leading dim ld)."""
    dt = _dtype_code(P) if dtype is None else dtype
    pp, kp = _ptr(P)
    py, ky = _ptr(Y)
    pg, kg = _ptr(G)
    s = _lib.bk_block_apply(ctx.handle, ctypes.byref(A.op), float(mu), dt, int(m), pp, py, int(ld), pg)
    if s != BK_OK:
        raise BKError(s, "bk_block_apply", ctx.last_error())


def gram(ctx: Context, X, Y, G, d: int, m: int, ld: int) -> None:
    """bk_gram: G = X^T Y for d x m blocks in the panel layout."""
    px, kx = _ptr(X)
    py, ky = _ptr(Y)
    pg, kg = _ptr(G)
    s = _lib.bk_gram(ctx.handle, _dtype_code(X), int(d), int(m), px, py, int(ld), pg)
    if s != BK_OK:
        raise BKError(s, "bk_gram")


def chol_solve(ctx: Context, G, S, X, m: int) -> int:
    """bk_chol_solve: X = G^{-1} S (m x m, row-major FP64). Returns the status."""
    pg, kg = _ptr(G)
    ps, ks = _ptr(S)
    px, kx = _ptr(X)
    return _lib.bk_chol_solve(ctx.handle, int(m), pg, ps, px)


def gaussian(ctx: Context, seed: int, stream: int, out, offset: int = 0) -> None:
    """bk_gaussian: normals offset .. offset + len(out) - 1 of a Philox stream."""
    po, ko = _ptr(out)
    n = out.shape[0]
    s = _lib.bk_gaussian(ctx.handle, int(seed), int(stream), int(n), int(offset), po)
    if s != BK_OK:
        raise BKError(s, "bk_gaussian")


def block_apply_static(A: OperatorRef, mu: float, P, Y, G, m: int, ld: int, stream=None, dtype=None) -> int:
    """bk_block_apply_static: bk_block_apply without device allocation (device arrays
    only; scratch in a fixed static array shared by all calls on a device). Returns the
    status; callers that cannot allocate device memory use this entry point."""
    dt = _dtype_code(P) if dtype is None else dtype
    pp, kp = _ptr(P)
    py, ky = _ptr(Y)
    pg, kg = _ptr(G)
    return _lib.bk_block_apply_static(ctypes.byref(A.op), float(mu), dt, int(m), pp, py, int(ld), pg, stream)


def sqrt_quadrature(lo: float, hi: float, n: int):
    """bk_sqrt_quadrature: (z_j^2, w_j) with sqrt(x) ~= sum_j w_j x / (x + z_j^2) on [lo, hi]."""
    z2 = np.zeros(n)
    w = np.zeros(n)
    st = _lib.bk_sqrt_quadrature(float(lo), float(hi), int(n), z2.ctypes.data, w.ctypes.data)
    if st != BK_OK:
        raise BKError(st, "bk_sqrt_quadrature")
    return z2, w


def sample(ctx: Context, K: OperatorRef, nugget: float, B, S, n_quad: int = 32, opts: Opts | None = None,
           check=True) -> Info:
    """bk_sample: S ~= (K + nugget I)^{1/2} B (B, S d x m column-major)."""
    info = Info()
    pb, kb = _ptr(B)
    ps, ks = _ptr(S)
    m = B.shape[1]
    o = opts if opts is not None else default_opts()
    st = _lib.bk_sample(ctx.handle, ctypes.byref(K.op), float(nugget), int(m), pb, ps, int(n_quad),
                        ctypes.byref(o), ctypes.byref(info))
    if check and st != BK_OK:
        raise BKError(st, "bk_sample", ctx.last_error())
    return info


class Batch:
    """Marshalled arguments of a batch of dense systems (operator array, shift array,
    pointer arrays of b and x) for bk_solve_batched and bk_autotune."""

    def __init__(self, mats, mus, bs, xs):
        n = len(mats)
        self.ops = [dense_operator(a) for a in mats]
        self.op_arr = (Operator * n)(*[o.op for o in self.ops])
        self.mu = np.ascontiguousarray(np.asarray(mus, dtype=np.float64))
        self.b_arr = (ctypes.c_void_p * n)(*[_ptr(v)[0] for v in bs])
        self.x_arr = (ctypes.c_void_p * n)(*[_ptr(v)[0] for v in xs])
        self.keep = (mats, bs, xs)
        self.n = n


def autotune_save(ctx: Context, path: str) -> None:
    """bk_autotune_save: the context's autotune table to a text file."""
    s = _lib.bk_autotune_save(ctx.handle, str(path).encode())
    if s != BK_OK:
        raise BKError(s, "bk_autotune_save", ctx.last_error())


def autotune_load(ctx: Context, path: str) -> None:
    """bk_autotune_load: replace the context's autotune table with a saved one."""
    s = _lib.bk_autotune_load(ctx.handle, str(path).encode())
    if s != BK_OK:
        raise BKError(s, "bk_autotune_load", ctx.last_error())


def autotune_table(ctx: Context, path: str) -> dict:
    """The context's autotune table {floor(log2 d): (sketch, kernel)} (written through
    bk_autotune_save to `path`, then parsed)."""
    autotune_save(ctx, path)
    table = {}
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            bkt, sk, tc = (int(v) for v in line.split())
            table[bkt] = (sk, {0: "cuda", 1: "tensor", 2: "cuda32"}[tc])
    return table


def solve_batched(ctx: Context, batch: Batch, opts: Opts | None = None, check=True):
    """bk_solve_batched: returns the list of per-system Info records."""
    infos = (Info * batch.n)()
    o = opts if opts is not None else default_opts()
    st = _lib.bk_solve_batched(ctx.handle, batch.n, ctypes.cast(batch.op_arr, ctypes.c_void_p),
                               batch.mu.ctypes.data, ctypes.cast(batch.b_arr, ctypes.c_void_p),
                               ctypes.cast(batch.x_arr, ctypes.c_void_p), ctypes.byref(o),
                               ctypes.cast(infos, ctypes.c_void_p))
    if check and st != BK_OK:
        raise BKError(st, "bk_solve_batched", ctx.last_error())
    return list(infos)


def autotune(ctx: Context, batch: Batch, candidates, opts: Opts | None = None):
    """bk_autotune: returns the chosen sketch per calibration system."""
    cand = np.ascontiguousarray(np.asarray(candidates, dtype=np.int32))
    chosen = np.zeros(batch.n, dtype=np.int32)
    o = opts if opts is not None else default_opts()
    st = _lib.bk_autotune(ctx.handle, batch.n, ctypes.cast(batch.op_arr, ctypes.c_void_p), batch.mu.ctypes.data,
                          ctypes.cast(batch.b_arr, ctypes.c_void_p), cand.ctypes.data, len(cand), ctypes.byref(o),
                          chosen.ctypes.data)
    if st != BK_OK:
        raise BKError(st, "bk_autotune", ctx.last_error())
    return chosen
