// C ABI of the block-CG library (include/bk.h): context, workspace, argument checks
// and the host control of the solve. Every arithmetic step runs in the kernels of
// k_ops.cu, k_block.cu and k_rng.cu; the host only orders launches, reads the device
// control block every `check_every` steps and sums small partial vectors.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/bk.h"
#include "bk_common.cuh"
#include "bk_ctx.h"

using bk::DevState;

using namespace bkx;

namespace {

size_t dtype_size(int dt) { return dt == BK_F64 ? 8 : 4; }

struct OpDev {
  int kind, dtype;
  int64_t d, lda, nnz;
  const void* vals;
  const int* rowptr;
  const int* colidx;
};

cudaError_t stage_operator(bk_ctx* c, const bk_operator* A, OpDev* o) {
  o->kind = A->kind;
  o->dtype = A->dtype;
  o->d = A->rows;
  o->nnz = A->nnz;
  o->lda = A->ld;
  size_t es = dtype_size(A->dtype);
  cudaError_t e;
  if (A->kind == BK_DENSE) {
    size_t bytes = ((size_t)(A->rows - 1) * A->ld + A->cols) * es;
    e = stage_in(c, WS_OP_VALS, A->vals, bytes, &o->vals);
    o->rowptr = o->colidx = nullptr;
    return e;
  }
  e = stage_in(c, WS_OP_ROW, A->rowptr, (size_t)(A->rows + 1) * 4, (const void**)&o->rowptr);
  if (e != cudaSuccess) return e;
  e = stage_in(c, WS_OP_COL, A->colidx, (size_t)A->nnz * 4, (const void**)&o->colidx);
  if (e != cudaSuccess) return e;
  return stage_in(c, WS_OP_VALS, A->vals, (size_t)A->nnz * es, &o->vals);
}

// Values of the operator in the inner precision (converted copy when needed).
cudaError_t inner_values(bk_ctx* c, const OpDev& o, int want_f64, const void** out, int64_t* lda_out) {
  *lda_out = o.lda;
  int have_f64 = o.dtype == BK_F64;
  if (have_f64 == want_f64) {
    *out = o.vals;
    return cudaSuccess;
  }
  void* buf = nullptr;
  cudaError_t e;
  if (o.kind == BK_CSR) {
    e = ws_get(c, WS_VALS_INNER, (size_t)o.nnz * (want_f64 ? 8 : 4), &buf);
    if (e != cudaSuccess) return e;
    e = want_f64 ? bk::launch_to_f64(o.nnz, (const float*)o.vals, (double*)buf, c->stream)
                 : bk::launch_to_f32(o.nnz, (const double*)o.vals, (float*)buf, c->stream);
  } else {
    int64_t lda2 = (o.d + 3) & ~int64_t(3);
    e = ws_get(c, WS_VALS_INNER, (size_t)o.d * lda2 * (want_f64 ? 8 : 4), &buf);
    if (e != cudaSuccess) return e;
    if (want_f64) {
      // FP32 storage, FP64 inner: promote row by row (the dense copy keeps lda)
      e = bk::launch_to_f64((o.d - 1) * o.lda + o.d, (const float*)o.vals, (double*)buf, c->stream);
      lda2 = o.lda;
    } else {
      e = bk::launch_dense_to_f32(o.d, (const double*)o.vals, o.lda, (float*)buf, lda2, c->stream);
    }
    *lda_out = lda2;
  }
  *out = buf;
  return e;
}

cudaError_t residual(bk_ctx* c, const OpDev& o, double mu, const double* x, const double* b, double* r,
                     double* normp, double* rnorm) {
  int np = bk::residual_parts(o.d);
  cudaError_t e = (o.kind == BK_CSR)
                      ? bk::launch_csr_residual(o.dtype == BK_F64, o.d, o.rowptr, o.colidx, o.vals, mu, x, b, r,
                                                normp, np, c->stream)
                      : bk::launch_dense_residual(o.dtype == BK_F64, o.d, o.vals, o.lda, mu, x, b, r, normp, np,
                                                  c->stream);
  if (e != cudaSuccess) return e;
  double s2 = 0.0;
  e = host_sum(c, normp, np, &s2);
  *rnorm = std::sqrt(s2);
  return e;
}

struct SolveBufs {
  void *P, *Q, *Y, *omega, *gi_t, *xc_t, *ti_t, *t_t;
  float* pt = nullptr;  // P^T head/tail for the tensor-core dense product
  double *xin, *x64, *r64, *partsG, *partsS, *G, *S, *cvec, *normp;
  DevState* state;
  int npG, npS;
};

}  // namespace

extern "C" {

void bk_default_opts(bk_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-10;
  o->max_loads = 20000;
  o->sketch = 20;
  o->seed = 0;
  o->inner = BK_PREC_FP64;
  o->inner_tol = 1e-6;
  o->max_refine = 8;
  o->check_every = 8;
  o->profile = 0;
}

const char* bk_status_string(bk_status s) {
  switch (s) {
    case BK_OK: return "ok";
    case BK_ERR_ARG: return "invalid argument";
    case BK_ERR_CUDA: return "CUDA error";
    case BK_ERR_OOM: return "device out of memory";
    case BK_NOT_CONVERGED: return "not converged";
    case BK_BREAKDOWN: return "block breakdown (Gram matrix not positive definite)";
    case BK_STAGNATED: return "refinement stagnated";
    case BK_TIMEOUT: return "device wait timed out";
    case BK_ERR_UNSUPPORTED: return "unsupported operator, dtype or block width";
    case BK_ERR_TOO_LARGE: return "problem exceeds the fixed static scratch";
  }
  return "unknown status";
}

bk_status bk_create(bk_ctx** out, int device, void* cuda_stream) {
  if (!out) return BK_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return BK_ERR_CUDA;
  }
  BK_CK(cudaSetDevice(device));
  bk_ctx* c = new bk_ctx();
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  if (!c->stream) {
    // The legacy default stream cannot be captured into a CUDA graph. A blocking
    // stream of our own is implicitly ordered with it, so callers that use the
    // default stream see the same ordering.
    if (cudaStreamCreate(&c->own_stream) != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return BK_ERR_CUDA;
    }
    c->stream = c->own_stream;
  }
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  cudaError_t e = cudaMallocHost((void**)&c->hstate, sizeof(DevState));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->hparts, kHostParts * sizeof(double));
  if (e != cudaSuccess) {
    if (c->hstate) cudaFreeHost(c->hstate);
    delete c;
    return from_cuda(e);
  }
  *out = c;
  return BK_OK;
}

bk_status bk_destroy(bk_ctx* c) {
  if (!c) return BK_ERR_ARG;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (auto& b : c->ws)
    if (b.p) cudaFree(b.p);
  cudaFreeHost(c->hstate);
  cudaFreeHost(c->hparts);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
  return BK_OK;
}

bk_status bk_set_stream(bk_ctx* c, void* s) {
  if (!c) return BK_ERR_ARG;
  c->stream = s ? (cudaStream_t)s : c->own_stream;
  if (!c->stream) {
    if (cudaStreamCreate(&c->own_stream) != cudaSuccess) {
      cudaGetLastError();
      return BK_ERR_CUDA;
    }
    c->stream = c->own_stream;
  }
  return BK_OK;
}

const char* bk_last_error(const bk_ctx* c) { return c ? c->last_error : ""; }

bk_status bk_gaussian(bk_ctx* c, uint64_t seed, uint32_t stream, int64_t n, int64_t offset, double* out) {
  err_ctx() = c;
  if (c) c->last_error[0] = 0;
  if (!c || !out || n < 0 || offset < 0) return BK_ERR_ARG;
  if (n == 0) return BK_OK;
  BK_CK(cudaSetDevice(c->device));
  bool dev = is_device_ptr(out);
  double* d = out;
  if (!dev) BK_CK(ws_get(c, WS_TMP_OUT, (size_t)n * 8, (void**)&d));
  BK_CK(bk::launch_gaussian(seed, stream, n, offset, d, c->stream));
  if (!dev) BK_CK(cudaMemcpyAsync(out, d, (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream));
  BK_CK(cudaStreamSynchronize(c->stream));
  return BK_OK;
}

bk_status bk_chol_solve(bk_ctx* c, int64_t m, const double* G, const double* S, double* X) {
  err_ctx() = c;
  if (c) c->last_error[0] = 0;
  if (!c || !G || !S || !X || m < 1 || m > bk::kMaxWidth) return BK_ERR_ARG;
  BK_CK(cudaSetDevice(c->device));
  size_t bytes = (size_t)m * m * 8;
  const void *g = nullptr, *s = nullptr;
  BK_CK(stage_in(c, WS_TMP_G, G, bytes, &g));
  BK_CK(stage_in(c, WS_TMP_S, S, bytes, &s));
  bool dev = is_device_ptr(X);
  void* xo = X;
  if (!dev) BK_CK(ws_get(c, WS_TMP_OUT, bytes, &xo));
  int* flag = nullptr;
  BK_CK(ws_get(c, WS_STATE, 64, (void**)&flag));
  BK_CK(cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
  BK_CK(bk::launch_chol_solve((int)m, (const double*)g, (const double*)s, (double*)xo, flag, c->stream));
  int hflag = 0;
  BK_CK(cudaMemcpyAsync(c->hparts, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  if (!dev) BK_CK(cudaMemcpyAsync(X, xo, bytes, cudaMemcpyDeviceToHost, c->stream));
  BK_CK(cudaStreamSynchronize(c->stream));
  std::memcpy(&hflag, c->hparts, sizeof(int));
  return hflag ? BK_BREAKDOWN : BK_OK;
}

bk_status bk_gram(bk_ctx* c, int32_t dtype, int64_t d, int64_t m, const void* X, const void* Y, int64_t ld,
                  double* G) {
  err_ctx() = c;
  if (c) c->last_error[0] = 0;
  if (!c || !X || !Y || !G || d < 1 || m < 1 || ld < d) return BK_ERR_ARG;
  if (dtype != BK_F64 && dtype != BK_F32) return BK_ERR_UNSUPPORTED;
  int mp = bk::padded_width((int)m);
  if (mp < 0 || m > bk::kMaxWidth) return BK_ERR_UNSUPPORTED;
  BK_CK(cudaSetDevice(c->device));
  size_t es = dtype_size(dtype);
  size_t bytes = ((size_t)((m + 3) / 4 - 1) * ld + d) * 4 * es;  // panel layout
  const void *x = nullptr, *y = nullptr;
  BK_CK(stage_in(c, WS_TMP_IN, X, bytes, &x));
  BK_CK(stage_in(c, WS_TMP_G, Y, bytes, &y));
  int is64 = dtype == BK_F64;
  int np = bk::gram_grid(is64, mp, d, c->device);
  double* parts = nullptr;
  BK_CK(ws_get(c, WS_PARTS_S, (size_t)np * bk::gram_entries(mp) * 8, (void**)&parts));
  bool dev = is_device_ptr(G);
  double* go = G;
  if (!dev) BK_CK(ws_get(c, WS_TMP_OUT, (size_t)m * m * 8, (void**)&go));
  BK_CK(bk::launch_gram(is64, mp, d, x, y, ld, (int)m, parts, np, c->stream));
  BK_CK(bk::launch_reduce_gram(mp, (int)m, parts, np, go, nullptr, c->stream));
  if (!dev) BK_CK(cudaMemcpyAsync(G, go, (size_t)m * m * 8, cudaMemcpyDeviceToHost, c->stream));
  BK_CK(cudaStreamSynchronize(c->stream));
  return BK_OK;
}

bk_status bk_block_apply(bk_ctx* c, const bk_operator* A, double mu, int32_t dtype, int64_t m, const void* P,
                         void* Y, int64_t ld, double* G) {
  err_ctx() = c;
  if (c) c->last_error[0] = 0;
  if (!c || !P || !Y || !G) return BK_ERR_ARG;
  bk_status s = check_operator(A);
  if (s != BK_OK) return s;
  if (m < 1 || ld < A->rows || !std::isfinite(mu)) return BK_ERR_ARG;
  if (dtype != BK_F64 && dtype != BK_F32) return BK_ERR_UNSUPPORTED;
  int mp = bk::padded_width((int)m);
  if (mp < 0 || m > bk::kMaxWidth) return BK_ERR_UNSUPPORTED;
  BK_CK(cudaSetDevice(c->device));
  OpDev o;
  BK_CK(stage_operator(c, A, &o));
  int is64 = dtype == BK_F64;
  const void* vin = nullptr;
  int64_t lda_in = o.lda;
  BK_CK(inner_values(c, o, is64, &vin, &lda_in));
  int64_t d = o.d;
  size_t es = dtype_size(dtype);
  size_t bytes = ((size_t)((m + 3) / 4 - 1) * ld + d) * 4 * es;  // panel layout
  const void* p = nullptr;
  BK_CK(stage_in(c, WS_TMP_IN, P, bytes, &p));
  bool ydev = is_device_ptr(Y);
  void* yo = Y;
  if (!ydev) BK_CK(ws_get(c, WS_TMP_S, bytes, &yo));
  const bool use_tc = o.kind == BK_DENSE && !is64 && bk::dense_tc_usable(d, vin, lda_in, mp);
  int np = (o.kind == BK_CSR) ? bk::csr_spmm_gram_grid(is64, mp, d, c->device)
                              : (use_tc ? bk::dense_tc_tiles(d) : bk::dense_gram_grid(is64, mp, d, c->device));
  double* parts = nullptr;
  BK_CK(ws_get(c, WS_PARTS_G, (size_t)np * bk::gram_entries(mp) * 8, (void**)&parts));
  bool gdev = is_device_ptr(G);
  double* go = G;
  if (!gdev) BK_CK(ws_get(c, WS_TMP_OUT, (size_t)m * m * 8, (void**)&go));
  int* tcerr = nullptr;
  if (o.kind == BK_CSR)
    BK_CK(bk::launch_csr_spmm_gram(is64, mp, d, o.rowptr, o.colidx, vin, mu, p, yo, ld, (int)m, parts, np, nullptr,
                                   c->stream));
  else if (use_tc) {
    float* pt = nullptr;
    BK_CK(ws_get(c, WS_PT, bk::dense_tc_pt_bytes(d, mp), (void**)&pt));
    BK_CK(ws_get(c, WS_TCERR, 64, (void**)&tcerr));
    BK_CK(cudaMemsetAsync(tcerr, 0, sizeof(int), c->stream));
    BK_CK(bk::launch_dense_gram_tc(mp, d, (const float*)vin, lda_in, mu, (const float*)p, (float*)yo, ld, (int)m,
                                   parts, np, nullptr, pt, tcerr, 0, c->stream));
  } else
    BK_CK(bk::launch_dense_gram(is64, mp, d, vin, lda_in, mu, p, yo, ld, (int)m, parts, np, nullptr, c->stream));
  BK_CK(bk::launch_reduce_gram(mp, (int)m, parts, np, go, nullptr, c->stream));
  if (!ydev) BK_CK(cudaMemcpyAsync(Y, yo, bytes, cudaMemcpyDeviceToHost, c->stream));
  if (!gdev) BK_CK(cudaMemcpyAsync(G, go, (size_t)m * m * 8, cudaMemcpyDeviceToHost, c->stream));
  int herr = 0;
  if (tcerr) BK_CK(cudaMemcpyAsync(c->hparts, tcerr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  BK_CK(cudaStreamSynchronize(c->stream));
  if (tcerr) std::memcpy(&herr, c->hparts, sizeof(int));
  if (herr) {
    std::snprintf(c->last_error, sizeof(c->last_error), "tensor-core pipeline wait timed out");
    return BK_TIMEOUT;
  }
  return BK_OK;
}

// allow_fallback: FP32-block passes that stop reducing the residual hand the rest of
// the solve to FP64 blocks (a nested call on the residual system, which has no
// fallback itself).
static bk_status solve_impl(bk_ctx* c, const bk_operator* A, double mu, const double* b, double* x,
                            const bk_opts* opts_in, bk_info* info, bool allow_fallback) {
  err_ctx() = c;
  if (c && allow_fallback) c->last_error[0] = 0;
  if (info) std::memset(info, 0, sizeof(*info));
  if (!c || !b || !x) return BK_ERR_ARG;
  bk_status s = check_operator(A);
  if (s != BK_OK) return s;
  bk_opts opts;
  if (opts_in)
    opts = *opts_in;
  else
    bk_default_opts(&opts);
  if (!(mu >= 0.0) || !std::isfinite(mu) || !(opts.tol > 0.0) || opts.sketch < 0 || opts.max_loads < 1 ||
      opts.max_refine < 1 || !(opts.inner_tol > 0.0) || opts.check_every < 1 || opts.timeout_cycles < 0)
    return BK_ERR_ARG;
  if (opts.inner != BK_PREC_FP64 && opts.inner != BK_PREC_FP32) return BK_ERR_UNSUPPORTED;
  // a block wider than the space it lives in is rank deficient from the start
  const int m = (int)((int64_t)opts.sketch + 1 < A->rows ? opts.sketch + 1 : A->rows);
  const int mp = bk::padded_width(m);
  if (mp < 0 || m > bk::kMaxWidth) return BK_ERR_UNSUPPORTED;
  const int is64 = opts.inner == BK_PREC_FP64;
  BK_CK(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  cudaEvent_t ev0, ev1;
  BK_CK(cudaEventCreate(&ev0));
  BK_CK(cudaEventCreate(&ev1));
  BK_CK(cudaEventRecord(ev0, st));

  OpDev o;
  BK_CK(stage_operator(c, A, &o));
  const int64_t d = o.d;
  const void* vin = nullptr;
  int64_t lda_in = o.lda;
  BK_CK(inner_values(c, o, is64, &vin, &lda_in));
  const double* bd = nullptr;
  BK_CK(stage_in(c, WS_B64, b, (size_t)d * 8, (const void**)&bd));

  // workspace
  const int64_t ld = (d + 31) & ~int64_t(31);
  const size_t es = is64 ? 8 : 4;
  // every block holds all mp / 4 panels of the padded width (the step kernels are
  // compiled for it); padding columns stay zero
  const size_t blk = (size_t)ld * mp * es;
  SolveBufs w;
  BK_CK(ws_get(c, WS_P, blk, &w.P));
  BK_CK(ws_get(c, WS_R, blk, &w.Q));
  BK_CK(ws_get(c, WS_Y, blk, &w.Y));
  BK_CK(ws_get(c, WS_OMEGA, blk, &w.omega));
  BK_CK(cudaMemsetAsync(w.P, 0, blk, st));
  BK_CK(cudaMemsetAsync(w.Q, 0, blk, st));
  BK_CK(cudaMemsetAsync(w.Y, 0, blk, st));
  BK_CK(ws_get(c, WS_XIN, (size_t)d * 8, (void**)&w.xin));
  BK_CK(ws_get(c, WS_X64, (size_t)d * 8, (void**)&w.x64));
  BK_CK(ws_get(c, WS_R64, (size_t)d * 8, (void**)&w.r64));
  // trial iterate and residual of each refinement pass (swapped with x64 / r64 when kept)
  double *xt = nullptr, *rt = nullptr;
  BK_CK(ws_get(c, WS_XT, (size_t)d * 8, (void**)&xt));
  BK_CK(ws_get(c, WS_RT, (size_t)d * 8, (void**)&rt));
  // dense FP32 products run on the tensor cores when the matrix layout allows TMA
  const bool use_tc = o.kind == BK_DENSE && !is64 && bk::dense_tc_usable(d, vin, lda_in, mp);
  w.npG = (o.kind == BK_CSR) ? bk::csr_spmm_gram_grid(is64, mp, d, c->device)
                             : (use_tc ? bk::dense_tc_tiles(d) : bk::dense_gram_grid(is64, mp, d, c->device));
  if (use_tc) BK_CK(ws_get(c, WS_PT, bk::dense_tc_pt_bytes(d, mp), (void**)&w.pt));
  w.npS = bk::update_r_grid(is64, mp, d, c->device);
  int npStart = bk::gram_grid(is64, mp, d, c->device);
  int ne = bk::gram_entries(mp);
  int npSmax = w.npS > npStart ? w.npS : npStart;
  BK_CK(ws_get(c, WS_PARTS_G, (size_t)w.npG * ne * 8, (void**)&w.partsG));
  BK_CK(ws_get(c, WS_PARTS_S, (size_t)npSmax * ne * 8, (void**)&w.partsS));
  size_t mm = (size_t)m * m, mpp = (size_t)mp * mp;
  const size_t ncv = mp > 64 ? (size_t)mp : 64;  // slots of c (m <= mp)
  double* mats = nullptr;
  BK_CK(ws_get(c, WS_MATS, (2 * mm + ncv + 3 * mpp + mp) * 8 + 256, (void**)&mats));
  w.G = mats;
  w.S = w.G + mm;
  w.cvec = w.S + mm;
  w.gi_t = (void*)(w.cvec + ncv);
  w.ti_t = (void*)((char*)w.gi_t + mpp * 8);
  w.t_t = (void*)((char*)w.ti_t + mpp * 8);
  w.xc_t = (void*)((char*)w.t_t + mpp * 8);
  BK_CK(ws_get(c, WS_STATE, sizeof(DevState) + 64, (void**)&w.state));
  BK_CK(ws_get(c, WS_NORMP, kHostParts * 8, (void**)&w.normp));

  // Omega once per solve; its columns are scaled to unit expected norm (the Krylov
  // space, and so the column-0 iterate, does not depend on column scaling).
  BK_CK(cudaMemsetAsync(w.omega, 0, blk, st));  // column 0 and padding columns stay zero
  BK_CK(bk::launch_omega(is64, d, m - 1, ld, opts.seed, 1.0 / std::sqrt((double)d), w.omega, st));
  BK_CK(cudaMemsetAsync(w.x64, 0, (size_t)d * 8, st));
  BK_CK(cudaMemcpyAsync(w.r64, bd, (size_t)d * 8, cudaMemcpyDeviceToDevice, st));
  double bnorm2 = 0.0;
  int nnp = bk::residual_parts(d);
  BK_CK(bk::launch_norm2_parts(d, bd, w.normp, nnp, st));
  BK_CK(host_sum(c, w.normp, nnp, &bnorm2));
  const double bnorm = std::sqrt(bnorm2);

  int loads = 0, refinements = 0, residual_loads = 0, stagnant = 0, deflations = 0;
  bool fallback = false;
  // Inner target floor: an inner solve in FP32 blocks stops reducing the true residual
  // at a level set by the block precision and the conditioning (the recurrence keeps
  // going below it). When a pass that met its target reduced the FP64 residual by far
  // less, later passes stop at half the reduction that pass achieved.
  double floor_target = 0.0;
  int launches = 3;  // omega, norm, (x copy is a memcpy)
  bk_status result = BK_NOT_CONVERGED;
  double rnorm = bnorm;
  const bool use_graph = std::getenv("BK_NO_GRAPH") == nullptr;
  cudaGraphExec_t gexec = nullptr;

  // Scaled pivots below this count as dependent directions: the Gram matrices carry
  // the rounding of the block precision (about 1e-15 relative in FP64, 1e-7 in FP32).
  const double rank_tol = is64 ? 1e-12 : 1e-6;
  // profiling: one event before each of the 7 launches of a step and one after
  constexpr int kEv = 8;
  const int nprof = opts.profile ? opts.check_every : 0;
  std::vector<cudaEvent_t> pev((size_t)nprof * kEv);
  for (auto& e : pev) BK_CK(cudaEventCreate(&e));
  double ms_k[8] = {0};
  int n_k[8] = {0};
  static const int kClass[7] = {BK_K_OPERATOR, BK_K_REDUCE, BK_K_ALPHA, BK_K_UPDATE_R, BK_K_REDUCE, BK_K_BETA,
                                BK_K_UPDATE_P};
  int prof_it = 0;
  auto mark = [&](int k) -> cudaError_t {
    if (!nprof) return cudaSuccess;
    // inside stream capture an external record becomes an event-record node of the graph
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    cudaEvent_t ev = pev[(size_t)prof_it * kEv + k];
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal)
                                               : cudaEventRecord(ev, st);
  };
  auto step = [&]() -> cudaError_t {
    cudaError_t e;
    if ((e = mark(0)) != cudaSuccess) return e;
    if (o.kind == BK_CSR)
      e = bk::launch_csr_spmm_gram(is64, mp, d, o.rowptr, o.colidx, vin, mu, w.P, w.Y, ld, m, w.partsG, w.npG,
                                   w.state, st);
    else if (use_tc)
      e = bk::launch_dense_gram_tc(mp, d, (const float*)vin, lda_in, mu, (const float*)w.P, (float*)w.Y, ld, m,
                                   w.partsG, w.npG, w.state, w.pt, &w.state->timeout, opts.timeout_cycles, st);
    else
      e = bk::launch_dense_gram(is64, mp, d, vin, lda_in, mu, w.P, w.Y, ld, m, w.partsG, w.npG, w.state, st);
    if (e != cudaSuccess) return e;
    if ((e = mark(1)) != cudaSuccess) return e;
    if ((e = bk::launch_reduce_gram(mp, m, w.partsG, w.npG, w.G, w.state, st)) != cudaSuccess) return e;
    if ((e = mark(2)) != cudaSuccess) return e;
    if ((e = bk::launch_small_alpha(is64, mp, m, w.G, w.cvec, w.gi_t, w.xc_t, rank_tol, w.state, st)) != cudaSuccess)
      return e;
    if ((e = mark(3)) != cudaSuccess) return e;
    if ((e = bk::launch_update_r(is64, mp, d, m, w.Y, w.Q, ld, w.gi_t, w.partsS, w.npS, w.state, st)) != cudaSuccess)
      return e;
    if ((e = mark(4)) != cudaSuccess) return e;
    if ((e = bk::launch_reduce_gram(mp, m, w.partsS, w.npS, w.S, w.state, st)) != cudaSuccess) return e;
    if ((e = mark(5)) != cudaSuccess) return e;
    if ((e = bk::launch_small_beta(is64, mp, m, w.S, w.cvec, w.ti_t, w.t_t, rank_tol, w.state, st)) != cudaSuccess)
      return e;
    if ((e = mark(6)) != cudaSuccess) return e;
    if ((e = bk::launch_update_p(is64, mp, d, m, w.Q, w.P, ld, w.xc_t, w.ti_t, w.t_t, w.xin, w.state, st)) !=
        cudaSuccess)
      return e;
    if ((e = mark(7)) != cudaSuccess) return e;
    if (nprof) prof_it = (prof_it + 1) % nprof;
    return cudaSuccess;
  };

  if (bnorm == 0.0) {
    result = BK_OK;
    rnorm = 0.0;
  }
  while (result != BK_OK) {
    if (rnorm <= opts.tol * bnorm) {
      result = BK_OK;
      break;
    }
    if (refinements >= opts.max_refine || loads >= opts.max_loads) {
      result = BK_NOT_CONVERGED;
      break;
    }
    double target = std::fmax(std::fmax(opts.inner_tol, 0.5 * opts.tol * bnorm / rnorm), floor_target);
    if (target > 0.5) target = 0.5;
    // start block: Q = [r / ||r||, Omega], S = Q^T Q = T^T T, Q <- Q T^{-1}, P = Q, c = T e_1
    BK_CK(bk::launch_start_block(is64, d, m, ld, w.r64, 1.0 / rnorm, w.omega, w.Q, w.xin, st));
    BK_CK(bk::launch_gram(is64, mp, d, w.Q, w.Q, ld, m, w.partsS, npStart, st));
    BK_CK(bk::launch_reduce_gram(mp, m, w.partsS, npStart, w.S, nullptr, st));
    BK_CK(bk::launch_init_state(w.state, opts.max_loads - loads, target, w.cvec, m, st));
    BK_CK(bk::launch_small_beta(is64, mp, m, w.S, w.cvec, w.ti_t, w.t_t, rank_tol, w.state, st));
    BK_CK(bk::launch_update_p(is64, mp, d, m, w.Q, w.P, ld, w.xc_t, w.ti_t, w.t_t, w.xin, w.state, st));
    launches += 6;  // start block, Gram, reduce, state, factor, normalise
    for (int chunk = 0;; ++chunk) {
      if (use_graph && (chunk > 0 || gexec)) {
        if (!gexec) {
          cudaGraph_t g;
          BK_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
          cudaError_t ce = cudaSuccess;
          for (int it = 0; it < opts.check_every && ce == cudaSuccess; ++it) ce = step();
          cudaError_t ee = cudaStreamEndCapture(st, &g);
          if (ce != cudaSuccess) return from_cuda(ce);
          BK_CK(ee);
          ee = cudaGraphInstantiate(&gexec, g, 0);
          cudaGraphDestroy(g);
          BK_CK(ee);
        }
        BK_CK(cudaGraphLaunch(gexec, st));
      } else {
        for (int it = 0; it < opts.check_every; ++it) BK_CK(step());
      }
      launches += 7 * opts.check_every;
      const int loads_before = chunk == 0 ? 0 : c->hstate->loads;
      BK_CK(cudaMemcpyAsync(c->hstate, w.state, sizeof(DevState), cudaMemcpyDeviceToHost, st));
      BK_CK(cudaStreamSynchronize(st));
      if (nprof) {
        // steps of this chunk that did work: the first (loads delta) of them
        int active = c->hstate->loads - loads_before;
        for (int it = 0; it < active && it < nprof; ++it)
          for (int k = 0; k < 7; ++k) {
            float ms = 0.f;
            BK_CK(cudaEventElapsedTime(&ms, pev[(size_t)it * kEv + k], pev[(size_t)it * kEv + k + 1]));
            ms_k[kClass[k]] += ms;
            n_k[kClass[k]] += 1;
          }
      }
      if (c->hstate->done_a || c->hstate->done_b || c->hstate->timeout) break;
    }
    const DevState hs = *c->hstate;
    loads += hs.loads;
    deflations += m - hs.kept;
    refinements += 1;
    if (hs.timeout) {
      std::snprintf(c->last_error, sizeof(c->last_error), "tensor-core pipeline wait timed out");
      result = BK_TIMEOUT;
      break;
    }
    // trial iterate x + ||r|| xin and its FP64 residual. A pass whose residual is not
    // finite, or that broke down without reducing it, lost its recurrence: x stays as
    // it was (the next pass would repeat this one). Any other pass is kept, also one
    // capped by the load limit whose residual grew (the CG residual 2-norm is not
    // monotone).
    BK_CK(bk::launch_axpy_out(d, rnorm, w.xin, w.x64, xt, st));
    double rn = 0.0;
    BK_CK(residual(c, o, mu, xt, bd, rt, w.normp, &rn));
    residual_loads += 1;
    launches += 2;  // axpy, residual
    if (!std::isfinite(rn) || (hs.status == bk::ST_BREAKDOWN && !(rn < rnorm))) {
      if (!is64 && allow_fallback) {
        fallback = true;
        break;
      }
      result = BK_BREAKDOWN;
      break;
    }
    std::swap(w.x64, xt);
    std::swap(w.r64, rt);
    if (rn <= opts.tol * bnorm) {
      rnorm = rn;
      result = BK_OK;
      break;
    }
    const double achieved = rn / rnorm;
    if (hs.status == bk::ST_CONVERGED && achieved > 4.0 * target) floor_target = 0.5 * achieved;
    rnorm = rn;
    if (!(achieved < 0.5) && ++stagnant >= 2) {
      if (!is64 && allow_fallback) {
        fallback = true;
        break;
      }
      result = BK_STAGNATED;
      break;
    }
  }
  if (gexec) cudaGraphExecDestroy(gexec);
  for (auto& e : pev) cudaEventDestroy(e);

  if (fallback) {
    // FP32 blocks stopped reducing the residual: the correction delta of A_mu delta = r
    // is solved in FP64 blocks (a nested solve with FP64 residuals as before) and
    // x <- x + delta. x and r move to slots the nested solve does not use.
    double *fx = nullptr, *fr = nullptr, *fd = nullptr;
    BK_CK(ws_get(c, WS_FB_X, (size_t)d * 8, (void**)&fx));
    BK_CK(ws_get(c, WS_FB_R, (size_t)d * 8, (void**)&fr));
    BK_CK(ws_get(c, WS_FB_D, (size_t)d * 8, (void**)&fd));
    BK_CK(cudaMemcpyAsync(fx, w.x64, (size_t)d * 8, cudaMemcpyDeviceToDevice, st));
    BK_CK(cudaMemcpyAsync(fr, w.r64, (size_t)d * 8, cudaMemcpyDeviceToDevice, st));
    w.x64 = fx;
    result = BK_NOT_CONVERGED;
    if (opts.max_loads > loads) {
      bk_opts o64 = opts;
      o64.inner = BK_PREC_FP64;
      o64.tol = opts.tol * bnorm / rnorm;
      o64.max_loads = opts.max_loads - loads;
      o64.max_refine = std::max(1, opts.max_refine - refinements);
      bk_info sub;
      const bk_status ss = solve_impl(c, A, mu, fr, fd, &o64, &sub, false);
      if (ss != BK_OK && ss != BK_NOT_CONVERGED && ss != BK_BREAKDOWN && ss != BK_STAGNATED) return ss;
      BK_CK(bk::launch_axpy(d, 1.0, fd, fx, st));
      loads += sub.loads;
      refinements += sub.refinements;
      residual_loads += sub.residual_loads;
      deflations += sub.deflations;
      launches += sub.kernel_launches + 1;
      for (int k = 0; k < 8; ++k) {
        ms_k[k] += sub.ms_kernel[k];
        n_k[k] += sub.launches[k];
      }
      rnorm *= sub.rel_residual;
      result = ss;
    }
  }

  // result back to the caller's x
  BK_CK(cudaMemcpyAsync(x, w.x64, (size_t)d * 8, cudaMemcpyDefault, st));
  BK_CK(cudaEventRecord(ev1, st));
  BK_CK(cudaEventSynchronize(ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (info) {
    info->status = result;
    info->loads = loads;
    info->deflations = deflations;
    info->refinements = refinements;
    info->residual_loads = residual_loads;
    info->rel_residual = bnorm > 0 ? rnorm / bnorm : 0.0;
    info->ms_total = ms;
    for (int k = 0; k < 8; ++k) {
      info->ms_kernel[k] = ms_k[k];
      info->launches[k] = n_k[k];
    }
    info->kernel_launches = launches;
    info->fp64_fallback = fallback ? 1 : 0;
  }
  return result;
}

bk_status bk_solve(bk_ctx* c, const bk_operator* A, double mu, const double* b, double* x, const bk_opts* opts_in,
                   bk_info* info) {
  return solve_impl(c, A, mu, b, x, opts_in, info, true);
}

}  // extern "C"
