// Block-Lanczos drivers of the C ABI: bk_ridge_path (Sec. 3.2, Eq. bcg_alg, one basis
// for every shift) and bk_sample (Def. blansq). The host orders launches and reads
// small status vectors; the products, Grams, factorisations and shifted solves run in
// the kernels of k_gemm.cu and k_krylov.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/bk.h"
#include "bk_common.cuh"
#include "bk_ctx.h"

using namespace bkx;

namespace {

// The operator of a Lanczos run: A dense (d x d row-major) or A = Z^T Z (Z nrows x d
// row-major), values FP32 or FP64.
struct LzOp {
  int kind = BK_DENSE;
  int64_t d = 0, nrows = 0, ld = 0;
  const void* vals = nullptr;
  int vals_f64 = 0;
  double param = 0.0;           // BK_RBF: lengthscale (FP64 blocks only)
  const int* rowptr = nullptr;  // BK_CSR (FP64 blocks only)
  const int* colidx = nullptr;
  int64_t nnz = 0;
};

// CUDA events around kernel groups of a profiled driver call (opts.profile): one pair
// per group, summed per class (BK_K_*) once the call has finished.
struct Prof {
  bool on = false;
  cudaStream_t st = nullptr;
  std::vector<cudaEvent_t> ev[BK_K_CLASSES];
  cudaEvent_t open = nullptr;
  void begin() {
    if (!on) return;
    cudaEventCreate(&open);
    cudaEventRecord(open, st);
  }
  void end(int cls) {
    if (!on || !open) return;
    cudaEvent_t e1 = nullptr;
    cudaEventCreate(&e1);
    cudaEventRecord(e1, st);
    ev[cls].push_back(open);
    ev[cls].push_back(e1);
    open = nullptr;
  }
  // after the stream has been synchronised
  void report(bk_info* info) {
    for (int k = 0; k < BK_K_CLASSES; ++k) {
      double ms = 0.0;
      for (size_t i = 0; i + 1 < ev[k].size(); i += 2) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, ev[k][i], ev[k][i + 1]) == cudaSuccess) ms += t;
      }
      if (info) {
        info->ms_kernel[k] += ms;
        info->launches[k] += (int)(ev[k].size() / 2);
      }
      for (cudaEvent_t e : ev[k]) cudaEventDestroy(e);
      ev[k].clear();
    }
    if (open) cudaEventDestroy(open);
    open = nullptr;
  }
};

// FP64-accurate products of FP32-stored values through the compensated tall-skinny
// kernels: Y (d x nc, FP64) = A X (BK_DENSE) or Z^T (Z X) (BK_GRAM; V is an nrows x nc
// FP64 scratch). Each FP64 operand is split once into FP32 head and tail arrays.
cudaError_t df_apply(bk_ctx* c, const LzOp& o, const double* X, int64_t ldx, int nc, double* Y, int64_t ldy, double* V,
                     int64_t ldv, cudaStream_t st) {
  const int64_t lds = (o.d + 3) & ~int64_t(3);
  const int64_t ldr = (o.nrows + 3) & ~int64_t(3);
  const size_t need = (size_t)2 * lds * nc * 4 + (o.kind == BK_GRAM ? (size_t)2 * ldr * nc * 4 : 0) + 64;
  void* wsv = nullptr;
  cudaError_t e = ws_get(c, WS_SPLITB, need, &wsv);
  if (e != cudaSuccess) return e;
  float* Xh = (float*)wsv;
  float* Xl = Xh + (size_t)lds * nc;
  if ((e = bk::launch_split_f64(o.d, nc, X, ldx, Xh, Xl, lds, st)) != cudaSuccess) return e;
  const float* A = (const float*)o.vals;
  if (o.kind == BK_DENSE) return bk::launch_tsm_nn(1, o.d, nc, o.d, 1.0, A, o.ld, Xh, Xl, lds, 0.0, Y, ldy, st);
  if ((e = bk::launch_tsm_nn(1, o.nrows, nc, o.d, 1.0, A, o.ld, Xh, Xl, lds, 0.0, V, ldv, st)) != cudaSuccess) return e;
  float* Vh = Xl + (size_t)lds * nc;
  float* Vl = Vh + (size_t)ldr * nc;
  if ((e = bk::launch_split_f64(o.nrows, nc, V, ldv, Vh, Vl, ldr, st)) != cudaSuccess) return e;
  void* wk = nullptr;
  const size_t wb = bk::tsm_tn_work_bytes(o.nrows, o.d, nc, 1, c->sms);
  if ((e = ws_get(c, WS_TSM, wb, &wk)) != cudaSuccess) return e;
  return bk::launch_tsm_tn(1, o.nrows, o.d, nc, A, o.ld, Vh, Vl, ldr, 1.0, 0.0, Y, ldy, wk, wb, c->sms, st);
}

// Y (d x nc, FP64) = K X for the on-the-fly RBF operator (X split into FP32 head and tail).
cudaError_t rbf_apply(bk_ctx* c, const LzOp& o, const double* X, int64_t ldx, int nc, double* Y, int64_t ldy,
                      cudaStream_t st) {
  const int64_t lds = (o.d + 3) & ~int64_t(3);
  void* wsv = nullptr;
  cudaError_t e = ws_get(c, WS_SPLITB, (size_t)2 * lds * nc * 4 + 64, &wsv);
  if (e != cudaSuccess) return e;
  float* Xh = (float*)wsv;
  float* Xl = Xh + (size_t)lds * nc;
  if ((e = bk::launch_split_f64(o.d, nc, X, ldx, Xh, Xl, lds, st)) != cudaSuccess) return e;
  return bk::launch_rbf_apply(o.d, nc, (const double*)o.vals, o.ld, o.param, Xh, Xl, lds, Y, ldy, st);
}

// Block-Lanczos with full reorthogonalisation (classical Gram-Schmidt twice against
// every previous block) and CholQR2 for the block QR (Sec. 3.2, Thm. cost). Blocks are
// column-major with leading dimension ldq, in the precision of the run (FP32 or FP64);
// T_t is assembled in FP64 band storage from FP64 Grams.
struct Lanczos {
  bk_ctx* c = nullptr;
  cudaStream_t st = nullptr;
  int is64 = 1;
  size_t es = 8;
  LzOp op;
  int m = 0, tmax = 0;
  int64_t d = 0, ldq = 0, ncol_max = 0, ldv = 0;
  void *Q = nullptr, *W = nullptr, *V = nullptr, *C = nullptr, *Rt = nullptr, *M3 = nullptr;
  double *G = nullptr, *R1 = nullptr, *R2 = nullptr, *Ri1 = nullptr, *Ri2 = nullptr, *work = nullptr;
  double *Ak = nullptr, *Bk = nullptr, *R0 = nullptr, *band = nullptr;
  int *keep = nullptr, *rank = nullptr;
  double* ci_scratch = nullptr;
  Prof* prof = nullptr;  // optional event timing
  int df = 0;            // FP64 blocks: FP32 values through the compensated products
  // FP32 blocks of a Gram-form operator on BF16 tensor cores (k_bf16.cu): the BF16
  // copies of Z, the products' workspace and the timeout flag; null otherwise
  const void* bz = nullptr;
  void* bwork = nullptr;
  size_t bwork_bytes = 0;
  int* berr = nullptr;
  // FP64 blocks of a dense FP32 operator through the Ozaki split on the BF16 tensor
  // cores (k_ozaki.cu): the operator's digits, the block's workspace, the timeout flag
  const void* oza = nullptr;
  void* ozx = nullptr;
  int* ozerr = nullptr;
  bool ozb = false;  // FP64 basis products (Grams, reorthogonalisation, Q = W R^{-1}) split too
  int t = 0;      // blocks in T_t
  int loads = 0;  // operator applications
  double rank_tol = 1e-12;

  int n() const { return t * m; }
  int ldb() const { return (int)ncol_max; }
  void* qblock(int k) const { return (char*)Q + (size_t)k * m * ldq * es; }

  cudaError_t init(bk_ctx* ctx, const LzOp& o, int is64_, int m_, int tmax_) {
    c = ctx;
    st = ctx->stream;
    op = o;
    is64 = is64_;
    es = is64 ? 8 : 4;
    m = m_;
    tmax = tmax_;
    d = o.d;
    ldq = (d + 31) & ~int64_t(31);
    ncol_max = (int64_t)m * (tmax + 1);
    rank_tol = is64 ? 1e-12 : 1e-6;
    cudaError_t e;
    if ((e = ws_get(c, WS_LQ, (size_t)ldq * ncol_max * es, &Q)) != cudaSuccess) return e;
    if ((e = ws_get(c, WS_LW, (size_t)ldq * m * es, &W)) != cudaSuccess) return e;
    ldv = (op.nrows + 3) & ~int64_t(3);
    if (op.kind == BK_GRAM)
      if ((e = ws_get(c, WS_LV, (size_t)ldv * m * es, &V)) != cudaSuccess) return e;
    if ((e = ws_get(c, WS_LC, (size_t)ncol_max * m * es, &C)) != cudaSuccess) return e;
    if ((e = ws_get(c, WS_LQ2, (size_t)2 * m * m * es, &M3)) != cudaSuccess) return e;
    double* sm = nullptr;
    const size_t mm = (size_t)m * m;
    if ((e = ws_get(c, WS_LSMALL, (11 * mm + 2 * m + 64) * 8, (void**)&sm)) != cudaSuccess) return e;
    G = sm;
    R1 = G + mm;
    R2 = R1 + mm;
    Ri1 = R2 + mm;
    Ri2 = Ri1 + mm;
    work = Ri2 + mm;
    Ak = work + mm;
    Bk = Ak + mm;
    R0 = Bk + mm;
    Rt = (void*)(R0 + mm);  // m x m in the block precision
    keep = (int*)(R0 + 2 * mm);
    rank = keep + m + 8;
    ci_scratch = R0 + 2 * mm + m + 16;  // 2 m doubles after keep and rank
    if ((e = ws_get(c, WS_LBAND, (size_t)(m + 1) * ncol_max * 8, (void**)&band)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(band, 0, (size_t)(m + 1) * ncol_max * 8, st)) != cudaSuccess) return e;
    t = 0;
    loads = 0;
    return cudaSuccess;
  }

  // Y (d x nc, ldy) = A X (d x nc, ldx), block precision. FP32 runs use the tall-skinny
  // product kernels (k_tsm.cu); FP64 runs the general GEMM.
  cudaError_t apply(const void* X, int64_t ldx, void* Y, int64_t ldy, int nc) {
    cudaError_t e;
    const int af = op.vals_f64;  // 1: FP64 values, 0: FP32 values
    if (!is64 && af) return cudaErrorInvalidValue;  // FP32 runs use FP32 values
    if (is64 && oza && op.kind == BK_DENSE && !af)
      return bk::launch_ozaki_apply(d, nc, oza, (const double*)X, ldx, (double*)Y, ldy, ozx, 0, ozerr, c->sms, st);
    if (!is64 && bz && op.kind == BK_GRAM)
      return bk::launch_bf16_gram_apply(op.nrows, d, nc, bz, (const float*)X, ldx, (float*)Y, ldy, 1.0, 0.0, bwork,
                                        bwork_bytes, 0, berr, c->sms, st);
    if (is64 && df && !af && (op.kind == BK_DENSE || op.kind == BK_GRAM) && bk::tsm_supported(op.vals, op.ld))
      return df_apply(c, op, (const double*)X, ldx, nc, (double*)Y, ldy, (double*)V, ldv, st);
    if (!is64 && (op.kind == BK_DENSE || op.kind == BK_GRAM) && bk::tsm_supported(op.vals, op.ld) &&
        bk::tsm_supported(X, ldx)) {
      const float* A = (const float*)op.vals;
      const float* Xf = (const float*)X;
      if (op.kind == BK_DENSE) return bk::launch_tsm_nn(0, d, nc, d, 1.0, A, op.ld, Xf, nullptr, ldx, 0.0, Y, ldy, st);
      if ((e = bk::launch_tsm_nn(0, op.nrows, nc, d, 1.0, A, op.ld, Xf, nullptr, ldx, 0.0, V, ldv, st)) != cudaSuccess)
        return e;
      void* wk = nullptr;
      const size_t wb = bk::tsm_tn_work_bytes(op.nrows, d, nc, 0, c->sms);
      if ((e = ws_get(c, WS_TSM, wb, &wk)) != cudaSuccess) return e;
      return bk::launch_tsm_tn(0, op.nrows, d, nc, A, op.ld, (const float*)V, nullptr, ldv, 1.0, 0.0, Y, ldy, wk, wb,
                               c->sms, st);
    }
    if (op.kind == BK_RBF) {
      if (!is64) return cudaErrorInvalidValue;
      return rbf_apply(c, op, (const double*)X, ldx, nc, (double*)Y, ldy, st);
    }
    if (op.kind == BK_CSR) {
      if (!is64) return cudaErrorInvalidValue;
      return bk::launch_csr_cols(af, d, op.rowptr, op.colidx, op.vals, nc, (const double*)X, ldx, (double*)Y, ldy,
                                 st);
    }
    if (op.kind == BK_DENSE) {
      e = bk::launch_gemm(is64, d, nc, d, 1.0, op.vals, af, op.ld, 1, X, 1, ldx, 0.0, Y, ldy, st);
    } else {
      e = bk::launch_gemm(is64, op.nrows, nc, d, 1.0, op.vals, af, op.ld, 1, X, 1, ldx, 0.0, V, ldv, st);
      if (e != cudaSuccess) return e;
      e = bk::launch_gemm(is64, d, nc, op.nrows, 1.0, op.vals, af, 1, op.ld, V, 1, ldv, 0.0, Y, ldy, st);
    }
    return e;
  }

  // Split-K general product for tall reductions (Grams, Q^T W): K = d is long and the
  // output has few tiles.
  // In an F32X2 run the products that build the basis (reorthogonalisation, the
  // three-term step, Q = W R^{-1}) use the double-float GEMM, about 2^-44 relative
  // (CholQR2's second pass restores orthogonality); the Grams that give the entries of
  // T_t (allow_dd = false) stay in FP64, since the shifted solves and the square root
  // resolve T_t's smallest eigenvalues. FP64 runs use the FP64 GEMM throughout. In an
  // Ozaki run (ozb) every FP64 basis product, the Grams of T_t included, goes through
  // the Ozaki split: 2^-45 of the block bounds, the order of an FP64 GEMM's rounding
  // over K = d (about sqrt(d) u).
  cudaError_t gemm_k(int out64, int64_t M, int64_t N, int64_t K, double alpha, const void* A, int a_f64, int64_t sai,
                     int64_t sak, const void* B, int64_t sbk, int64_t sbj, double beta, void* C, int64_t ldc,
                     bool allow_dd = true) {
    const size_t wb = bk::gemm_split_work_bytes(out64, M, N, K, c->sms);
    void* wk = nullptr;
    if (wb) {
      cudaError_t e = ws_get(c, WS_SPLIT, wb, &wk);
      if (e != cudaSuccess) return e;
    }
    if (ozb && is64 && out64 && a_f64 == 1 && bk::ozaki_gemm_usable(M, N, K, sai, sak, sbk, sbj)) {
      void* ow = nullptr;
      cudaError_t e = ws_get(c, WS_OZ_G, bk::ozaki_gemm_work_bytes(M, N, K, c->sms), &ow);
      if (e != cudaSuccess) return e;
      return bk::launch_ozaki_gemm(M, N, K, alpha, (const double*)A, sai, sak, (const double*)B, sbk, sbj, beta,
                                   (double*)C, ldc, ow, 0, ozerr, c->sms, st);
    }
    if (allow_dd && df && is64 && out64 && a_f64 == 1)
      return bk::launch_gemm_dd(M, N, K, alpha, (const double*)A, sai, sak, (const double*)B, sbk, sbj, beta,
                                (double*)C, ldc, wk, wb, c->sms, st);
    return bk::launch_gemm_split(out64, M, N, K, alpha, A, a_f64, sai, sak, B, sbk, sbj, beta, C, ldc, wk, wb, c->sms,
                                 st);
  }

  // CholQR2: Wb (d x m) = Qout Bout, Bout upper triangular (m x m row-major FP64).
  cudaError_t qr(void* Wb, void* Qout, double* Bout) {
    cudaError_t e;
    const int gaf = is64 ? 1 : 2;  // Gram of the block: FP64 accumulation of exact products
    for (int pass = 0; pass < 2; ++pass) {
      const void* src = pass == 0 ? Wb : Qout;
      double* R = pass == 0 ? R1 : R2;
      double* Ri = pass == 0 ? Ri1 : Ri2;
      if ((e = gemm_k(1, m, m, d, 1.0, src, gaf, ldq, 1, src, 1, ldq, 0.0, G, m, false)) != cudaSuccess)
        return e;
      if ((e = bk::launch_chol_inv(m, G, rank_tol, work, R, Ri, keep, rank, ci_scratch, st)) != cudaSuccess)
        return e;
      // Qout = src * Ri (Ri row-major: element (k, j) at Ri[k m + j])
      if (is64) {
        e = gemm_k(1, d, m, m, 1.0, src, 1, 1, ldq, Ri, m, 1, 0.0, Qout, ldq);
      } else {
        if ((e = bk::launch_copy_cols(1, 0, (int64_t)m * m, 1, Ri, (int64_t)m * m, Rt, (int64_t)m * m, st)) !=
            cudaSuccess)
          return e;
        e = bk::launch_gemm(0, d, m, m, 1.0, src, 0, 1, ldq, Rt, m, 1, 0.0, Qout, ldq, st);
      }
      if (e != cudaSuccess) return e;
    }
    // Bout = R2 R1 in row-major: computed as (R2 R1)^T in column-major
    return bk::launch_gemm(1, m, m, m, 1.0, R1, 1, 1, m, R2, 1, m, 0.0, Bout, m, st);
  }

  // Start block B0 (d x m, block precision, ldq) -> Q_0 and R_0.
  cudaError_t start(const void* B0) { return qr(const_cast<void*>(B0), qblock(0), R0); }

  // One Lanczos step: Q_t, A_t, B_t, Q_{t+1}; T grows by one block.
  cudaError_t step() {
    cudaError_t e;
    const int k = t;
    const void* Qk = qblock(k);
    if (prof) prof->begin();
    if ((e = apply(Qk, ldq, W, ldq, m)) != cudaSuccess) return e;
    if (prof) prof->end(BK_K_OPERATOR);
    ++loads;
    if (prof) prof->begin();
    // A_k = Q_k^T (A Q_k) with FP64 accumulation
    const int gaf = is64 ? 1 : 2;
    if ((e = gemm_k(1, m, m, d, 1.0, Qk, gaf, ldq, 1, W, 1, ldq, 0.0, Ak, m, false)) != cudaSuccess) return e;
    // three-term recurrence W -= Q_{k-1} B_{k-1}^T + Q_k A_k (Bk still holds B_{k-1}),
    // then one classical Gram-Schmidt pass against Q_0..Q_k for what rounding left along
    // the older blocks (full reorthogonalisation; the first pass of a CGS2 against all
    // blocks would remove the same two terms, so the result equals it up to rounding)
    if ((e = bk::launch_three_term(is64, m, k == 0, Ak, Bk, M3, st)) != cudaSuccess) return e;
    if (k == 0)
      e = gemm_k(is64, d, m, m, -1.0, Qk, is64, 1, ldq, (const char*)M3 + (size_t)m * es, 1, 2 * m, 1.0, W, ldq);
    else
      e = gemm_k(is64, d, m, 2 * m, -1.0, qblock(k - 1), is64, 1, ldq, M3, 1, 2 * m, 1.0, W, ldq);
    if (e != cudaSuccess) return e;
    const int64_t nk = (int64_t)(k + 1) * m;
    if ((e = gemm_k(is64, nk, m, d, 1.0, Q, is64, ldq, 1, W, 1, ldq, 0.0, C, nk)) != cudaSuccess) return e;
    if ((e = gemm_k(is64, d, m, nk, -1.0, Q, is64, 1, ldq, C, 1, nk, 1.0, W, ldq)) != cudaSuccess) return e;
    if ((e = qr(W, qblock(k + 1), Bk)) != cudaSuccess) return e;
    if (prof) prof->end(BK_K_ORTH);
    if ((e = bk::launch_band_put(ldb(), m, m, k, Ak, Bk, band, st)) != cudaSuccess) return e;
    ++t;
    return cudaSuccess;
  }
};

bk_status check_lz_operator(const bk_operator* A, LzOp* o) {
  if (!A || !A->vals) return BK_ERR_ARG;
  if (A->dtype != BK_F64 && A->dtype != BK_F32) return BK_ERR_UNSUPPORTED;
  o->vals_f64 = A->dtype == BK_F64;
  if (A->kind == BK_DENSE) {
    if (A->rows <= 0 || A->rows != A->cols || A->ld < A->cols) return BK_ERR_ARG;
    o->kind = BK_DENSE;
    o->d = A->rows;
    o->ld = A->ld;
    o->nrows = 0;
    return BK_OK;
  }
  if (A->kind == BK_RBF) {
    if (A->rows <= 0 || A->rows != A->cols || A->ld < 3 || !(A->param > 0.0)) return BK_ERR_ARG;
    if (A->dtype != BK_F64) return BK_ERR_UNSUPPORTED;
    o->kind = BK_RBF;
    o->d = A->rows;
    o->ld = A->ld;
    o->nrows = 0;
    o->param = A->param;
    return BK_OK;
  }
  if (A->kind == BK_GRAM) {
    if (A->rows <= 0 || A->cols <= 0 || A->ld < A->cols) return BK_ERR_ARG;
    o->kind = BK_GRAM;
    o->d = A->cols;
    o->nrows = A->rows;
    o->ld = A->ld;
    return BK_OK;
  }
  return BK_ERR_UNSUPPORTED;
}

// Device copy of the operator values, in FP32 when the run is FP32 and they are FP64.
cudaError_t stage_lz_values(bk_ctx* c, const bk_operator* A, LzOp* o, int want_f64, const void** staged) {
  const size_t es = A->dtype == BK_F64 ? 8 : 4;
  const int64_t rows = A->rows;
  if (A->kind == BK_RBF) {  // the points (FP64, d x 3 with row stride ld)
    const void* dv = nullptr;
    cudaError_t e = stage_in(c, WS_OP_VALS, A->vals, ((size_t)(rows - 1) * A->ld + 3) * 8, &dv);
    o->vals = dv;
    *staged = dv;
    return e;
  }
  const size_t bytes = ((size_t)(rows - 1) * A->ld + A->cols) * es;
  const void* dv = nullptr;
  cudaError_t e = stage_in(c, WS_OP_VALS, A->vals, bytes, &dv);
  if (e != cudaSuccess) return e;
  o->vals = dv;
  *staged = dv;
  if (!want_f64 && o->vals_f64) {
    void* f = nullptr;
    if ((e = ws_get(c, WS_VALS_INNER, ((size_t)(rows - 1) * A->ld + A->cols) * 4, &f)) != cudaSuccess) return e;
    if ((e = bk::launch_to_f32((int64_t)(rows - 1) * A->ld + A->cols, (const double*)dv, (float*)f, c->stream)) !=
        cudaSuccess)
      return e;
    o->vals = f;
    o->vals_f64 = 0;
  }
  return cudaSuccess;
}

// FP64 products A X for L columns (refinement residuals): X, AX d x L column-major (ld).
// With allow_df, FP32 values go through the compensated tall-skinny products (about
// 2^-44 relative to sum |a_ik x_k|, on the FP32 pipe); otherwise, and for FP64 values,
// through the FP64 GEMM.
cudaError_t apply_fp64(bk_ctx* c, const LzOp& o, const double* X, int64_t ld, int L, double* AX, double* Vw,
                       bool allow_df) {
  if (o.kind == BK_CSR)
    return bk::launch_csr_cols(o.vals_f64, o.d, o.rowptr, o.colidx, o.vals, L, X, ld, AX, ld, c->stream);
  if (o.kind == BK_RBF) return rbf_apply(c, o, X, ld, L, AX, ld, c->stream);
  if (allow_df && !o.vals_f64 && (o.kind == BK_DENSE || o.kind == BK_GRAM) && bk::tsm_supported(o.vals, o.ld))
    return df_apply(c, o, X, ld, L, AX, ld, Vw, o.nrows, c->stream);
  if (o.kind == BK_DENSE) return bk::launch_gemm(1, o.d, L, o.d, 1.0, o.vals, o.vals_f64, o.ld, 1, X, 1, ld, 0.0, AX,
                                                 ld, c->stream);
  cudaError_t e =
      bk::launch_gemm(1, o.nrows, L, o.d, 1.0, o.vals, o.vals_f64, o.ld, 1, X, 1, ld, 0.0, Vw, o.nrows, c->stream);
  if (e != cudaSuccess) return e;
  return bk::launch_gemm(1, o.d, L, o.nrows, 1.0, o.vals, o.vals_f64, 1, o.ld, Vw, 1, o.nrows, 0.0, AX, ld,
                         c->stream);
}

// ---------------------------------------------------------------- sqrt quadrature
// Complete elliptic integral of the first kind K(m) = pi / (2 AGM(1, sqrt(1 - m))),
// 0 <= m < 1 (arithmetic-geometric mean).
double ellip_k(double m) {
  double a = 1.0, b = std::sqrt(1.0 - m);
  for (int it = 0; it < 64 && std::fabs(a - b) > 1e-16 * a; ++it) {
    const double an = 0.5 * (a + b);
    b = std::sqrt(a * b);
    a = an;
  }
  return 3.14159265358979323846 / (2.0 * a);
}

// Jacobi elliptic functions sn, cn, dn of parameter m by the arithmetic-geometric mean
// scale and descending recursion of Abramowitz & Stegun 16.4: a_0 = 1, b_0 = sqrt(1-m),
// c_0 = sqrt(m); phi_N = 2^N a_N u; phi_{n-1} = (phi_n + asin(c_n sin(phi_n) / a_n)) / 2;
// sn = sin phi_0, cn = cos phi_0, dn = cos phi_0 / cos(phi_1 - phi_0).
void ellip_j(double u, double m, double* sn, double* cn, double* dn) {
  if (m < 1e-300) {
    *sn = std::sin(u);
    *cn = std::cos(u);
    *dn = 1.0;
    return;
  }
  double a[64], c[64];
  a[0] = 1.0;
  double b = std::sqrt(1.0 - m);
  c[0] = std::sqrt(m);
  int n = 0;
  while (n < 62 && std::fabs(c[n]) > 1e-17) {
    a[n + 1] = 0.5 * (a[n] + b);
    c[n + 1] = 0.5 * (a[n] - b);
    b = std::sqrt(a[n] * b);
    ++n;
  }
  double phi = std::ldexp(a[n] * u, n);
  double prev = phi;
  for (int j = n; j > 0; --j) {
    prev = phi;
    phi = 0.5 * (phi + std::asin(c[j] * std::sin(phi) / a[j]));
  }
  *sn = std::sin(phi);
  *cn = std::cos(phi);
  *dn = (n > 0) ? std::cos(phi) / std::cos(prev - phi) : 1.0;
}

// Nodes and weights of (2/pi) int_0^inf lambda / (lambda + z^2) dz = sqrt(lambda) for
// lambda in [lo, hi]: the substitution z = sqrt(lo) sc(u | 1 - lo/hi) maps [0, inf) to
// [0, K] and turns dz / sqrt((lo + z^2)(hi + z^2)) into du / sqrt(hi) (the identity of
// Eq. ellipticK_eval); the midpoint rule in u then converges geometrically for every
// lambda in [lo, hi]. Returns z_j^2 and (2/pi) w_j.
void sqrt_quadrature(double lo, double hi, int N, double* z2, double* w) {
  const double m = 1.0 - lo / hi;
  const double K = ellip_k(m);
  for (int j = 0; j < N; ++j) {
    const double u = (j + 0.5) * K / N;
    double sn, cn, dn;
    ellip_j(u, m, &sn, &cn, &dn);
    const double z = std::sqrt(lo) * sn / cn;
    z2[j] = z * z;
    w[j] = (2.0 / 3.14159265358979323846) * (K / N) * std::sqrt(lo) * dn / (cn * cn);
  }
}

}  // namespace

extern "C" bk_status bk_sqrt_quadrature(double lo, double hi, int32_t n, double* z2, double* w) {
  if (!z2 || !w || n < 1 || !(lo > 0.0) || !(hi >= lo) || !std::isfinite(hi)) return BK_ERR_ARG;
  sqrt_quadrature(lo, hi, n, z2, w);
  return BK_OK;
}

extern "C" bk_status bk_ridge_path(bk_ctx* c, const bk_operator* A, int32_t L, const double* mus, const double* b,
                                   double* X, const bk_opts* opts_in, bk_info* info) {
  if (info) std::memset(info, 0, sizeof(*info));
  if (!c || !b || !X || !mus || L < 1 || L > 1024) return BK_ERR_ARG;
  err_ctx() = c;
  c->last_error[0] = 0;
  LzOp o;
  bk_status s = check_lz_operator(A, &o);
  if (s != BK_OK) return s;
  bk_opts opts;
  if (opts_in)
    opts = *opts_in;
  else
    bk_default_opts(&opts);
  if (!(opts.tol > 0.0) || opts.sketch < 0 || opts.max_loads < 1 || opts.max_refine < 1) return BK_ERR_ARG;
  if (opts.inner != BK_PREC_FP64 && opts.inner != BK_PREC_FP32 && opts.inner != BK_PREC_F32X2 &&
      opts.inner != BK_PREC_BF16)
    return BK_ERR_UNSUPPORTED;
  if (o.kind == BK_RBF && opts.inner == BK_PREC_FP32) return BK_ERR_UNSUPPORTED;
  const bool bf16 = opts.inner == BK_PREC_BF16;
  if (bf16 && (o.kind != BK_GRAM || !bk::bf16_gram_usable(o.nrows, o.d, (int)std::min<int64_t>(
                                                                   std::max<int64_t>(L, (int64_t)opts.sketch + 1), o.d))))
    return BK_ERR_UNSUPPORTED;
  std::vector<double> hmu(L);
  BK_CK(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  // shifts to the host (validation) and the device
  BK_CK(cudaMemcpy(hmu.data(), mus, (size_t)L * 8, cudaMemcpyDefault));
  for (double v : hmu)
    if (!(v >= 0.0) || !std::isfinite(v)) return BK_ERR_ARG;
  const int is64 = opts.inner != BK_PREC_FP32 && !bf16;
  const int64_t d = o.d;
  const int m = (int)std::min<int64_t>((int64_t)opts.sketch + 1, d);
  Prof prof;
  prof.on = opts.profile != 0;
  prof.st = st;
  if (m > 256) return BK_ERR_UNSUPPORTED;
  cudaEvent_t ev0, ev1;
  BK_CK(cudaEventCreate(&ev0));
  BK_CK(cudaEventCreate(&ev1));
  BK_CK(cudaEventRecord(ev0, st));

  const void* staged = nullptr;
  LzOp o64 = o;  // refinement residuals use the values as given
  BK_CK(stage_lz_values(c, A, &o, is64, &staged));
  o64.vals = staged;
  // BF16 loads: head/tail copies of Z (row-major and transposed), made once per call
  void *bzc = nullptr, *bzw = nullptr;
  size_t bzw_bytes = 0;
  int* bzerr = nullptr;
  if (bf16) {
    const int nmax = (int)std::min<int64_t>(std::max<int64_t>(L, m), d);
    BK_CK(ws_get(c, WS_BF16, bk::bf16_gram_copy_bytes(o.nrows, d), &bzc));
    bzw_bytes = bk::bf16_gram_work_bytes(o.nrows, d, nmax, c->sms);
    BK_CK(ws_get(c, WS_BF16W, bzw_bytes + 256, &bzw));
    bzerr = (int*)((char*)bzw + bzw_bytes);
    BK_CK(cudaMemsetAsync(bzerr, 0, sizeof(int), st));
    BK_CK(bk::launch_bf16_gram_split(o.nrows, d, (const float*)o.vals, o.ld, bzc, st));
  }
  // BF16 runs also take their FP64-accurate residual products to the tensor cores: the
  // Ozaki-split digits of the stored Z and Z^T, made once per call
  void *ozz = nullptr, *ozw = nullptr;
  int* ozerr = nullptr;
  if (bf16 && o64.kind == BK_GRAM && bk::ozaki_gram_usable(o64.nrows, d, L)) {
    const size_t wb = bk::ozaki_gram_work_bytes(o64.nrows, d, L, c->sms);
    BK_CK(ws_get(c, WS_OZ_A, bk::ozaki_gram_bytes(o64.nrows, d), &ozz));
    BK_CK(ws_get(c, WS_OZ_X, wb + 256, &ozw));
    ozerr = (int*)((char*)ozw + wb);
    BK_CK(cudaMemsetAsync(ozerr, 0, sizeof(int), st));
    BK_CK(bk::launch_ozaki_split_gram(o64.nrows, d, o64.vals_f64, o64.vals, o64.ld, ozz, c->sms, st));
  }
  const double* bd = nullptr;
  BK_CK(stage_in(c, WS_B64, b, (size_t)d * 8, (const void**)&bd));
  double* dmu = nullptr;
  BK_CK(ws_get(c, WS_LSHIFT, (size_t)L * 8 + 4096, (void**)&dmu));
  BK_CK(cudaMemcpyAsync(dmu, hmu.data(), (size_t)L * 8, cudaMemcpyHostToDevice, st));
  int* rhs_col = (int*)(dmu + L);
  int* flags = rhs_col + 1024;

  const int64_t ldx = d;
  double *Xd = nullptr, *AX = nullptr, *Rres = nullptr, *norms = nullptr, *Vw = nullptr, *B0 = nullptr;
  BK_CK(ws_get(c, WS_LX, (size_t)ldx * L * 8, (void**)&Xd));
  BK_CK(ws_get(c, WS_LAX, (size_t)ldx * L * 8, (void**)&AX));
  BK_CK(ws_get(c, WS_LRES, (size_t)ldx * L * 8 + (size_t)L * 8 * 4, (void**)&Rres));
  norms = Rres + (size_t)ldx * L;
  if (o.kind == BK_GRAM) BK_CK(ws_get(c, WS_LB64, (size_t)o.nrows * L * 8, (void**)&Vw));
  BK_CK(cudaMemsetAsync(Xd, 0, (size_t)ldx * L * 8, st));

  // ||b||
  int nnp = bk::residual_parts(d);
  double* normp = nullptr;
  BK_CK(ws_get(c, WS_NORMP, kHostParts * 8, (void**)&normp));
  BK_CK(bk::launch_norm2_parts(d, bd, normp, nnp, st));
  double bn2 = 0.0;
  BK_CK(host_sum(c, normp, nnp, &bn2));
  const double bnorm = std::sqrt(bn2);

  int loads = 0, residual_loads = 0, refinements = 0;
  bk_status result = BK_NOT_CONVERGED;
  double worst = 1.0;
  // compensated FP32 residual products allowed (not on the plain FP64 path) and still
  // accurate enough
  bool df_ok = opts.inner != BK_PREC_FP64;
  int skipped_shifts = 0;  // shifted solves that failed (reported through last_error)
  bool escalated = false;  // FP32 run moved to FP64 bases
  if (bnorm == 0.0) {
    result = BK_OK;
    worst = 0.0;
  }
  const int tmax_cap = (int)std::min<int64_t>((d + m - 1) / m + 1, opts.max_loads);

  // Each pass runs a block-Lanczos basis on a start block and adds the shifted
  // solutions: pass 0 on [b/||b||, Omega/sqrt(d)] (column 0 feeds every shift), later
  // passes on the FP64 residual block [r_1 .. r_L] (column j feeds shift j).
  for (int pass = 0; result != BK_OK && pass < opts.max_refine; ++pass) {
    const int mb = pass == 0 ? m : (int)std::min<int64_t>(L, d);
    const int tmax = (int)std::min<int64_t>((d + mb - 1) / mb + 1, std::max(1, opts.max_loads - loads));
    // basis precision of this pass: FP32 runs escalate to FP64 blocks with FP64-accurate
    // products once an FP32 basis has produced indefinite shifted systems (its rounding,
    // about u ||A||, reached the smallest shifted eigenvalues)
    const int pis64 = is64 || escalated;
    Lanczos lz;
    LzOp ol = o;
    BK_CK(lz.init(c, ol, pis64, mb, tmax));
    lz.prof = &prof;
    lz.df = opts.inner == BK_PREC_F32X2 || escalated;
    if (bf16 && !pis64) {
      lz.bz = bzc;
      lz.bwork = bzw;
      lz.bwork_bytes = bzw_bytes;
      lz.berr = bzerr;
    }
    bool pass_flagged = false;
    // start block into W (block precision), column scales applied in FP64 first
    double* B0d = nullptr;
    BK_CK(ws_get(c, WS_LB0, (size_t)d * std::max(mb, 1) * 8 + 4096 * 8, (void**)&B0d));
    double* scales = B0d + (size_t)d * mb;
    std::vector<double> hs(mb);
    if (pass == 0) {
      BK_CK(cudaMemcpyAsync(B0d, bd, (size_t)d * 8, cudaMemcpyDeviceToDevice, st));
      if (mb > 1) BK_CK(bk::launch_gaussian(opts.seed, 3u, d * (int64_t)(mb - 1), 0, B0d + d, st));
      hs[0] = 1.0 / bnorm;
      for (int q = 1; q < mb; ++q) hs[q] = 1.0 / std::sqrt((double)d);
    } else {
      BK_CK(cudaMemcpyAsync(B0d, Rres, (size_t)d * mb * 8, cudaMemcpyDeviceToDevice, st));
      for (int q = 0; q < mb; ++q) hs[q] = 1.0;
    }
    BK_CK(cudaMemcpyAsync(scales, hs.data(), (size_t)mb * 8, cudaMemcpyHostToDevice, st));
    BK_CK(bk::launch_scale_cols(1, d, mb, d, scales, B0d, st));
    BK_CK(bk::launch_copy_cols(1, pis64, d, mb, B0d, d, lz.W, lz.ldq, st));
    BK_CK(lz.start(lz.W));
    // right-hand sides of the projected systems: columns of E_1 R_0 (R_0 row-major)
    double* rhs = nullptr;
    BK_CK(ws_get(c, WS_LRHS, (size_t)lz.ncol_max * mb * 8, (void**)&rhs));
    std::vector<int> hcol(L);
    for (int j = 0; j < L; ++j) hcol[j] = pass == 0 ? 0 : j;
    BK_CK(cudaMemcpyAsync(rhs_col, hcol.data(), (size_t)L * 4, cudaMemcpyHostToDevice, st));
    double *bwork = nullptr, *Z = nullptr;
    const int bw = mb;
    BK_CK(ws_get(c, WS_LBWORK, (size_t)L * (bw + 2) * lz.ncol_max * 8, (void**)&bwork));
    BK_CK(ws_get(c, WS_LZ, (size_t)L * lz.ncol_max * 8, (void**)&Z));
    // pass 0 works on the unit column b / ||b||; later passes on the raw residuals
    const double target = pass == 0 ? std::max(opts.inner_tol, 0.25 * opts.tol) : 0.25 * opts.tol * bnorm;
    int done = 0;
    std::vector<double> hres(L);
    while (!done) {
      BK_CK(lz.step());
      const int n = lz.n();
      const bool last = lz.t >= tmax || n >= d;
      if (!last && (lz.t % opts.check_every) != 0) continue;
      // right-hand sides E_1 R_0 of the projected systems (n x mb, leading dimension n)
      BK_CK(bk::launch_e1r0(n, mb, lz.R0, rhs, st));
      BK_CK(bk::launch_band_solve(n, bw, lz.band, lz.ldb(), L, dmu, rhs, rhs_col, 1, bwork, Z, flags, st));
      // residual estimate ||B_t z_last|| for every shift
      BK_CK(bk::launch_lanczos_res(n, mb, L, 1, lz.Bk, Z, norms, st));
      BK_CK(cudaMemcpyAsync(c->hparts, norms, (size_t)L * 8, cudaMemcpyDeviceToHost, st));
      BK_CK(cudaStreamSynchronize(st));
      double est = 0.0;
      for (int j = 0; j < L; ++j) est = std::max(est, c->hparts[j]);
      int* hf = (int*)c->hparts;
      BK_CK(cudaMemcpyAsync(hf, flags, (size_t)L * 4, cudaMemcpyDeviceToHost, st));
      BK_CK(cudaStreamSynchronize(st));
      // T_t + mu_j I not positive definite: only possible through rounding in the basis
      // (A + mu_j I is positive definite for mu_j > 0); the solve dropped the offending
      // directions and the FP64 residual of that shift drives the next basis
      for (int j = 0; j < L; ++j)
        if (hf[j]) {
          ++skipped_shifts;
          pass_flagged = true;
        }
      if (est <= target || last) done = 1;
    }
    loads += lz.loads;
    // X += Q_t Z (pass 0 scaled back by ||b||: the start column was b / ||b||)
    const int n = lz.n();
    BK_CK(lz.gemm_k(1, d, L, n, pass == 0 ? bnorm : 1.0, lz.Q, pis64, 1, lz.ldq, Z, 1, n, 1.0, Xd, ldx));
    ++refinements;
    if (pass_flagged && !pis64) escalated = true;
    // FP64 residuals of every shift. The compensated FP32 products carry about 44 bits:
    // their error in b - A_mu x is about 1e-13 ||A|| ||X|| (cancellation when x is
    // large). Use them only while that floor is below tol / 10 (||A|| <= the
    // Gershgorin bound of T_t, ||X|| <= its Frobenius norm), and take the FP64 GEMM
    // once a pass stops reducing the residual.
    if (df_ok && !o64.vals_f64) {
      double xn2 = 0.0;
      const int npx = bk::residual_parts(d * L);
      BK_CK(bk::launch_norm2_parts(d * L, Xd, normp, npx, st));
      BK_CK(host_sum(c, normp, npx, &xn2));
      BK_CK(bk::launch_band_gersh(n, mb, lz.band, lz.ldb(), norms, st));
      BK_CK(cudaMemcpyAsync(c->hparts, norms, 8, cudaMemcpyDeviceToHost, st));
      BK_CK(cudaStreamSynchronize(st));
      if (1e-13 * c->hparts[0] * std::sqrt(xn2) > 0.1 * opts.tol * bnorm) df_ok = false;
    }
    const double prev_worst = worst;
    for (int attempt = 0; attempt < 2; ++attempt) {
      prof.begin();
      if (ozz && df_ok)
        BK_CK(bk::launch_ozaki_gram_apply(o64.nrows, d, L, ozz, Xd, ldx, AX, ldx, ozw, 0, ozerr, c->sms, st));
      else
        BK_CK(apply_fp64(c, o64, Xd, ldx, L, AX, Vw, df_ok));
      prof.end(BK_K_RESIDUAL);
      BK_CK(bk::launch_shift_residual(d, L, bd, AX, Xd, ldx, dmu, Rres, norms, st));
      residual_loads += 1;
      BK_CK(cudaMemcpyAsync(c->hparts, norms, (size_t)L * 8, cudaMemcpyDeviceToHost, st));
      BK_CK(cudaStreamSynchronize(st));
      worst = 0.0;
      for (int j = 0; j < L; ++j) worst = std::max(worst, std::sqrt(c->hparts[j]) / bnorm);
      const bool stalled = pass > 0 && worst > 0.25 * prev_worst && worst > opts.tol;
      if (!(df_ok && !o64.vals_f64 && stalled)) break;
      df_ok = false;  // recompute this residual in FP64
    }
    if (worst <= opts.tol) result = BK_OK;
  }
  if (ozerr) {  // an Ozaki-split residual product whose pipeline wait gave up
    int herr = 0;
    BK_CK(cudaMemcpyAsync(c->hparts, ozerr, sizeof(int), cudaMemcpyDeviceToHost, st));
    BK_CK(cudaStreamSynchronize(st));
    std::memcpy(&herr, c->hparts, sizeof(int));
    if (herr) {
      std::snprintf(c->last_error, sizeof(c->last_error), "tensor-core pipeline wait timed out");
      result = BK_TIMEOUT;
    }
  }
  if (bzerr) {  // a BF16 product whose pipeline wait gave up left an invalid load
    BK_CK(cudaMemcpyAsync(c->hparts, bzerr, sizeof(int), cudaMemcpyDeviceToHost, st));
    BK_CK(cudaStreamSynchronize(st));
    int herr = 0;
    std::memcpy(&herr, c->hparts, sizeof(int));
    if (herr) {
      result = BK_TIMEOUT;
      std::snprintf(c->last_error, sizeof(c->last_error), "tensor-core pipeline wait timed out");
    }
  }
  BK_CK(cudaMemcpyAsync(X, Xd, (size_t)d * L * 8, cudaMemcpyDefault, st));
  BK_CK(cudaEventRecord(ev1, st));
  BK_CK(cudaEventSynchronize(ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (info) {
    info->status = result;
    info->loads = loads;
    info->refinements = refinements;
    info->residual_loads = residual_loads;
    info->rel_residual = worst;
    info->ms_total = ms;
  }
  if (skipped_shifts && result != BK_OK)
    std::snprintf(c->last_error, sizeof(c->last_error), "%d shifted projected solves dropped non-positive pivots",
                  skipped_shifts);
  prof.report(info);
  return result;
}

namespace {

// bk_sample (inverse = false: (K + nugget I)^{1/2} B) and bk_sample_isqrt (inverse =
// true: (K + nugget I)^{-1/2} B) share the basis, the shifts and the weights: with
// Ybar = sum_j w_j (T_t + (nugget + z_j^2) I)^{-1} E_1 R_0, the square root is
// Q_t (T_t + nugget) Ybar + Q_{t+1} B_t E_t^T Ybar (Def. blansq) and the inverse square
// root Q_t Ybar (the integrand without the factor A).
bk_status sample_driver(bk_ctx* c, const bk_operator* Kop, double nugget, int32_t m, const double* B, double* S,
                        int32_t n_quad, const bk_opts* opts_in, bk_info* info, bool inverse) {
  if (info) std::memset(info, 0, sizeof(*info));
  if (!c || !B || !S || m < 1 || m > 256 || n_quad < 1 || n_quad > 1024 || !(nugget >= 0.0) ||
      !std::isfinite(nugget))
    return BK_ERR_ARG;
  err_ctx() = c;
  c->last_error[0] = 0;
  LzOp o;
  bk_status s = check_lz_operator(Kop, &o);
  if (s != BK_OK) return s;
  bk_opts opts;
  if (opts_in)
    opts = *opts_in;
  else
    bk_default_opts(&opts);
  if (!(opts.tol > 0.0) || opts.max_loads < 1 || opts.check_every < 1) return BK_ERR_ARG;
  if (opts.inner != BK_PREC_FP64 && opts.inner != BK_PREC_FP32 && opts.inner != BK_PREC_F32X2 &&
      opts.inner != BK_PREC_OZAKI)
    return BK_ERR_UNSUPPORTED;
  const int is64 = opts.inner != BK_PREC_FP32;
  const bool oz = opts.inner == BK_PREC_OZAKI;
  const int64_t d = o.d;
  if (m > d) return BK_ERR_ARG;
  if (o.kind == BK_RBF && !is64) return BK_ERR_UNSUPPORTED;
  // the Ozaki split is built for stored dense FP32 operators
  if (oz && (o.kind != BK_DENSE || Kop->dtype != BK_F32 || !bk::ozaki_usable(d, m))) return BK_ERR_UNSUPPORTED;
  BK_CK(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  cudaEvent_t ev0, ev1;
  BK_CK(cudaEventCreate(&ev0));
  BK_CK(cudaEventCreate(&ev1));
  BK_CK(cudaEventRecord(ev0, st));
  const void* staged = nullptr;
  BK_CK(stage_lz_values(c, Kop, &o, is64, &staged));
  const double* Bd = nullptr;
  BK_CK(stage_in(c, WS_B64, B, (size_t)d * m * 8, (const void**)&Bd));

  const int tmax = (int)std::min<int64_t>((d + m - 1) / m + 1, opts.max_loads);
  Prof prof;
  prof.on = opts.profile != 0;
  prof.st = st;
  Lanczos lz;
  BK_CK(lz.init(c, o, is64, m, tmax));
  lz.prof = &prof;
  lz.df = opts.inner == BK_PREC_F32X2 || oz;
  int* ozerr = nullptr;
  if (oz) {  // digits of K once per call; the loads then run on the tensor cores
    void *oza = nullptr, *ozx = nullptr;
    BK_CK(ws_get(c, WS_OZ_A, bk::ozaki_a_bytes(d), &oza));
    BK_CK(ws_get(c, WS_OZ_X, bk::ozaki_x_bytes(d, m, c->sms) + 256, &ozx));
    ozerr = (int*)((char*)ozx + bk::ozaki_x_bytes(d, m, c->sms));
    BK_CK(cudaMemsetAsync(ozerr, 0, sizeof(int), st));
    BK_CK(bk::launch_ozaki_split_a(d, (const float*)o.vals, o.ld, oza, c->sms, st));
    lz.oza = oza;
    lz.ozx = ozx;
    lz.ozerr = ozerr;
    lz.ozb = true;
  }
  BK_CK(bk::launch_copy_cols(1, is64, d, m, Bd, d, lz.W, lz.ldq, st));
  BK_CK(lz.start(lz.W));

  const int N = n_quad;
  double *dmu = nullptr, *rhs = nullptr, *bwork = nullptr, *Z = nullptr, *Ybar = nullptr, *M1 = nullptr;
  double *Sd = nullptr, *Sprev = nullptr, *small = nullptr;
  BK_CK(ws_get(c, WS_LSHIFT, (size_t)N * 8 * 2 + 8192, (void**)&dmu));
  double* dw = dmu + N;
  int* rhs_col = (int*)(dw + N);
  int* flags = rhs_col + 1024;
  BK_CK(cudaMemsetAsync(rhs_col, 0, (size_t)N * 4, st));
  const int64_t nmax = lz.ncol_max;
  BK_CK(ws_get(c, WS_LRHS, (size_t)nmax * m * 8 * 3 + (size_t)m * m * 8, (void**)&rhs));
  Ybar = rhs + (size_t)nmax * m;
  M1 = Ybar + (size_t)nmax * m;
  small = M1 + (size_t)nmax * m;
  BK_CK(ws_get(c, WS_LBWORK, (size_t)N * (m + 2) * nmax * 8, (void**)&bwork));
  BK_CK(ws_get(c, WS_LZ, (size_t)N * nmax * m * 8, (void**)&Z));
  BK_CK(ws_get(c, WS_LX, (size_t)d * m * 8, (void**)&Sd));
  BK_CK(ws_get(c, WS_LAX, (size_t)d * m * 8, (void**)&Sprev));
  double* normp = nullptr;
  BK_CK(ws_get(c, WS_NORMP, kHostParts * 8, (void**)&normp));
  std::vector<double> hz2(N), hw(N), hmu(N);

  bk_status result = BK_NOT_CONVERGED;
  double change = 1.0;
  int checks = 0;
  for (;;) {
    BK_CK(lz.step());
    const int n = lz.n();
    const bool last = lz.t >= tmax || n >= d;
    if (!last && (lz.t % opts.check_every) != 0) continue;
    // spectrum interval of A = K + nugget I: [nugget, Gershgorin bound of T_t + nugget]
    BK_CK(bk::launch_band_gersh(n, m, lz.band, lz.ldb(), small, st));
    BK_CK(cudaMemcpyAsync(c->hparts, small, 8, cudaMemcpyDeviceToHost, st));
    BK_CK(cudaStreamSynchronize(st));
    const double hi = c->hparts[0] + nugget;
    const double lo = nugget > 0.0 ? nugget : 1e-12 * hi;
    sqrt_quadrature(lo, std::max(hi, lo), N, hz2.data(), hw.data());
    for (int j = 0; j < N; ++j) hmu[j] = nugget + hz2[j];
    BK_CK(cudaMemcpyAsync(dmu, hmu.data(), (size_t)N * 8, cudaMemcpyHostToDevice, st));
    BK_CK(cudaMemcpyAsync(dw, hw.data(), (size_t)N * 8, cudaMemcpyHostToDevice, st));
    // Y_j = (T_K + (nugget + z_j^2) I)^{-1} E_1 R_0 for all j in one launch
    BK_CK(bk::launch_e1r0(n, m, lz.R0, rhs, st));
    BK_CK(bk::launch_band_solve(n, m, lz.band, lz.ldb(), N, dmu, rhs, rhs_col, m, bwork, Z, flags, st));
    {
      // a shifted T_t that is not positive definite (A indefinite in the stored
      // precision) leaves that shift's solve unfinished: stop with BK_BREAKDOWN
      int* hf = (int*)c->hparts;
      BK_CK(cudaMemcpyAsync(hf, flags, (size_t)N * 4, cudaMemcpyDeviceToHost, st));
      BK_CK(cudaStreamSynchronize(st));
      bool bad = false;
      for (int j = 0; j < N; ++j) bad = bad || hf[j] != 0;
      if (bad) {
        result = BK_BREAKDOWN;
        break;
      }
    }
    // Ybar = sum_j w_j Y_j; S = Q_t (T_t + nugget) Ybar + Q_{t+1} B_t E_t^T Ybar
    BK_CK(bk::launch_combine_shifts(n, m, N, Z, dw, Ybar, st));
    // the basis products of the combination (d x m from the d x n basis) go through the
    // Ozaki split in Ozaki runs, FP64 GEMMs otherwise
    auto basis_gemm = [&](int64_t M_, int64_t N_, int64_t K_, const void* A_, int64_t sai, int64_t sak,
                          const double* B_, int64_t sbk, int64_t sbj, double beta_, double* C_,
                          int64_t ldc_) -> cudaError_t {
      if (oz) return lz.gemm_k(1, M_, N_, K_, 1.0, A_, is64, sai, sak, B_, sbk, sbj, beta_, C_, ldc_, false);
      return bk::launch_gemm(1, M_, N_, K_, 1.0, A_, is64, sai, sak, B_, sbk, sbj, beta_, C_, ldc_, st);
    };
    if (inverse) {
      BK_CK(basis_gemm(d, m, n, lz.Q, 1, lz.ldq, Ybar, 1, n, 0.0, Sd, d));
    } else {
      BK_CK(bk::launch_band_mult(n, m, lz.band, lz.ldb(), nugget, Ybar, m, M1, st));
      BK_CK(basis_gemm(d, m, n, lz.Q, 1, lz.ldq, M1, 1, n, 0.0, Sd, d));
      // small = B_t (rows n-m.. of Ybar): B_t row-major m x m, Ybar rows n-m..n-1 (ld n)
      BK_CK(bk::launch_gemm(1, m, m, m, 1.0, lz.Bk, 1, m, 1, Ybar + (n - m), 1, n, 0.0, small, m, st));
      BK_CK(basis_gemm(d, m, m, lz.qblock(lz.t), 1, lz.ldq, small, 1, m, 1.0, Sd, d));
    }
    // relative change against the previous check (a-posteriori stopping, Sec. 4 remark)
    int np = bk::residual_parts(d * m);
    double s2 = 0.0, d2 = 0.0;
    BK_CK(bk::launch_norm2_parts(d * m, Sd, normp, np, st));
    BK_CK(host_sum(c, normp, np, &s2));
    if (checks > 0) {
      BK_CK(bk::launch_axpy(d * m, -1.0, Sd, Sprev, st));
      BK_CK(bk::launch_norm2_parts(d * m, Sprev, normp, np, st));
      BK_CK(host_sum(c, normp, np, &d2));
      change = std::sqrt(d2 / std::max(s2, 1e-300));
    }
    ++checks;
    BK_CK(cudaMemcpyAsync(Sprev, Sd, (size_t)d * m * 8, cudaMemcpyDeviceToDevice, st));
    if ((checks > 1 && change <= opts.tol) || n >= d) {
      result = BK_OK;
      break;
    }
    if (last) break;
  }
  BK_CK(cudaMemcpyAsync(S, Sd, (size_t)d * m * 8, cudaMemcpyDefault, st));
  if (ozerr) {  // a tensor-core load whose pipeline wait gave up left an invalid block
    int herr = 0;
    BK_CK(cudaMemcpyAsync(c->hparts, ozerr, sizeof(int), cudaMemcpyDeviceToHost, st));
    BK_CK(cudaStreamSynchronize(st));
    std::memcpy(&herr, c->hparts, sizeof(int));
    if (herr) {
      std::snprintf(c->last_error, sizeof(c->last_error), "tensor-core pipeline wait timed out");
      result = BK_TIMEOUT;
    }
  }
  BK_CK(cudaEventRecord(ev1, st));
  BK_CK(cudaEventSynchronize(ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (info) {
    info->status = result;
    info->loads = lz.loads;
    info->refinements = checks;
    info->rel_residual = change;
    info->ms_total = ms;
  }
  prof.report(info);
  return result;
}

}  // namespace

extern "C" bk_status bk_sample(bk_ctx* c, const bk_operator* Kop, double nugget, int32_t m, const double* B,
                               double* S, int32_t n_quad, const bk_opts* opts_in, bk_info* info) {
  return sample_driver(c, Kop, nugget, m, B, S, n_quad, opts_in, info, false);
}

extern "C" bk_status bk_sample_isqrt(bk_ctx* c, const bk_operator* Kop, double nugget, int32_t m, const double* B,
                                     double* S, int32_t n_quad, const bk_opts* opts_in, bk_info* info) {
  return sample_driver(c, Kop, nugget, m, B, S, n_quad, opts_in, info, true);
}

// ---------------------------------------------------------------- Nystrom PCG
namespace {

// Eigen-decomposition of a symmetric n x n matrix (row-major, overwritten) by cyclic
// Jacobi rotations (Golub & Van Loan, Sec. 8.5: sym.schur2 and cyclic sweeps):
// eigenvalues ascending in w, eigenvectors as the columns of V (row-major n x n).
void jacobi_eigh(int n, std::vector<double>& A, std::vector<double>& w, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  double fro = 0.0;
  for (double a : A) fro += a * a;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
    if (off <= 1e-32 * fro || off == 0.0) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double tau = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = t * cs;
        for (int k = 0; k < n; ++k) {  // A J
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = cs * akp - sn * akq;
          A[(size_t)k * n + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < n; ++k) {  // J^T A
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = cs * apk - sn * aqk;
          A[(size_t)q * n + k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < n; ++k) {  // V J
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = cs * vkp - sn * vkq;
          V[(size_t)k * n + q] = sn * vkp + cs * vkq;
        }
      }
  }
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return A[(size_t)a * n + a] < A[(size_t)b * n + b]; });
  w.resize(n);
  std::vector<double> Vs((size_t)n * n);
  for (int j = 0; j < n; ++j) {
    w[j] = A[(size_t)ord[j] * n + ord[j]];
    for (int k = 0; k < n; ++k) Vs[(size_t)k * n + j] = V[(size_t)k * n + ord[j]];
  }
  V.swap(Vs);
}

bk_status check_pcg_operator(const bk_operator* A, LzOp* o) {
  if (A && A->kind == BK_CSR) {
    if (!A->vals || !A->rowptr || !A->colidx || A->rows <= 0 || A->rows != A->cols || A->nnz < 0) return BK_ERR_ARG;
    if (A->dtype != BK_F64 && A->dtype != BK_F32) return BK_ERR_UNSUPPORTED;
    o->kind = BK_CSR;
    o->d = A->rows;
    o->nnz = A->nnz;
    o->vals_f64 = A->dtype == BK_F64;
    return BK_OK;
  }
  return check_lz_operator(A, o);
}

cudaError_t stage_pcg_operator(bk_ctx* c, const bk_operator* A, LzOp* o) {
  if (o->kind != BK_CSR) {
    const void* staged = nullptr;
    return stage_lz_values(c, A, o, 1, &staged);
  }
  const void *rp = nullptr, *ci = nullptr, *va = nullptr;
  cudaError_t e = stage_in(c, WS_OP_ROW, A->rowptr, (size_t)(o->d + 1) * 4, &rp);
  if (e != cudaSuccess) return e;
  if ((e = stage_in(c, WS_OP_COL, A->colidx, (size_t)std::max<int64_t>(o->nnz, 1) * 4, &ci)) != cudaSuccess) return e;
  if ((e = stage_in(c, WS_OP_VALS, A->vals, (size_t)std::max<int64_t>(o->nnz, 1) * (o->vals_f64 ? 8 : 4), &va)) !=
      cudaSuccess)
    return e;
  o->rowptr = (const int*)rp;
  o->colidx = (const int*)ci;
  o->vals = va;
  return cudaSuccess;
}

}  // namespace

extern "C" bk_status bk_nystrom_pcg(bk_ctx* c, const bk_operator* A, double mu, const double* b, double* x,
                                    int32_t s_ny, const bk_opts* opts_in, bk_info* info) {
  if (info) std::memset(info, 0, sizeof(*info));
  if (!c || !b || !x || s_ny < 1 || s_ny > 16 || !(mu >= 0.0) || !std::isfinite(mu)) return BK_ERR_ARG;
  err_ctx() = c;
  c->last_error[0] = 0;
  LzOp o;
  bk_status s = check_pcg_operator(A, &o);
  if (s != BK_OK) return s;
  bk_opts opts;
  if (opts_in)
    opts = *opts_in;
  else
    bk_default_opts(&opts);
  if (!(opts.tol > 0.0) || opts.sketch < 1 || opts.max_loads < 1 || opts.check_every < 1) return BK_ERR_ARG;
  const int64_t d = o.d;
  const int l = (int)std::min<int64_t>(opts.sketch, d);
  if (l > 256) return BK_ERR_UNSUPPORTED;
  BK_CK(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  cudaEvent_t ev0, ev1;
  BK_CK(cudaEventCreate(&ev0));
  BK_CK(cudaEventCreate(&ev1));
  BK_CK(cudaEventRecord(ev0, st));
  BK_CK(stage_pcg_operator(c, A, &o));
  const double* bd = nullptr;
  BK_CK(stage_in(c, WS_B64, b, (size_t)d * 8, (const void**)&bd));

  // --- Nystrom approximation of depth s (Eq. nystromBKI_def) from s block-Lanczos
  // steps on Omega: V = [Q_0 .. Q_{s-1}] spans K_s(A, Omega), and the Lanczos relation
  // A V = V T_s + Q_s B E_s^T gives Y = A V = [V Q_s] [T_s; B E_s^T] without another
  // load. With T_s = W diag(lam) W^T (numerically nonzero part), F = Y W lam^{-1/2}
  // satisfies F F^T = Y (V^T Y)^+ Y^T = A<K_s>, and F = [V Q_s] H with
  // H = [W lam^{1/2}; B E_s^T W lam^{-1/2}]; H^T H = G sig^2 G^T then gives
  // U = [V Q_s] H G sig^{-1} and D = sig^2.
  Lanczos lz;
  const int tmax = s_ny;
  BK_CK(lz.init(c, o, 1, l, tmax));
  double* Om = nullptr;
  BK_CK(ws_get(c, WS_LB0, (size_t)d * l * 8 + 4096 * 8, (void**)&Om));
  BK_CK(bk::launch_gaussian(opts.seed, 3u, d * (int64_t)l, 0, Om, st));
  BK_CK(bk::launch_copy_cols(1, 1, d, l, Om, d, lz.W, lz.ldq, st));
  BK_CK(lz.start(lz.W));
  for (int k = 0; k < s_ny; ++k) BK_CK(lz.step());
  const int n = lz.n();  // s l
  const int nb = n + l;  // columns of [V Q_s]
  std::vector<double> hband((size_t)(l + 1) * lz.ldb()), hB((size_t)l * l);
  BK_CK(cudaMemcpyAsync(hband.data(), lz.band, hband.size() * 8, cudaMemcpyDeviceToHost, st));
  BK_CK(cudaMemcpyAsync(hB.data(), lz.Bk, hB.size() * 8, cudaMemcpyDeviceToHost, st));
  BK_CK(cudaStreamSynchronize(st));
  std::vector<double> T((size_t)n * n, 0.0);
  for (int col = 0; col < n; ++col)
    for (int r = 0; r <= l && col + r < n; ++r) {
      const double v = hband[(size_t)r * lz.ldb() + col];
      T[(size_t)(col + r) * n + col] = v;
      T[(size_t)col * n + col + r] = v;
    }
  std::vector<double> lam, W;
  jacobi_eigh(n, T, lam, W);
  const double lmax = lam.empty() ? 0.0 : lam.back();
  std::vector<int> keep;
  for (int i = 0; i < n; ++i)
    if (lam[i] > 1e-13 * lmax) keep.push_back(i);
  const int k1 = (int)keep.size();
  if (k1 == 0) {
    std::snprintf(c->last_error, sizeof(c->last_error), "Nystrom approximation is zero");
    return BK_BREAKDOWN;
  }
  std::vector<double> H((size_t)nb * k1, 0.0);  // row-major nb x k1
  for (int j = 0; j < k1; ++j) {
    const int e = keep[j];
    const double sl = std::sqrt(lam[e]);
    for (int i = 0; i < n; ++i) H[(size_t)i * k1 + j] = W[(size_t)i * n + e] * sl;
    // bottom block: B (row-major l x l) times the last l rows of W, scaled by lam^{-1/2}
    for (int i = 0; i < l; ++i) {
      double acc = 0.0;
      for (int q = 0; q < l; ++q) acc += hB[(size_t)i * l + q] * W[(size_t)(n - l + q) * n + e];
      H[(size_t)(n + i) * k1 + j] = acc / sl;
    }
  }
  std::vector<double> M((size_t)k1 * k1, 0.0);
  for (int a = 0; a < k1; ++a)
    for (int bb = a; bb < k1; ++bb) {
      double acc = 0.0;
      for (int i = 0; i < nb; ++i) acc += H[(size_t)i * k1 + a] * H[(size_t)i * k1 + bb];
      M[(size_t)a * k1 + bb] = M[(size_t)bb * k1 + a] = acc;
    }
  std::vector<double> sig2, G;
  jacobi_eigh(k1, M, sig2, G);
  const double smax = sig2.back();
  std::vector<int> kept;
  for (int i = k1 - 1; i >= 0; --i)  // descending, as the oracle's SVD
    if (sig2[i] > 1e-13 * smax) kept.push_back(i);
  const int r = (int)kept.size();
  std::vector<double> Gc((size_t)nb * r), Dv(r);  // column-major nb x r: H G sig^{-1}
  for (int j = 0; j < r; ++j) {
    const int e = kept[j];
    Dv[j] = sig2[e];
    const double is = 1.0 / std::sqrt(sig2[e]);
    for (int i = 0; i < nb; ++i) {
      double acc = 0.0;
      for (int q = 0; q < k1; ++q) acc += H[(size_t)i * k1 + q] * G[(size_t)q * k1 + e];
      Gc[(size_t)j * nb + i] = acc * is;
    }
  }
  const double theta = Dv.back();  // smallest eigenvalue of the approximation (Sec. 7)
  std::vector<double> f(r);
  for (int j = 0; j < r; ++j) f[j] = (theta + mu) / (Dv[j] + mu) - 1.0;

  // --- device buffers: U (d x r), coefficients, PCG vectors and scalars
  double *U = nullptr, *pw = nullptr;
  BK_CK(ws_get(c, WS_NYU, (size_t)d * r * 8 + (size_t)nb * r * 8 + 2 * (size_t)r * 8 + 4096, (void**)&U));
  double* Gd = U + (size_t)d * r;
  double* fd = Gd + (size_t)nb * r;
  double* cv = fd + r;
  BK_CK(ws_get(c, WS_PCG, (size_t)d * 5 * 8 + 4096 * 8, (void**)&pw));
  double *xd = pw, *rd = pw + d, *zd = pw + 2 * d, *pd = pw + 3 * d, *qd = pw + 4 * d;
  double* parts = pw + 5 * d;
  double* sc = parts + bk::pcg_parts();
  BK_CK(cudaMemcpyAsync(Gd, Gc.data(), Gc.size() * 8, cudaMemcpyHostToDevice, st));
  BK_CK(cudaMemcpyAsync(fd, f.data(), f.size() * 8, cudaMemcpyHostToDevice, st));
  BK_CK(bk::launch_gemm(1, d, r, nb, 1.0, lz.Q, 1, 1, lz.ldq, Gd, 1, nb, 0.0, U, d, st));
  // U split once into FP32 head and tail arrays: its two products per iteration then run
  // in compensated FP32-pair arithmetic (about 2^-44 relative) and are bound by HBM, not
  // by the FP64 pipe
  float* Uh = nullptr;
  BK_CK(ws_get(c, WS_DEFL, (size_t)2 * d * r * 4 + 256, (void**)&Uh));
  float* Ul = Uh + (size_t)d * r;
  BK_CK(bk::launch_split_f64(d, r, U, d, Uh, Ul, d, st));
  double* gparts = nullptr;
  BK_CK(ws_get(c, WS_SPLIT, (size_t)bk::defl_parts(d) * r * 8 + 4096, (void**)&gparts));
  auto precond = [&](const double* rin, double* zout) -> cudaError_t {
    // z = r + U diag(f) U^T r  ==  (theta + mu) U (D + mu)^{-1} U^T r + (I - U U^T) r
    cudaError_t e = bk::launch_defl_t(d, r, Uh, Ul, d, rin, gparts, cv, st);
    if (e != cudaSuccess) return e;
    if ((e = bk::launch_scale_vec(r, fd, cv, st)) != cudaSuccess) return e;
    return bk::launch_defl_n(d, r, Uh, Ul, d, cv, rin, zout, c->sms, st);
  };
  double* Vw = nullptr;
  if (o.kind == BK_GRAM) BK_CK(ws_get(c, WS_LB64, (size_t)o.nrows * 8, (void**)&Vw));

  // --- PCG from x = 0 (Def. PCG); scalars stay on the device
  double bn2 = 0.0;
  BK_CK(bk::launch_dot_scalar(3, d, bd, bd, parts, sc, st));
  BK_CK(cudaMemsetAsync(xd, 0, (size_t)d * 8, st));
  BK_CK(cudaMemsetAsync(sc + 5, 0, 8, st));
  BK_CK(cudaMemcpyAsync(rd, bd, (size_t)d * 8, cudaMemcpyDeviceToDevice, st));
  BK_CK(precond(rd, zd));
  BK_CK(cudaMemcpyAsync(pd, zd, (size_t)d * 8, cudaMemcpyDeviceToDevice, st));
  BK_CK(bk::launch_dot_scalar(2, d, rd, zd, parts, sc, st));
  BK_CK(cudaMemcpyAsync(c->hparts, sc, 8 * 8, cudaMemcpyDeviceToHost, st));
  BK_CK(cudaStreamSynchronize(st));
  bn2 = c->hparts[3];
  const double bnorm = std::sqrt(bn2);
  int loads = lz.loads, iters = 0;
  bk_status result = BK_NOT_CONVERGED;
  double rel = bnorm > 0.0 ? 1.0 : 0.0;
  if (bnorm == 0.0) result = BK_OK;
  double* rtrue = qd;  // scratch for the recomputed residual
  int checks = 0;
  while (result != BK_OK && loads < opts.max_loads) {
    BK_CK(apply_fp64(c, o, pd, d, 1, qd, Vw, true));  // q = A p
    ++loads;
    ++iters;
    if (mu != 0.0) BK_CK(bk::launch_axpy(d, mu, pd, qd, st));  // q = (A + mu) p
    BK_CK(bk::launch_dot_scalar(0, d, pd, qd, parts, sc, st));  // alpha = rz / p^T q
    BK_CK(bk::launch_pcg_xr(d, sc, 0.0, pd, qd, xd, rd, parts, st));
    BK_CK(precond(rd, zd));
    BK_CK(bk::launch_dot_scalar(1, d, rd, zd, parts, sc, st));
    BK_CK(bk::launch_pcg_p(d, sc, zd, pd, st));
    if (iters % opts.check_every != 0 && loads < opts.max_loads) continue;
    BK_CK(cudaMemcpyAsync(c->hparts, sc, 8 * 8, cudaMemcpyDeviceToHost, st));
    BK_CK(cudaStreamSynchronize(st));
    if (c->hparts[5] != 0.0) {
      result = BK_BREAKDOWN;
      break;
    }
    if (std::sqrt(c->hparts[3]) > opts.tol * bnorm && loads < opts.max_loads) continue;
    // the recurrence residual met tol (or the cap): confirm with the FP64 residual
    BK_CK(apply_fp64(c, o, xd, d, 1, rtrue, Vw, true));
    BK_CK(bk::launch_axpy(d, mu, xd, rtrue, st));
    BK_CK(bk::launch_axpy(d, -1.0, bd, rtrue, st));
    BK_CK(bk::launch_dot_scalar(3, d, rtrue, rtrue, parts, sc + 8, st));
    BK_CK(cudaMemcpyAsync(c->hparts, sc + 8, 8 * 8, cudaMemcpyDeviceToHost, st));
    BK_CK(cudaStreamSynchronize(st));
    rel = std::sqrt(c->hparts[3]) / bnorm;
    ++checks;
    if (rel <= opts.tol) result = BK_OK;
    if (loads >= opts.max_loads) break;
  }
  BK_CK(cudaMemcpyAsync(x, xd, (size_t)d * 8, cudaMemcpyDefault, st));
  BK_CK(cudaEventRecord(ev1, st));
  BK_CK(cudaEventSynchronize(ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (info) {
    info->status = result;
    info->loads = loads;
    info->refinements = r;  // rank of the Nystrom approximation
    info->residual_loads = checks;
    info->rel_residual = rel;
    info->ms_total = ms;
  }
  return result;
}

namespace {

// Cholesky of the symmetric band matrix T + mu I (bandwidth bw, Lb[r * n + c] = T(c + r, c),
// n x (bw + 1) entries) in place: Lb then holds L with L L^T = T + mu I. A diagonal entry
// of T that is exactly zero (a direction the block QR dropped: its row and column are
// zero) is replaced by 1, which decouples it. Returns false on a non-positive pivot.
bool host_band_chol(int n, int bw, std::vector<double>& Lb, double mu) {
  for (int c = 0; c < n; ++c) Lb[c] = Lb[c] == 0.0 ? 1.0 : Lb[c] + mu;
  for (int c = 0; c < n; ++c) {
    const double x = Lb[c];
    if (!(x > 0.0) || !std::isfinite(x)) return false;
    const double l = std::sqrt(x);
    Lb[c] = l;
    const int w = std::min(bw, n - 1 - c);
    for (int r = 1; r <= w; ++r) Lb[(size_t)r * n + c] /= l;
    for (int a = 1; a <= w; ++a)
      for (int b = 1; b <= a; ++b) Lb[(size_t)(a - b) * n + c + b] -= Lb[(size_t)a * n + c] * Lb[(size_t)b * n + c];
  }
  return true;
}

// y = (L L^T)^{-1} y for the factor of host_band_chol.
void host_band_solve(int n, int bw, const std::vector<double>& Lb, double* y) {
  for (int c = 0; c < n; ++c) {
    double s = y[c];
    for (int r = 1; r <= bw && c - r >= 0; ++r) s -= Lb[(size_t)r * n + c - r] * y[c - r];
    y[c] = s / Lb[c];
  }
  for (int c = n - 1; c >= 0; --c) {
    double s = y[c];
    for (int r = 1; r <= bw && c + r < n; ++r) s -= Lb[(size_t)r * n + c] * y[c + r];
    y[c] = s / Lb[c];
  }
}

}  // namespace

extern "C" bk_status bk_solve_shrink(bk_ctx* c, const bk_operator* A, double mu, const double* b, double* x,
                                     int32_t s_lock, const bk_opts* opts_in, bk_info* info) {
  if (info) std::memset(info, 0, sizeof(*info));
  if (!c || !b || !x || s_lock < 1 || s_lock > 16 || !(mu >= 0.0) || !std::isfinite(mu)) return BK_ERR_ARG;
  err_ctx() = c;
  c->last_error[0] = 0;
  LzOp o;
  bk_status s = check_pcg_operator(A, &o);
  if (s != BK_OK) return s;
  bk_opts opts;
  if (opts_in)
    opts = *opts_in;
  else
    bk_default_opts(&opts);
  if (!(opts.tol > 0.0) || opts.sketch < 0 || opts.max_loads < 1 || opts.check_every < 1) return BK_ERR_ARG;
  const int64_t d = o.d;
  const int l = (int)std::min<int64_t>(opts.sketch, d - 1);
  const int m = 1 + l;                 // block [b Omega]
  const int n = s_lock * m;            // columns of the locked basis V
  const int nb = n + m;                // columns of [V Q_s]
  if (nb > 768) return BK_ERR_UNSUPPORTED;
  BK_CK(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  cudaEvent_t ev0, ev1;
  BK_CK(cudaEventCreate(&ev0));
  BK_CK(cudaEventCreate(&ev1));
  BK_CK(cudaEventRecord(ev0, st));
  Prof prof;  // with opts.profile: events around the one-column loads and the deflation
  prof.on = opts.profile != 0;
  prof.st = st;
  BK_CK(stage_pcg_operator(c, A, &o));
  const double* bd = nullptr;
  BK_CK(stage_in(c, WS_B64, b, (size_t)d * 8, (const void**)&bd));
  double* pw = nullptr;
  BK_CK(ws_get(c, WS_PCG, (size_t)d * 5 * 8 + 4096 * 8, (void**)&pw));
  double *xd = pw, *rd = pw + d, *zd = pw + 2 * d, *pd = pw + 3 * d, *qd = pw + 4 * d;
  double* parts = pw + 5 * d;
  double* sc = parts + bk::pcg_parts();
  BK_CK(bk::launch_dot_scalar(3, d, bd, bd, parts, sc, st));
  BK_CK(cudaMemcpyAsync(c->hparts, sc, 8 * 8, cudaMemcpyDeviceToHost, st));
  BK_CK(cudaStreamSynchronize(st));
  const double bnorm = std::sqrt(c->hparts[3]);
  if (bnorm == 0.0) {
    BK_CK(cudaMemsetAsync(xd, 0, (size_t)d * 8, st));
    BK_CK(cudaMemcpyAsync(x, xd, (size_t)d * 8, cudaMemcpyDefault, st));
    BK_CK(cudaStreamSynchronize(st));
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (info) info->status = BK_OK;
    return BK_OK;
  }

  // --- block phase (Sec. CG_pro): s block-Lanczos steps with full reorthogonalisation on
  // [b / ||b||, Omega / sqrt(d)] (the column scales change R_0, not the spans), giving
  // V = [Q_0 .. Q_{s-1}] of K_s(A, [b Omega]), T_s = V^T A V and the Lanczos relation
  // A V = V T_s + Q_s B_s E_s^T.
  Lanczos lz;
  BK_CK(lz.init(c, o, 1, m, s_lock));
  double* B0 = nullptr;
  BK_CK(ws_get(c, WS_LB0, (size_t)d * m * 8 + 4096 * 8, (void**)&B0));
  double* scales = B0 + (size_t)d * m;
  BK_CK(cudaMemcpyAsync(B0, bd, (size_t)d * 8, cudaMemcpyDeviceToDevice, st));
  if (l > 0) BK_CK(bk::launch_gaussian(opts.seed, 3u, d * (int64_t)l, 0, B0 + d, st));
  std::vector<double> hs(m, 1.0 / std::sqrt((double)d));
  hs[0] = 1.0 / bnorm;
  BK_CK(cudaMemcpyAsync(scales, hs.data(), (size_t)m * 8, cudaMemcpyHostToDevice, st));
  BK_CK(bk::launch_scale_cols(1, d, m, d, scales, B0, st));
  BK_CK(bk::launch_copy_cols(1, 1, d, m, B0, d, lz.W, lz.ldq, st));
  BK_CK(lz.start(lz.W));
  for (int k = 0; k < s_lock; ++k) BK_CK(lz.step());
  // [Q_0 .. Q_s] split once into FP32 head and tail arrays (column-major, ld ldq): the
  // products with the locked basis then run in compensated FP32-pair arithmetic
  float* Vh = nullptr;
  BK_CK(ws_get(c, WS_DEFL, (size_t)2 * lz.ldq * nb * 4 + 256, (void**)&Vh));
  float* Vl = Vh + (size_t)lz.ldq * nb;
  BK_CK(bk::launch_split_f64(d, nb, (const double*)lz.Q, lz.ldq, Vh, Vl, lz.ldq, st));

  // --- small host work: (T_s + mu I) = L L^T, y_0 = (T_s + mu I)^{-1} V^T b and
  // K = (T_s + mu I)^{-1} E_s B_s^T (n x m), so that for any r
  //   (T_s + mu I)^{-1} (A_mu V)^T r = V^T r + K Q_s^T r.
  double* small = nullptr;
  BK_CK(ws_get(c, WS_NYU, ((size_t)n * m + 2 * (size_t)nb + n + 64) * 8, (void**)&small));
  double* Kd = small;
  double* g = Kd + (size_t)n * m;     // [V Q_s]^T r  (nb)
  double* coef = g + nb;              // -(V^T r + K Q_s^T r)  (n)
  double* y0 = coef + n;              // n
  double* gparts = nullptr;
  BK_CK(ws_get(c, WS_SPLIT, (size_t)bk::defl_parts(d) * nb * 8 + 4096, (void**)&gparts));
  BK_CK(bk::launch_defl_t(d, n, Vh, Vl, lz.ldq, bd, gparts, g, st));
  std::vector<double> hband((size_t)(m + 1) * lz.ldb()), hB((size_t)m * m), hg(n);
  BK_CK(cudaMemcpyAsync(hband.data(), lz.band, hband.size() * 8, cudaMemcpyDeviceToHost, st));
  BK_CK(cudaMemcpyAsync(hB.data(), lz.Bk, hB.size() * 8, cudaMemcpyDeviceToHost, st));
  BK_CK(cudaMemcpyAsync(hg.data(), g, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
  BK_CK(cudaStreamSynchronize(st));
  std::vector<double> Lb((size_t)(m + 1) * n, 0.0);
  for (int r = 0; r <= m; ++r)
    for (int col = 0; col + r < n; ++col) Lb[(size_t)r * n + col] = hband[(size_t)r * lz.ldb() + col];
  if (!host_band_chol(n, m, Lb, mu)) {
    std::snprintf(c->last_error, sizeof(c->last_error), "T_s + mu I not positive definite");
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    return BK_BREAKDOWN;
  }
  host_band_solve(n, m, Lb, hg.data());
  std::vector<double> hK((size_t)n * m, 0.0);
  for (int q = 0; q < m; ++q) {
    double* col = hK.data() + (size_t)q * n;
    // column q of E_s B_s^T: B_s(q, i) in row n - m + i (B_s row-major)
    for (int i = 0; i < m; ++i) col[n - m + i] = hB[(size_t)q * m + i];
    host_band_solve(n, m, Lb, col);
  }
  BK_CK(cudaMemcpyAsync(Kd, hK.data(), hK.size() * 8, cudaMemcpyHostToDevice, st));
  BK_CK(cudaMemcpyAsync(y0, hg.data(), (size_t)n * 8, cudaMemcpyHostToDevice, st));

  // --- x_0 = V y_0 (the block-CG iterate after s loads), r_0 = b - A_mu x_0 (one load)
  double* Vw = nullptr;
  if (o.kind == BK_GRAM) BK_CK(ws_get(c, WS_LB64, (size_t)o.nrows * 8, (void**)&Vw));
  BK_CK(cudaMemsetAsync(xd, 0, (size_t)d * 8, st));
  BK_CK(bk::launch_defl_n(d, n, Vh, Vl, lz.ldq, y0, xd, xd, c->sms, st));
  BK_CK(apply_fp64(c, o, xd, d, 1, qd, Vw, true));
  BK_CK(bk::launch_axpy(d, mu, xd, qd, st));
  BK_CK(cudaMemcpyAsync(rd, bd, (size_t)d * 8, cudaMemcpyDeviceToDevice, st));
  BK_CK(bk::launch_axpy(d, -1.0, qd, rd, st));
  // The direction p = r - V (V^T r + K Q_s^T r) + beta p is A_mu-orthogonal to V (Def-CG
  // with the coefficients from the Lanczos relation); one pass over [V Q_s] for the
  // coefficients, one over V for the update.
  auto direction = [&]() -> cudaError_t {
    cudaError_t e = bk::launch_defl_t(d, nb, Vh, Vl, lz.ldq, rd, gparts, g, st);
    if (e != cudaSuccess) return e;
    if ((e = bk::launch_defl_coef(n, m, Kd, g, coef, st)) != cudaSuccess) return e;
    return bk::launch_defl_np(d, n, Vh, Vl, lz.ldq, coef, sc, rd, pd, c->sms, st);
  };
  BK_CK(cudaMemsetAsync(sc, 0, 16 * 8, st));  // beta = 0 and no breakdown for p_0
  BK_CK(cudaMemsetAsync(pd, 0, (size_t)d * 8, st));
  BK_CK(direction());
  BK_CK(bk::launch_dot_scalar(2, d, rd, rd, parts, sc, st));  // rz := r^T r

  // --- one-column deflated CG; scalars stay on the device. r_0 was formed from the
  // stored values, so x_0 may already meet tol (a locked basis that spans R^d).
  int loads = lz.loads + 1, iters = 0, checks = 0;
  bk_status result = BK_NOT_CONVERGED;
  BK_CK(cudaMemcpyAsync(c->hparts, sc, 8, cudaMemcpyDeviceToHost, st));
  BK_CK(cudaStreamSynchronize(st));
  double rel = std::sqrt(c->hparts[0]) / bnorm;
  if (rel <= opts.tol) result = BK_OK;
  double* rtrue = qd;
  while (result != BK_OK && loads < opts.max_loads) {
    prof.begin();
    BK_CK(apply_fp64(c, o, pd, d, 1, qd, Vw, true));  // q = A p
    prof.end(BK_K_OPERATOR);
    ++loads;
    ++iters;
    BK_CK(bk::launch_dot_shift_scalar(0, d, pd, qd, mu, parts, sc, st));  // alpha = r^T r / p^T A_mu p
    BK_CK(bk::launch_pcg_xr(d, sc, mu, pd, qd, xd, rd, parts, st));       // x, r and rr = r^T r
    BK_CK(bk::launch_dot_shift_scalar(4, d, nullptr, nullptr, 0.0, parts, sc, st));  // beta = rr / rz
    prof.begin();
    BK_CK(direction());
    prof.end(BK_K_ORTH);
    if (iters % opts.check_every != 0 && loads < opts.max_loads) continue;
    BK_CK(cudaMemcpyAsync(c->hparts, sc, 8 * 8, cudaMemcpyDeviceToHost, st));
    BK_CK(cudaStreamSynchronize(st));
    if (c->hparts[5] != 0.0) {
      result = BK_BREAKDOWN;
      break;
    }
    if (std::sqrt(c->hparts[3]) > opts.tol * bnorm && loads < opts.max_loads) continue;
    // the recurrence residual met tol (or the cap): confirm with the FP64 residual
    BK_CK(apply_fp64(c, o, xd, d, 1, rtrue, Vw, true));
    BK_CK(bk::launch_axpy(d, mu, xd, rtrue, st));
    BK_CK(bk::launch_axpy(d, -1.0, bd, rtrue, st));
    BK_CK(bk::launch_dot_scalar(3, d, rtrue, rtrue, parts, sc + 8, st));
    BK_CK(cudaMemcpyAsync(c->hparts, sc + 8, 8 * 8, cudaMemcpyDeviceToHost, st));
    BK_CK(cudaStreamSynchronize(st));
    rel = std::sqrt(c->hparts[3]) / bnorm;
    ++checks;
    if (rel <= opts.tol) result = BK_OK;
    if (loads >= opts.max_loads) break;
  }
  BK_CK(cudaMemcpyAsync(x, xd, (size_t)d * 8, cudaMemcpyDefault, st));
  BK_CK(cudaEventRecord(ev1, st));
  BK_CK(cudaEventSynchronize(ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  prof.report(info);
  if (info) {
    info->status = result;
    info->loads = loads;
    info->refinements = n;  // columns of the locked basis
    info->residual_loads = checks;
    info->rel_residual = rel;
    info->ms_total = ms;
  }
  return result;
}

extern "C" bk_status bk_apply_ozaki(bk_ctx* c, const bk_operator* A, double mu, int32_t L, const double* X,
                                    int64_t ldx, double* Y, int64_t ldy) {
  if (!c || !X || !Y || L < 1 || !std::isfinite(mu)) return BK_ERR_ARG;
  err_ctx() = c;
  c->last_error[0] = 0;
  LzOp o;
  bk_status s = check_pcg_operator(A, &o);
  if (s != BK_OK) return s;
  const int64_t d = o.d;
  if (ldx < d || ldy < d) return BK_ERR_ARG;
  const bool gram = A->kind == BK_GRAM;
  if (gram ? !bk::ozaki_gram_usable(o.nrows, d, L)
           : (A->kind != BK_DENSE || A->dtype != BK_F32 || !bk::ozaki_usable(d, L)))
    return BK_ERR_UNSUPPORTED;
  BK_CK(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  BK_CK(stage_pcg_operator(c, A, &o));
  const size_t xbytes = ((size_t)(L - 1) * ldx + d) * 8;
  const double* Xd = nullptr;
  BK_CK(stage_in(c, WS_TMP_IN, X, xbytes, (const void**)&Xd));
  double* Yd = Y;
  const bool direct = is_device_ptr(Y) && ldy == ldx;
  if (!direct) BK_CK(ws_get(c, WS_TMP_OUT, xbytes, (void**)&Yd));
  void *oza = nullptr, *ozx = nullptr;
  const size_t ab = gram ? bk::ozaki_gram_bytes(o.nrows, d) : bk::ozaki_a_bytes(d);
  const size_t xb = gram ? bk::ozaki_gram_work_bytes(o.nrows, d, L, c->sms) : bk::ozaki_x_bytes(d, L, c->sms);
  BK_CK(ws_get(c, WS_OZ_A, ab, &oza));
  BK_CK(ws_get(c, WS_OZ_X, xb + 256, &ozx));
  int* err = (int*)((char*)ozx + xb);
  BK_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
  if (gram) {
    BK_CK(bk::launch_ozaki_split_gram(o.nrows, d, o.vals_f64, o.vals, o.ld, oza, c->sms, st));
    BK_CK(bk::launch_ozaki_gram_apply(o.nrows, d, L, oza, Xd, ldx, Yd, ldx, ozx, 0, err, c->sms, st));
  } else {
    BK_CK(bk::launch_ozaki_split_a(d, (const float*)o.vals, o.ld, oza, c->sms, st));
    BK_CK(bk::launch_ozaki_apply(d, L, oza, Xd, ldx, Yd, ldx, ozx, 0, err, c->sms, st));
  }
  if (mu != 0.0)
    for (int j = 0; j < L; ++j) BK_CK(bk::launch_axpy(d, mu, Xd + (size_t)j * ldx, Yd + (size_t)j * ldx, st));
  if (!direct)
    BK_CK(cudaMemcpy2DAsync(Y, (size_t)ldy * 8, Yd, (size_t)ldx * 8, (size_t)d * 8, L, cudaMemcpyDefault, st));
  int herr = 0;
  BK_CK(cudaMemcpyAsync(c->hparts, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  BK_CK(cudaStreamSynchronize(st));
  std::memcpy(&herr, c->hparts, sizeof(int));
  if (herr) {
    std::snprintf(c->last_error, sizeof(c->last_error), "tensor-core pipeline wait timed out");
    return BK_TIMEOUT;
  }
  return BK_OK;
}

extern "C" bk_status bk_apply(bk_ctx* c, const bk_operator* A, double mu, int32_t L, const double* X, int64_t ldx,
                              double* Y, int64_t ldy) {
  if (!c || !X || !Y || L < 1 || !std::isfinite(mu)) return BK_ERR_ARG;
  err_ctx() = c;
  c->last_error[0] = 0;
  LzOp o;
  bk_status s = check_pcg_operator(A, &o);
  if (s != BK_OK) return s;
  const int64_t d = o.d;
  if (ldx < d || ldy < d) return BK_ERR_ARG;
  BK_CK(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  BK_CK(stage_pcg_operator(c, A, &o));
  const size_t xbytes = ((size_t)(L - 1) * ldx + d) * 8;
  const double* Xd = nullptr;
  BK_CK(stage_in(c, WS_TMP_IN, X, xbytes, (const void**)&Xd));
  // the products write d x L with leading dimension ldx; Y itself when it is device
  // memory with the same leading dimension, otherwise a workspace copied out after
  double* Yd = Y;
  const bool direct = is_device_ptr(Y) && ldy == ldx;
  if (!direct) BK_CK(ws_get(c, WS_TMP_OUT, xbytes, (void**)&Yd));
  double* Vw = nullptr;
  if (o.kind == BK_GRAM) BK_CK(ws_get(c, WS_LV, (size_t)o.nrows * L * 8, (void**)&Vw));
  BK_CK(apply_fp64(c, o, Xd, ldx, L, Yd, Vw, true));
  if (mu != 0.0)
    for (int j = 0; j < L; ++j) BK_CK(bk::launch_axpy(d, mu, Xd + (size_t)j * ldx, Yd + (size_t)j * ldx, st));
  if (!direct)
    BK_CK(cudaMemcpy2DAsync(Y, (size_t)ldy * 8, Yd, (size_t)ldx * 8, (size_t)d * 8, L, cudaMemcpyDefault, st));
  BK_CK(cudaStreamSynchronize(st));
  return BK_OK;
}
