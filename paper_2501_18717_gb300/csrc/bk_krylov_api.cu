// Block-Lanczos drivers of the C ABI: bk_ridge_path (Sec. 3.2, Eq. bcg_alg, one basis
// for every shift) and bk_sample (Def. blansq). The host orders launches and reads
// small status vectors; the products, Grams, factorisations and shifted solves run in
// the kernels of k_gemm.cu and k_krylov.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
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
};

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
  int64_t d = 0, ldq = 0, ncol_max = 0;
  void *Q = nullptr, *W = nullptr, *V = nullptr, *C = nullptr, *Rt = nullptr;
  double *G = nullptr, *R1 = nullptr, *R2 = nullptr, *Ri1 = nullptr, *Ri2 = nullptr, *work = nullptr;
  double *Ak = nullptr, *Bk = nullptr, *R0 = nullptr, *band = nullptr;
  int *keep = nullptr, *rank = nullptr;
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
    if (op.kind == BK_GRAM)
      if ((e = ws_get(c, WS_LV, (size_t)op.nrows * m * es, &V)) != cudaSuccess) return e;
    if ((e = ws_get(c, WS_LC, (size_t)ncol_max * m * es, &C)) != cudaSuccess) return e;
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
    if ((e = ws_get(c, WS_LBAND, (size_t)(m + 1) * ncol_max * 8, (void**)&band)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(band, 0, (size_t)(m + 1) * ncol_max * 8, st)) != cudaSuccess) return e;
    t = 0;
    loads = 0;
    return cudaSuccess;
  }

  // Y (d x nc, ldy) = A X (d x nc, ldx), block precision.
  cudaError_t apply(const void* X, int64_t ldx, void* Y, int64_t ldy, int nc) {
    cudaError_t e;
    const int af = op.vals_f64;  // 1: FP64 values, 0: FP32 values
    if (!is64 && af) return cudaErrorInvalidValue;  // FP32 runs use FP32 values
    if (op.kind == BK_DENSE) {
      e = bk::launch_gemm(is64, d, nc, d, 1.0, op.vals, af, op.ld, 1, X, 1, ldx, 0.0, Y, ldy, st);
    } else {
      e = bk::launch_gemm(is64, op.nrows, nc, d, 1.0, op.vals, af, op.ld, 1, X, 1, ldx, 0.0, V, op.nrows, st);
      if (e != cudaSuccess) return e;
      e = bk::launch_gemm(is64, d, nc, op.nrows, 1.0, op.vals, af, 1, op.ld, V, 1, op.nrows, 0.0, Y, ldy, st);
    }
    return e;
  }

  // CholQR2: Wb (d x m) = Qout Bout, Bout upper triangular (m x m row-major FP64).
  cudaError_t qr(void* Wb, void* Qout, double* Bout) {
    cudaError_t e;
    const int gaf = is64 ? 1 : 2;  // Gram of the block: FP64 accumulation of exact products
    for (int pass = 0; pass < 2; ++pass) {
      const void* src = pass == 0 ? Wb : Qout;
      double* R = pass == 0 ? R1 : R2;
      double* Ri = pass == 0 ? Ri1 : Ri2;
      if ((e = bk::launch_gemm(1, m, m, d, 1.0, src, gaf, ldq, 1, src, 1, ldq, 0.0, G, m, st)) != cudaSuccess)
        return e;
      if ((e = bk::launch_chol_inv(m, G, rank_tol, work, R, Ri, keep, rank, st)) != cudaSuccess) return e;
      // Qout = src * Ri (Ri row-major: element (k, j) at Ri[k m + j])
      if (is64) {
        e = bk::launch_gemm(1, d, m, m, 1.0, src, 1, 1, ldq, Ri, m, 1, 0.0, Qout, ldq, st);
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
    if ((e = apply(Qk, ldq, W, ldq, m)) != cudaSuccess) return e;
    ++loads;
    // A_k = Q_k^T (A Q_k) with FP64 accumulation
    const int gaf = is64 ? 1 : 2;
    if ((e = bk::launch_gemm(1, m, m, d, 1.0, Qk, gaf, ldq, 1, W, 1, ldq, 0.0, Ak, m, st)) != cudaSuccess) return e;
    // full reorthogonalisation against Q_0..Q_k, twice
    const int64_t nk = (int64_t)(k + 1) * m;
    for (int pass = 0; pass < 2; ++pass) {
      if ((e = bk::launch_gemm(is64, nk, m, d, 1.0, Q, is64, ldq, 1, W, 1, ldq, 0.0, C, nk, st)) != cudaSuccess)
        return e;
      if ((e = bk::launch_gemm(is64, d, m, nk, -1.0, Q, is64, 1, ldq, C, 1, nk, 1.0, W, ldq, st)) != cudaSuccess)
        return e;
    }
    if ((e = qr(W, qblock(k + 1), Bk)) != cudaSuccess) return e;
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
cudaError_t apply_fp64(bk_ctx* c, const LzOp& o, const double* X, int64_t ld, int L, double* AX, double* Vw) {
  if (o.kind == BK_DENSE) return bk::launch_gemm(1, o.d, L, o.d, 1.0, o.vals, o.vals_f64, o.ld, 1, X, 1, ld, 0.0, AX,
                                                 ld, c->stream);
  cudaError_t e =
      bk::launch_gemm(1, o.nrows, L, o.d, 1.0, o.vals, o.vals_f64, o.ld, 1, X, 1, ld, 0.0, Vw, o.nrows, c->stream);
  if (e != cudaSuccess) return e;
  return bk::launch_gemm(1, o.d, L, o.nrows, 1.0, o.vals, o.vals_f64, 1, o.ld, Vw, 1, o.nrows, 0.0, AX, ld,
                         c->stream);
}

}  // namespace

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
  if (opts.inner != BK_PREC_FP64 && opts.inner != BK_PREC_FP32) return BK_ERR_UNSUPPORTED;
  std::vector<double> hmu(L);
  BK_CK(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  // shifts to the host (validation) and the device
  BK_CK(cudaMemcpy(hmu.data(), mus, (size_t)L * 8, cudaMemcpyDefault));
  for (double v : hmu)
    if (!(v >= 0.0) || !std::isfinite(v)) return BK_ERR_ARG;
  const int is64 = opts.inner == BK_PREC_FP64;
  const int64_t d = o.d;
  const int m = (int)std::min<int64_t>((int64_t)opts.sketch + 1, d);
  if (m > 256) return BK_ERR_UNSUPPORTED;
  cudaEvent_t ev0, ev1;
  BK_CK(cudaEventCreate(&ev0));
  BK_CK(cudaEventCreate(&ev1));
  BK_CK(cudaEventRecord(ev0, st));

  const void* staged = nullptr;
  LzOp o64 = o;  // refinement residuals use the values as given
  BK_CK(stage_lz_values(c, A, &o, is64, &staged));
  o64.vals = staged;
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
    Lanczos lz;
    LzOp ol = o;
    BK_CK(lz.init(c, ol, is64, mb, tmax));
    const size_t es = is64 ? 8 : 4;
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
    BK_CK(bk::launch_copy_cols(1, is64, d, mb, B0d, d, lz.W, lz.ldq, st));
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
      if (est <= target || last) done = 1;
    }
    loads += lz.loads;
    // X += Q_t Z (pass 0 scaled back by ||b||: the start column was b / ||b||)
    const int n = lz.n();
    BK_CK(bk::launch_gemm(1, d, L, n, pass == 0 ? bnorm : 1.0, lz.Q, is64, 1, lz.ldq, Z, 1, n, 1.0, Xd, ldx, st));
    ++refinements;
    // FP64 residuals of every shift
    BK_CK(apply_fp64(c, o64, Xd, ldx, L, AX, Vw));
    BK_CK(bk::launch_shift_residual(d, L, bd, AX, Xd, ldx, dmu, Rres, norms, st));
    residual_loads += 1;
    BK_CK(cudaMemcpyAsync(c->hparts, norms, (size_t)L * 8, cudaMemcpyDeviceToHost, st));
    BK_CK(cudaStreamSynchronize(st));
    worst = 0.0;
    for (int j = 0; j < L; ++j) worst = std::max(worst, std::sqrt(c->hparts[j]) / bnorm);
    if (worst <= opts.tol) result = BK_OK;
    (void)es;
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
  return result;
}
