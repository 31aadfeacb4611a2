// Shared declarations of the CUDA side of the block-CG library (device code and the
// host launchers used by the C ABI). Nothing here is visible through include/bk.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bk {

// Device-side control block of one inner block-CG solve. Written and read by the
// step kernels so that the iteration needs no host round trip; the host reads it
// every `check_every` block products.
//
// Race-free ownership: every field is written by exactly one kind of kernel (and the
// reset kernel), and no kernel reads a field that its own launch writes.
//   done_a, pending_x, loads, first   written by the alpha small-solve (CTA 0); loads
//                                     is read back only by the beta small-solve, first
//                                     only by the direction update
//   done_b, res, kept                 written by the beta small-solve (CTA 0)
//   status                            written by whichever sets a done flag
struct DevState {
  int done_a;       // G unusable (negative or non-finite diagonal, or no kept column)
  int done_b;       // residual met its target, load cap, or S unusable
  int pending_x;    // this step's xc is valid: the x update must run
  int first;        // no load yet in this inner solve (direction update only normalises)
  int loads;        // block products completed in this inner solve
  int status;       // ST_* below
  int max_loads;    // cap for this inner solve
  int timeout;      // set by a kernel whose bounded wait on a pipeline barrier gave up
  int kept;         // columns kept by the latest factorisation of S = W^T W (block rank)
  double tol_abs;   // target on ||R e_1|| = ||c|| (column 0 starts with norm 1)
  double res;       // latest ||c|| from the recurrence
};

enum { ST_RUNNING = 0, ST_CONVERGED = 1, ST_BREAKDOWN = 2, ST_LOADCAP = 3 };

// The recurrence's residual estimate ||c|| starts at 1; the CG residual 2-norm can grow
// transiently, by at most about sqrt(kappa). An estimate above this bound, or not
// finite, means the finite-precision recurrence has lost its orthogonality (seen with
// FP32 blocks wider than about 48 on systems of a few hundred unknowns, where a few
// loads exhaust the space): the inner solve stops as a breakdown.
constexpr double kDivergedRes = 1e8;

// Padded block widths the kernels are compiled for (multiples of 4 for the 4x4
// register blocks of the Gram kernels). Width 65 (sketch 64) pads to 68.
constexpr int kMaxWidth = 65;
inline int padded_width(int m) {
  if (m <= 4) return 4;
  if (m <= 8) return 8;
  if (m <= 16) return 16;
  if (m <= 24) return 24;
  if (m <= 36) return 36;
  if (m <= 68) return 68;
  return -1;
}
// Widest padded block the tensor-core dense products are built for.
constexpr int kTcMaxPadded = 36;
// Entries of one Gram partial: upper-triangular 4x4 blocks, 16 entries each.
inline int gram_entries(int mp) {
  int nb = mp / 4;
  return nb * (nb + 1) / 2 * 16;
}

// ---------------------------------------------------------------- launchers
// All launchers enqueue on `st` and return the launch status.

// Y = A P + mu P and the per-CTA partials of G = P^T Y, CSR operator.
cudaError_t launch_csr_spmm_gram(int is_f64, int mp, int64_t d, const int* rowptr, const int* colidx,
                                 const void* vals, double mu, const void* P, void* Y, int64_t ld, int m,
                                 double* parts, int nparts, const DevState* state, cudaStream_t st);
int csr_spmm_gram_grid(int is_f64, int mp, int64_t d, int device);

// Same for a dense row-major operator with leading dimension lda.
cudaError_t launch_dense_gram(int is_f64, int mp, int64_t d, const void* A, int64_t lda, double mu,
                              const void* P, void* Y, int64_t ld, int m, double* parts, int nparts,
                              const DevState* state, cudaStream_t st);
int dense_gram_grid(int is_f64, int mp, int64_t d, int device);

// Tensor-core variant for FP32 values (k_tc.cu): usable when A is 16-byte aligned, lda
// is a multiple of 4 and mp <= 36. One CTA per 128-row tile (nparts = dense_tc_tiles(d));
// pt is scratch for P^T head and tail (dense_tc_pt_bytes). *err is set to 1 if a
// pipeline wait gave up after wait_cycles SM clocks (0: the default, about 2 s); the
// product is then invalid.
bool dense_tc_usable(int64_t d, const void* A, int64_t lda, int mp);
int dense_tc_tiles(int64_t d);
size_t dense_tc_pt_bytes(int64_t d, int mp);
cudaError_t launch_dense_gram_tc(int mp, int64_t d, const float* A, int64_t lda, double mu, const float* P, float* Y,
                                 int64_t ld, int m, double* parts, int nparts, const DevState* state, float* pt,
                                 int* err, long long wait_cycles, cudaStream_t st);

// Partials of G = X^T Y.
cudaError_t launch_gram(int is_f64, int mp, int64_t d, const void* X, const void* Y, int64_t ld, int m,
                        double* parts, int nparts, cudaStream_t st);
int gram_grid(int is_f64, int mp, int64_t d, int device);

// Sum of partials (fixed order) into a full symmetric m x m FP64 matrix.
cudaError_t launch_reduce_gram(int mp, int m, const double* parts, int nparts, double* out,
                               const DevState* state, cudaStream_t st);

// Small solves of the orthonormal-residual step (k_block.cu). alpha: Gi = G^+ and
// xc = G^+ c as mp x mp / mp copies in the block precision. beta: S = T^T T, writes
// T (row-major) and (T^+)^T (row-major) in the block precision, c <- T c, and the
// stopping decision on ||c||. rank_tol: pivots of the unit-diagonal scaled matrix at
// or below it count as dependent columns.
cudaError_t launch_small_alpha(int is_f64, int mp, int m, const double* G, const double* cvec, void* gi_t,
                               void* xc_t, double rank_tol, DevState* state, cudaStream_t st);
cudaError_t launch_small_beta(int is_f64, int mp, int m, const double* S, double* cvec, void* ti_t, void* t_t,
                              double rank_tol, DevState* state, cudaStream_t st);
// Stand-alone X = G^{-1} S (no state); status word set to 1 on breakdown.
cudaError_t launch_chol_solve(int m, const double* G, const double* S, double* X, int* flag, cudaStream_t st);

// W = Q - Y Gi (in place in Q) with per-CTA partials of W^T W.
cudaError_t launch_update_r(int is_f64, int mp, int64_t d, int m, const void* Y, void* R, int64_t ld,
                            const void* alpha_t, double* parts, int nparts, const DevState* state,
                            cudaStream_t st);
int update_r_grid(int is_f64, int mp, int64_t d, int device);

// x += P xc (FP64 accumulator) and, unless the solve stopped, Q = W T^{-1}, P = Q + P T^T.
cudaError_t launch_update_p(int is_f64, int mp, int64_t d, int m, void* Q, void* P, int64_t ld, const void* xc_t,
                            const void* ti_t, const void* t_t, double* x, const DevState* state, cudaStream_t st);

// Start block of an inner solve: Q[:,0] = r * scale, Q[:,1:] = Omega, x = 0.
cudaError_t launch_start_block(int is_f64, int64_t d, int m, int64_t ld, const double* r, double scale,
                               const void* omega, void* Q, double* x, cudaStream_t st);
// Omega (d x l) from Philox stream 3, times `scale`, written as columns 1..l of a panel
// block with leading dimension ld (the caller zeroes column 0 and the padding).
cudaError_t launch_omega(int is_f64, int64_t d, int l, int64_t ld, uint64_t seed, double scale, void* out,
                         cudaStream_t st);
// Standard normals of a stream (FP64).
cudaError_t launch_gaussian(uint64_t seed, uint32_t stream, int64_t n, int64_t offset, double* out,
                            cudaStream_t st);

// FP64-accurate dense products Y = A X (A: d x d FP32 row-major, lda; X, Y: d x N FP64
// column-major) by an Ozaki split on the BF16 tensor cores (k_ozaki.cu). The digits of
// A are made once per operator into `abuf` (ozaki_a_bytes); each product splits X
// into `xbuf` (ozaki_x_bytes). *err is set if a pipeline wait gave up.
bool ozaki_usable(int64_t d, int N);
size_t ozaki_a_bytes(int64_t d);
size_t ozaki_x_bytes(int64_t d, int N, int sms);
cudaError_t launch_ozaki_split_a(int64_t d, const float* A, int64_t lda, void* abuf, int sms, cudaStream_t st);
cudaError_t launch_ozaki_apply(int64_t d, int N, const void* abuf, const double* X, int64_t ldx, double* Y,
                               int64_t ldy, void* xbuf, long long wait_cycles, int* err, int sms, cudaStream_t st);
// Gram form A = Z^T Z (Z: n x d row-major, FP32 or FP64, ldz): the digits of Z and of Z^T
// go into `zbuf` (ozaki_gram_bytes) once per operator; a product Y = Z^T (Z X) uses
// `work` (ozaki_gram_work_bytes).
// General FP64 product C = alpha A B + beta C by the Ozaki split (strides as in
// launch_gemm; each operand contiguous along K or along its other index).
bool ozaki_gemm_usable(int64_t M, int64_t N, int64_t K, int64_t sai, int64_t sak, int64_t sbk, int64_t sbj);
size_t ozaki_gemm_work_bytes(int64_t M, int64_t N, int64_t K, int sms);
cudaError_t launch_ozaki_gemm(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t sai,
                              int64_t sak, const double* B, int64_t sbk, int64_t sbj, double beta, double* C,
                              int64_t ldc, void* work, long long wait_cycles, int* err, int sms, cudaStream_t st);
bool ozaki_gram_usable(int64_t n, int64_t d, int N);
size_t ozaki_gram_bytes(int64_t n, int64_t d);
size_t ozaki_gram_work_bytes(int64_t n, int64_t d, int N, int sms);
cudaError_t launch_ozaki_split_gram(int64_t n, int64_t d, int z_f64, const void* Z, int64_t ldz, void* zbuf, int sms,
                                    cudaStream_t st);
cudaError_t launch_ozaki_gram_apply(int64_t n, int64_t d, int N, const void* zbuf, const double* X, int64_t ldx,
                                    double* Y, int64_t ldy, void* work, long long wait_cycles, int* err, int sms,
                                    cudaStream_t st);

// FP64 residual r = b - (A x + mu x) and per-CTA partials of ||r||^2.
cudaError_t launch_csr_residual(int vals_f64, int64_t d, const int* rowptr, const int* colidx,
                                const void* vals, double mu, const double* x, const double* b, double* r,
                                double* norm_parts, int nparts, cudaStream_t st);
cudaError_t launch_dense_residual(int vals_f64, int64_t d, const void* A, int64_t lda, double mu,
                                  const double* x, const double* b, double* r, double* norm_parts,
                                  int nparts, cudaStream_t st);
// x += a * y (FP64)
cudaError_t launch_axpy(int64_t d, double a, const double* y, double* x, cudaStream_t st);
// out = x + a y (out may alias y)
cudaError_t launch_axpy_out(int64_t d, double a, const double* y, const double* x, double* out, cudaStream_t st);
// FP64 -> FP32 copy
cudaError_t launch_to_f32(int64_t n, const double* in, float* out, cudaStream_t st);
// FP32 -> FP64 copy
cudaError_t launch_to_f64(int64_t n, const float* in, double* out, cudaStream_t st);
// ||v||^2 partials (nparts CTAs of 256 threads)
cudaError_t launch_norm2_parts(int64_t d, const double* v, double* parts, int nparts, cudaStream_t st);
// Dense: FP64 -> FP32 copy of a d x d row-major matrix with leading dimension lda into lda32.
cudaError_t launch_dense_to_f32(int64_t d, const double* in, int64_t lda, float* out, int64_t lda32,
                                cudaStream_t st);
// C = alpha A B + beta C (column-major C, general strides for A and B; see k_gemm.cu).
// is_f64: element type of B and C (and the accumulation). a_f64: 1 A is FP64, 0 A is
// FP32; with is_f64 = 1, a_f64 = 2 means A and B are FP32 (FP64 accumulation/output).
cudaError_t launch_gemm(int is_f64, int64_t M, int64_t N, int64_t K, double alpha, const void* A, int a_f64,
                        int64_t sai, int64_t sak, const void* B, int64_t sbk, int64_t sbj, double beta, void* C,
                        int64_t ldc, cudaStream_t st);
// Split-K form of launch_gemm for few output tiles and a long K (tall Gram products):
// the K range is cut into chunks whose partial products go to `work` and are added in
// chunk order in FP64. Falls back to launch_gemm when splitting does not pay or `work`
// is too small (gemm_split_work_bytes gives the size it wants).
cudaError_t launch_gemm_split(int is_f64, int64_t M, int64_t N, int64_t K, double alpha, const void* A, int a_f64,
                              int64_t sai, int64_t sak, const void* B, int64_t sbk, int64_t sbj, double beta, void* C,
                              int64_t ldc, void* work, size_t work_bytes, int sms, cudaStream_t st);
size_t gemm_split_work_bytes(int is_f64, int64_t M, int64_t N, int64_t K, int sms);
// Double-float launch_gemm_split for FP64 A, B, C (compensated FP32-pair products,
// about 2^-44 relative; see k_gemm.cu); same strides, same split-K work size.
cudaError_t launch_gemm_dd(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t sai, int64_t sak,
                           const double* B, int64_t sbk, int64_t sbj, double beta, double* C, int64_t ldc, void* work,
                           size_t work_bytes, int sms, cudaStream_t st);
// ---- tall-skinny products of the Lanczos drivers (k_tsm.cu)
// df = 0: FP32 B / T (the *lo arguments unused) and FP32 output; df = 1: B / T is an
// FP64 operand given as its FP32 head and tail (launch_split_f64, same leading
// dimension), FP64 output with compensated FP32 arithmetic (FP64-accurate for FP32 A /
// Z). Every FP32 array must be 16-byte aligned with a leading dimension that is a
// multiple of 4 floats; tsm_supported checks one.
bool tsm_supported(const void* A, int64_t lda);
cudaError_t launch_split_f64(int64_t rows, int cols, const double* src, int64_t lds, float* hi, float* lo, int64_t ldd,
                             cudaStream_t st);
cudaError_t launch_tsm_nn(int df, int64_t M, int N, int64_t K, double alpha, const float* A, int64_t lda,
                          const float* B, const float* Blo, int64_t ldb, double beta, void* C, int64_t ldc,
                          cudaStream_t st);
cudaError_t launch_tsm_tn(int df, int64_t R, int64_t D, int N, const float* Z, int64_t ldz, const float* T,
                          const float* Tlo, int64_t ldt, double alpha, double beta, void* Y, int64_t ldy, void* work,
                          size_t work_bytes, int sms, cudaStream_t st);
size_t tsm_tn_work_bytes(int64_t R, int64_t D, int N, int df, int sms);
// ---- BF16 tensor-core Gram-form products (k_bf16.cu): Y = alpha Z^T (Z X) + beta Y for
// FP32 X (d x N column-major, ldx) and Y (ldy), N <= 128, from BF16 head/tail copies of
// the FP32 Z (n x d row-major, ldz) that launch_bf16_gram_split writes into `buf`
// (bf16_gram_copy_bytes) once per operator. `work` holds bf16_gram_work_bytes; *err is
// set to 1 if a pipeline wait gave up after wait_cycles SM clocks (0: the default).
bool bf16_gram_usable(int64_t n, int64_t d, int N);
size_t bf16_gram_copy_bytes(int64_t n, int64_t d);
size_t bf16_gram_work_bytes(int64_t n, int64_t d, int N, int sms);
cudaError_t launch_bf16_gram_split(int64_t n, int64_t d, const float* Z, int64_t ldz, void* buf, cudaStream_t st);
cudaError_t launch_bf16_gram_apply(int64_t n, int64_t d, int N, const void* buf, const float* X, int64_t ldx, float* Y,
                                   int64_t ldy, double alpha, double beta, void* work, size_t work_bytes,
                                   long long wait_cycles, int* err, int sms, cudaStream_t st);
// ---- Nystrom PCG (k_pcg.cu), FP64
cudaError_t launch_csr_cols(int vals_f64, int64_t d, const int* rowptr, const int* colidx, const void* vals, int nc,
                            const double* X, int64_t ldx, double* Y, int64_t ldy, cudaStream_t st);
int pcg_parts();
// kind 0: sc[1] = sc[0] / (a^T b); 1: sc[2] = (a^T b) / sc[0], sc[0] = a^T b; 2: sc[0] = a^T b;
// 3: sc[3] = a^T b. parts: pcg_parts() doubles.
cudaError_t launch_dot_scalar(int kind, int64_t n, const double* a, const double* b, double* parts, double* sc,
                              cudaStream_t st);
// the same with a^T (b + mu a); kind 4 (beta from sc[3], no dot) ignores a, b, mu
cudaError_t launch_dot_shift_scalar(int kind, int64_t n, const double* a, const double* b, double mu, double* parts,
                                    double* sc, cudaStream_t st);
cudaError_t launch_pcg_xr(int64_t d, const double* sc, double mu, const double* p, const double* q, double* x,
                          double* r, double* parts, cudaStream_t st);
cudaError_t launch_pcg_p(int64_t d, const double* sc, const double* z, double* p, cudaStream_t st);
cudaError_t launch_scale_vec(int n, const double* f, double* c, cudaStream_t st);
cudaError_t launch_defl_coef(int n, int m, const double* K, const double* g, double* out, cudaStream_t st);
// Products with a d x nc basis held as FP32 head/tail arrays (column-major, ld ldv), in
// compensated FP32-pair arithmetic (about 2^-44 relative): g = V^T r (parts:
// defl_parts(d) x nc doubles) and z = r + V c (z may alias r).
int defl_parts(int64_t d);
cudaError_t launch_defl_t(int64_t d, int nc, const float* Vh, const float* Vl, int64_t ldv, const double* r,
                          double* parts, double* g, cudaStream_t st);
cudaError_t launch_defl_n(int64_t d, int nc, const float* Vh, const float* Vl, int64_t ldv, const double* coef,
                          const double* r, double* z, int sms, cudaStream_t st);
// p = r + V c + sc[2] p in one pass
cudaError_t launch_defl_np(int64_t d, int nc, const float* Vh, const float* Vl, int64_t ldv, const double* coef,
                           const double* sc, const double* r, double* p, int sms, cudaStream_t st);
// ---- on-the-fly RBF kernel (k_rbf.cu): Y = K X, K_ij = exp(-|x_i - x_j|^2 / (2 l^2))
// accurate to about 2^-46, compensated FP32-pair products; X is given as the FP32 head
// and tail of an FP64 block (launch_split_f64, ldx a multiple of 4), Y d x N FP64.
cudaError_t launch_rbf_apply(int64_t d, int N, const double* pts, int64_t ldp, double lengthscale, const float* Xh,
                             const float* Xl, int64_t ldx, double* Y, int64_t ldy, cudaStream_t st);
// ---- block-Lanczos drivers (k_krylov.cu)
cudaError_t launch_e1r0(int n, int mb, const double* R0, double* rhs, cudaStream_t st);
// CholQR step: R (upper, row-major) with Wb = Q R and Rinv = R^+ of the scaled Gram G
// (m <= 256; work: m x m doubles, scratch: 2 m doubles, keep: m flags, rank: kept count)
cudaError_t launch_chol_inv(int m, const double* G, double rank_tol, double* work, double* R, double* Rinv,
                            int* keep, int* rank, double* scratch, cudaStream_t st);
cudaError_t launch_band_put(int ldb, int bw, int m, int k, const double* A, const double* B, double* band,
                            cudaStream_t st);
// M = [B^T; A] (2m x m column-major, block precision) for the three-term recurrence
cudaError_t launch_three_term(int is_f64, int m, int first, const double* A, const double* B, void* M,
                              cudaStream_t st);
cudaError_t launch_band_solve(int n, int bw, const double* band, int ldb, int L, const double* mus,
                              const double* rhs, const int* rhs_col, int nrhs, double* work, double* Z, int* flags,
                              cudaStream_t st);
cudaError_t launch_band_mult(int n, int bw, const double* band, int ldb, double shift, const double* Y, int nc,
                             double* out, cudaStream_t st);
cudaError_t launch_band_gersh(int n, int bw, const double* band, int ldb, double* out, cudaStream_t st);
cudaError_t launch_combine_shifts(int n, int nc, int L, const double* Z, const double* c, double* Y,
                                  cudaStream_t st);
cudaError_t launch_lanczos_res(int n, int m, int L, int nrhs, const double* Blast, const double* Z, double* out,
                               cudaStream_t st);
cudaError_t launch_scale_cols(int is_f64, int64_t d, int m, int64_t ld, const double* scale, void* X,
                              cudaStream_t st);
cudaError_t launch_copy_cols(int in_f64, int out_f64, int64_t d, int m, const void* in, int64_t ldi, void* out,
                             int64_t ldo, cudaStream_t st);
cudaError_t launch_shift_residual(int64_t d, int L, const double* b, const double* AX, const double* X, int64_t ld,
                                  const double* mus, double* R, double* norms2, cudaStream_t st);
// Reset the control block for a new inner solve; c = e_1.
cudaError_t launch_init_state(DevState* state, int max_loads, double tol_abs, double* cvec, int m, cudaStream_t st);
// Norm partial count used by the residual launchers.
int residual_parts(int64_t d);

}  // namespace bk
