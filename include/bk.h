/*
 * bk.h -- C ABI of the randomized ("augmented") block-CG library for GB300 (sm_103a).
 *
 * The method: to solve A_mu x = b with A_mu = A + mu I, A symmetric positive
 * definite and mu >= 0 (paper Sec. 1, Eq. regularized_ls), run block-CG on the
 * augmented start block B = [b Omega], Omega a d x l Gaussian sketch, and keep the
 * iterate of the first column, bcg_t^(1)(mu) (Sec. 3, Def. BCG and Thm. main).
 * The iterate is the minimiser of the A_mu-norm error over the block Krylov space
 * K_t(A_mu, B); by Thm. main it is at least as accurate, after the same number of
 * passes over A ("matrix-loads", Sec. 1.2), as CG preconditioned by any Nystrom
 * preconditioner built from Omega.
 *
 * Conventions for every entry point
 *   - Memory: every array argument may be a host pointer or a device pointer of the
 *     context's device; the library detects which (cudaPointerGetAttributes) and
 *     copies host arrays through its own workspace. Arrays are borrowed for the call
 *     only; the caller keeps ownership. The library owns the context's workspace.
 *   - Layout: dense matrices are row-major with leading dimension ld (>= cols).
 *     Block vectors (d x m) are stored in panels of four columns: element (i, c) is at
 *     offset ((c / 4) * ld + i) * 4 + c % 4 (ld >= d rows per panel), so each row of a
 *     panel is one 16-byte (FP32) or 32-byte (FP64) vector. Columns m .. 4*ceil(m/4)-1
 *     of the last panel are padding: they are read, must hold finite values, and are
 *     written as zeros. CSR uses int32 rowptr (d+1 entries, rowptr[0] = 0) and int32
 *     colidx.
 *   - Streams: work is ordered on the context's stream. Each call returns after its
 *     results are complete (it synchronises that stream).
 *   - Errors: functions return a bk_status and never throw. On BK_ERR_* the outputs
 *     are undefined. BK_NOT_CONVERGED and BK_BREAKDOWN leave the best iterate so far
 *     in x. A CUDA error is reported as BK_ERR_CUDA and leaves the context usable
 *     unless the CUDA context itself was lost.
 *   - Threads: a context is not thread-safe; use one context per host thread.
 */
#ifndef BK_H
#define BK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bk_ctx bk_ctx;

typedef enum {
  BK_OK = 0,
  BK_ERR_ARG = 1,          /* invalid argument (null pointer, bad size, bad enum) */
  BK_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  BK_ERR_OOM = 3,          /* device workspace could not be allocated */
  BK_NOT_CONVERGED = 4,    /* max_loads or max_refine reached before tol */
  BK_BREAKDOWN = 5,        /* a block Gram matrix lost positive definiteness */
  BK_STAGNATED = 6,        /* refinement stopped reducing the FP64 residual */
  BK_TIMEOUT = 7,          /* reserved: a device wait ran past its limit */
  BK_ERR_UNSUPPORTED = 8,  /* operator kind / dtype / width not built */
  BK_ERR_TOO_LARGE = 9     /* the call needs more than the fixed static scratch holds */
} bk_status;

typedef enum { BK_DENSE = 0, BK_CSR = 1, BK_GRAM = 2, BK_RBF = 3 } bk_op_kind;
typedef enum { BK_F64 = 0, BK_F32 = 1 } bk_dtype;

/* Precision of the inner block-CG iteration (block vectors, block products,
 * updates). Gram matrices, the small Cholesky solves, the solution accumulator and
 * the refinement residual are FP64 in every mode.
 *   BK_PREC_F32X2: FP64 blocks; block products of FP32-stored values (16-byte aligned
 *   rows) in compensated FP32-pair arithmetic on the FP32 pipe (each product exact,
 *   sums to about 2^-44 of sum |a_ik p_k|), and the basis products (reorthogonalisation,
 *   block QR) in the same arithmetic; the Grams that give T_t, the band solves and the
 *   refinement stay FP64. Lanczos drivers only (bk_ridge_path, bk_sample,
 *   bk_sample_isqrt); bk_solve and bk_solve_batched return BK_ERR_UNSUPPORTED.
 *   BK_PREC_BF16: FP32 blocks; the block products of a Gram-form operator (BK_GRAM,
 *   FP32 or FP64 Z, promoted to FP32) run on the BF16 tensor cores with FP32
 *   accumulation. Z is split once per call into a BF16 head and tail (a row-major and
 *   a transposed copy, 4 n d bytes each) and the block likewise at every product; a
 *   product is the sum of the three head/tail products, about 2^-16 of
 *   sum |z_ik x_k|. The refinement residual stays FP64-accurate: its products with
 *   the stored Z run on the BF16 tensor cores too, through the error-free digit
 *   splitting of bk_apply_ozaki (digits of Z and Z^T made once per call, 28 n d
 *   bytes), under the same accuracy guard as the compensated FP32-pair products
 *   (and in FP64 GEMMs once a pass stops reducing the residual). bk_ridge_path
 *   only, with at most 128 block columns;
 *   other entry points and operator kinds return BK_ERR_UNSUPPORTED.
 *   BK_PREC_OZAKI: FP64 blocks; the block products of a stored dense FP32 operator and
 *   the FP64 basis products (the Grams that give T_t, the reorthogonalisation, the
 *   three-term step, Q = W R^{-1}) run on the BF16 tensor cores through an error-free
 *   splitting (Ozaki, Ogita and Oishi, 2012; see bk_apply_ozaki for the digits and the
 *   error bound: 2^-45 of the block bounds, the order of an FP64 GEMM's rounding over
 *   K = d). The digits of the operator (7 planes of BF16, 14 d^2 bytes) are made once
 *   per call, those of each basis product's operands at the product. bk_sample and bk_sample_isqrt with a BK_DENSE FP32 operator only; other
 *   entry points and operators return BK_ERR_UNSUPPORTED. */
typedef enum {
  BK_PREC_FP64 = 0,
  BK_PREC_FP32 = 1,
  BK_PREC_F32X2 = 2,
  BK_PREC_BF16 = 3,
  BK_PREC_OZAKI = 4
} bk_prec;

/* The matrix A (without the shift mu).
 *   BK_DENSE: vals is rows x cols row-major with leading dimension ld, rows = cols = d.
 *   BK_CSR:   rowptr[rows+1], colidx[nnz], vals[nnz]; rows = cols = d; ld ignored.
 *   BK_GRAM:  A = Z^T Z applied matrix-free as Z^T (Z P) (ridge regression, Sec. 1);
 *             vals is Z, rows x cols row-major with leading dimension ld; d = cols.
 *             Accepted by bk_ridge_path and bk_sample.
 *   BK_RBF:   K_ij = exp(-||x_i - x_j||^2 / (2 param^2)) formed on the fly, never stored
 *             (the matrix-free access mode of Sec. 1): vals is d points of 3 FP64
 *             coordinates, row stride ld >= 3, rows = cols = d, dtype BK_F64, param > 0
 *             the lengthscale. Each entry exp(t) is evaluated in FP32-pair arithmetic
 *             from the FP64 exponent t: relative error about 2^-46 for t >= -70;
 *             below, the pair's tail leaves the FP32 normal range and the absolute
 *             error stays under 2^-126; entries with t < -100 are 0. Products in
 *             compensated FP32 pairs (about 2^-44). Accepted by bk_sample,
 *             bk_sample_isqrt (FP64 blocks: inner BK_PREC_FP64 or BK_PREC_F32X2) and
 *             bk_apply.
 *   dtype gives the element type of vals. A must be symmetric positive definite
 *   (or positive semi-definite with mu > 0); the library does not check symmetry. */
typedef struct {
  int32_t kind;           /* bk_op_kind */
  int32_t dtype;          /* bk_dtype of vals */
  int64_t rows, cols, ld;
  const void* vals;
  const int32_t* rowptr;
  const int32_t* colidx;
  int64_t nnz;
  double param;           /* BK_RBF: the lengthscale; ignored by the other kinds */
} bk_operator;

typedef struct {
  double tol;             /* stop when ||b - A_mu x||_2 <= tol ||b||_2, the residual
                             recomputed in FP64 from the stored A (Sec. 4 remark on
                             a-posteriori residual checks) */
  int32_t max_loads;      /* cap on block products over all refinement steps */
  int32_t sketch;         /* l, the columns of Omega; block width m = l + 1 (<= 64) */
  uint64_t seed;          /* Philox4x32-10 key of Omega (stream 3, see bk_gaussian) */
  int32_t inner;          /* bk_prec of the inner iteration */
  double inner_tol;       /* inner solve stops when its column-0 residual has been
                             reduced by this factor (or enough to meet tol) */
  int32_t max_refine;     /* cap on FP64 refinement restarts */
  int32_t check_every;    /* block products between host polls of the device flag */
  int32_t profile;        /* nonzero: time every step kernel with CUDA events recorded
                             between launches (kept inside the CUDA graph) and report
                             the sums in bk_info.ms_kernel / launches */
  int64_t timeout_cycles; /* limit, in SM clock cycles, of each bounded wait of the
                             tensor-core block products on their copy and MMA
                             pipeline barriers (bk_solve, bk_solve_batched); 0 = the
                             library default of 4e9 cycles (about 2 s). A wait that
                             gives up makes the kernel drain the copies and MMAs it
                             has issued, free its tensor memory and return; the call
                             then returns BK_TIMEOUT and the context stays usable.
                             Negative values are BK_ERR_ARG. */
} bk_opts;

/* Kernel classes reported by a profiled solve. */
enum {
  BK_K_OPERATOR = 0,  /* block product Y = A_mu P with the Gram P^T Y */
  BK_K_REDUCE = 1,    /* Gram partial reductions (both per step) */
  BK_K_ALPHA = 2,     /* small solve alpha = G^+ S */
  BK_K_UPDATE_R = 3,  /* R -= Y alpha with the Gram R^T R */
  BK_K_BETA = 4,      /* residual test and small solve beta = S^+ S' */
  BK_K_UPDATE_P = 5,  /* x += P alpha e_1, P = R + P beta */
  BK_K_RESIDUAL = 6,  /* Lanczos drivers: FP64-accurate refinement residual products */
  BK_K_ORTH = 7,      /* Lanczos drivers: reorthogonalisation, block QR and Grams */
  BK_K_CLASSES = 8
};

typedef struct {
  int32_t status;         /* bk_status of the call */
  int32_t loads;          /* block products applied (the paper's matrix-loads) */
  int32_t refinements;    /* inner solves run (1 = no restart was needed) */
  int32_t residual_loads; /* single-column FP64 residual products */
  double rel_residual;    /* final ||b - A_mu x|| / ||b|| in FP64 */
  double ms_total;        /* wall time of the call on the context stream */
  double ms_kernel[8];    /* profiled solves: summed kernel time per class (BK_K_*) */
  int32_t launches[8];    /* profiled solves: active launches per class */
  int32_t kernel_launches;/* all kernels this call launched, including graph replays
                             and steps that found the solve already finished */
  int32_t deflations;     /* bk_solve, bk_solve_batched: block columns dropped as
                             numerically dependent (rank test of the small
                             factorisation of R^T R), summed over the inner solves; a
                             dropped column stays out until the next restart */
  int32_t fp64_fallback;  /* bk_solve, bk_solve_batched with BK_PREC_FP32: 1 if the
                             FP32-block passes stopped reducing the FP64 residual and
                             the rest of the solve ran in FP64 blocks */
} bk_info;

/* Fills *opts with defaults: tol 1e-10, max_loads 20000, sketch 20, seed 0,
 * inner FP64, inner_tol 1e-6, max_refine 8, check_every 8, profile 0. */
void bk_default_opts(bk_opts* opts);

/* Creates a context on CUDA device `device`, ordering work on `cuda_stream` (a
 * cudaStream_t). NULL makes the context create its own blocking stream, which is
 * ordered with the legacy default stream (needed because the solve captures its
 * step sequence into a CUDA graph, which the legacy stream does not allow). */
bk_status bk_create(bk_ctx** ctx, int device, void* cuda_stream);
bk_status bk_destroy(bk_ctx* ctx);
bk_status bk_set_stream(bk_ctx* ctx, void* cuda_stream);
const char* bk_status_string(bk_status s);
/* Text of the last CUDA failure seen by a call on this context ("" if none). The
 * string is owned by the context and valid until its next call. */
const char* bk_last_error(const bk_ctx* ctx);

/* Solves A_mu x = b by randomized block-CG on [b Omega] with FP64 residual
 * refinement (Def. BCG, Thm. main; stopping rule of the Sec. 4 remark).
 *   A    operator descriptor (see bk_operator)
 *   mu   shift, >= 0
 *   b    d doubles
 *   x    d doubles; output. Its input value is ignored (the solve starts at 0).
 *   opts NULL for defaults
 *   info may be NULL
 * With inner = BK_PREC_FP32 the block products use an FP32 copy of the values
 * (made by the library from FP64 values, or the values themselves when dtype is
 * FP32) and the refinement residual uses the values as given. Dense FP32 products run
 * on the tensor cores (TF32 with split operands and FP32 sums of 32-wide K slices,
 * FP32 accuracy) when the rows are 16-byte aligned (base 16-byte aligned, ld a
 * multiple of 4; the library's own FP32 copy always is), else on FFMA.
 * Each refinement pass forms x + ||r|| x_inner and its FP64 residual. An inner solve
 * stops as a breakdown when its recurrence estimate ||c|| is not finite or above 1e8
 * (the finite-precision recurrence lost orthogonality); a pass whose residual is not
 * finite, or that broke down without reducing it, is discarded (x stays as it was)
 * and ends the solve with BK_BREAKDOWN, and a second pass that reduces the residual
 * less than twofold ends it with BK_STAGNATED. With FP32 blocks either case instead
 * hands the rest of the solve to FP64 blocks on the residual system A_mu delta = r,
 * x <- x + delta (info->fp64_fallback = 1). FP32 blocks wider than about 48 on systems
 * of a few hundred unknowns, where a few loads exhaust the space, are the case seen
 * to need it.
 * Returns BK_TIMEOUT (x holds the last refined iterate) if a tensor-core pipeline
 * wait gave up. */
bk_status bk_solve(bk_ctx* ctx, const bk_operator* A, double mu, const double* b, double* x,
                   const bk_opts* opts, bk_info* info);

/* The whole ridge-regression path (Sec. 1, Sec. 3.2 Eq. bcg_alg, Thm. cost): for every
 * shift mu_j, X[:, j] ~= (A + mu_j I)^{-1} b, all from one block-Lanczos basis of
 * K_t(A, [b Omega]) with full reorthogonalisation (shift invariance, Eq.
 * shift_invariance). T_t is block tridiagonal with half-bandwidth m; the L shifted
 * banded systems (T_t + mu_j I) z_j = ||b|| e_1 are solved in one launch (one thread
 * block per shift, FP64) and combined as X = Q_t [z_1 .. z_L]. The run stops when the
 * Lanczos residual estimate ||B_t z_j,last|| of every shift meets the inner target.
 * FP64 refinement: the residuals r_j = b - (A + mu_j) x_j are formed from the stored
 * values to FP64 accuracy (FP32 values: compensated FP32-pair products while their
 * estimated error 1e-13 ||A|| ||X|| stays below tol ||b|| / 10, else, or once a basis
 * stops reducing the residual, FP64 products); while max_j ||r_j|| > tol ||b||, a
 * block-Lanczos basis of the residual block [r_1 .. r_L] (block width L) gives every
 * correction at once and x_j is updated. A shifted projected system that is not
 * positive definite (only through rounding in the basis) drops its non-positive pivots;
 * an FP32 run that meets one builds its later bases in FP64 blocks with FP64-accurate
 * products.
 *   A      BK_DENSE or BK_GRAM, FP32 or FP64 values (FP32 runs use FP32 values; FP64
 *          values are rounded by the library for them)
 *   L      number of shifts, 1 <= L <= 1024; mus: L shifts >= 0 (host or device)
 *   b      d doubles; X: d x L doubles, column-major (leading dimension d), output
 *   opts   sketch (l, block width l + 1 <= 256), seed, tol (relative residual of every
 *          shift), inner (bk_prec of the basis and products), inner_tol, max_loads (cap
 *          on operator applications per basis), max_refine (bases built), check_every,
 *          profile (CUDA-event sums per group in ms_kernel / launches: BK_K_OPERATOR,
 *          BK_K_RESIDUAL, BK_K_ORTH)
 *   info   loads (all bases), refinements (bases built), rel_residual (worst shift)
 * Returns BK_NOT_CONVERGED if the worst shift misses tol after max_refine bases. */
bk_status bk_ridge_path(bk_ctx* ctx, const bk_operator* A, int32_t L, const double* mus, const double* b,
                        double* X, const bk_opts* opts, bk_info* info);

/* Gaussian sampling S ~= (K + nugget I)^{1/2} B by the block-Lanczos square root of
 * Def. blansq (Sec. 5): block-Lanczos with full reorthogonalisation on (K, B) (block
 * width m, the samples themselves are the start block), then
 *   S = (2/pi) int_0^inf A bcg_t(z^2) dz,  A = K + nugget I,
 * evaluated with the quadrature of bk_sqrt_quadrature on [nugget, Gershgorin bound of
 * T_t + nugget] and the Lanczos relation A Q_t = Q_t T_t + Q_{t+1} B_t E_t^T:
 *   S = Q_t (T_t + nugget) Ybar + Q_{t+1} B_t E_t^T Ybar,  Ybar = sum_j w_j Y_j,
 *   Y_j = (T_t + (nugget + z_j^2) I)^{-1} E_1 R_0  (all n_quad shifts in one launch).
 * Stops when S changes by at most tol (relative Frobenius norm) between checks made
 * every check_every loads, or when K_t fills R^d.
 *   K      BK_DENSE or BK_GRAM (FP32 or FP64 values); nugget >= 0 (if 0, K must be
 *          positive definite and the interval starts at 1e-12 times its upper end)
 *   B      d x m column-major doubles (host or device), 1 <= m <= 256; S: d x m output
 *   n_quad quadrature nodes (1..1024; 32 gives about 1e-12 for a spectral ratio of 1e8)
 *   info   loads, refinements (= checks made), rel_residual (= last relative change)
 * Returns BK_BREAKDOWN if a shifted projected system T_t + (nugget + z_j^2) I is not
 * positive definite (K + nugget I indefinite in its stored precision). */
bk_status bk_sample(bk_ctx* ctx, const bk_operator* K, double nugget, int32_t m, const double* B, double* S,
                    int32_t n_quad, const bk_opts* opts, bk_info* info);

/* Inverse square root S ~= (K + nugget I)^{-1/2} B (Sec. 5, the whitening counterpart of
 * bk_sample): the same block-Lanczos basis, shifts and weights as bk_sample, since
 * (2/pi) int_0^inf (A + z^2 I)^{-1} dz = A^{-1/2}; S = Q_t Ybar with
 * Ybar = sum_j w_j (T_t + (nugget + z_j^2) I)^{-1} E_1 R_0. Arguments, stopping rule and
 * status as bk_sample. */
bk_status bk_sample_isqrt(bk_ctx* ctx, const bk_operator* K, double nugget, int32_t m, const double* B, double* S,
                          int32_t n_quad, const bk_opts* opts, bk_info* info);

/* Nystrom-preconditioned CG, the comparator of Thm. main (Def. PCG, preconditioner of
 * Eq. precond_def): the block-Krylov Nystrom approximation A<K_s> of Eq. nystromBKI_def
 * from the sketch Omega of opts (d x sketch Gaussian, the same Philox key and stream as
 * bk_solve's, so both methods see the same Omega), theta = its smallest eigenvalue
 * (Sec. 7), P^{-1} = (theta + mu) U (D + mu)^{-1} U^T + (I - U U^T), then PCG from
 * x = 0 on (A + mu I) x = b, on the device: vectors and scalars in FP64, the
 * preconditioner's products with U in compensated FP32-pair arithmetic on a copy of U
 * split once into FP32 head and tail arrays (about 2^-44 relative). The approximation comes
 * from s_ny block-Lanczos steps on Omega (s_ny loads): with V = [Q_0 .. Q_{s-1}] and the
 * Lanczos relation A V = V T + Q_s B E_s^T, the factor F = A V (V^T A V)^{+1/2} is
 * [V Q_s] H for a small H, so U and D follow from two small eigendecompositions on
 * the host (cyclic Jacobi) and one d x r product.
 *   A      BK_DENSE, BK_GRAM or BK_CSR; FP64 or FP32 values (promoted: FP32 dense and
 *          Gram products use the compensated FP32-pair kernels, about 2^-44 relative)
 *   s_ny   Krylov depth of the approximation, 1..16 (s_ny = 1 is the plain Nystrom
 *          approximation A Omega (Omega^T A Omega)^+ Omega^T A)
 *   b, x   d doubles (host or device); x is output (x_0 = 0)
 *   opts   sketch (columns of Omega, <= 256), seed, tol (stop when the recurrence
 *          residual meets tol ||b|| and the residual recomputed from the stored values
 *          confirms it; checked every check_every iterations), max_loads (cap on
 *          s_ny + PCG iterations)
 *   info   loads (s_ny + iterations), refinements (rank r of the approximation),
 *          residual_loads (recomputed residual checks), rel_residual (recomputed)
 * Returns BK_NOT_CONVERGED at the load cap (x holds the last iterate), BK_BREAKDOWN if
 * p^T A_mu p or r^T z stopped being positive. */
bk_status bk_nystrom_pcg(bk_ctx* ctx, const bk_operator* A, double mu, const double* b, double* x, int32_t s_ny,
                         const bk_opts* opts, bk_info* info);

/* Block-CG whose block shrinks to one column after s_lock steps (the outlook's
 * deflation to a smaller block; Sec. CG_pro's scheme of full reorthogonalisation for
 * the first blocks and orthogonalisation against only those afterwards), for
 * (A + mu I) x = b:
 *   1. s_lock block-Lanczos steps with full reorthogonalisation on [b Omega] (block width
 *      m = 1 + sketch; Omega as bk_solve's) lock V = [Q_0 .. Q_{s-1}], an orthonormal
 *      basis of K_s(A, [b Omega]), and T_s = V^T A V; x_0 = V (T_s + mu I)^{-1} V^T b is
 *      the block-CG iterate after s_lock loads (Eq. bcg_alg), r_0 = b - A_mu x_0.
 *   2. one-column deflated CG with deflation space V (Def-CG of Saad, Yeung, Erhel and
 *      Guyomarc'h, SIAM J. Sci. Comput. 21, 2000): directions are kept A_mu-orthogonal
 *      to V and residuals orthogonal to it, with the coefficients
 *      (T_s + mu I)^{-1} (A_mu V)^T r = V^T r + K Q_s^T r, K = (T_s + mu I)^{-1} E_s B_s^T,
 *      from the Lanczos relation A V = V T_s + Q_s B_s E_s^T (no stored A V). Each
 *      iteration is one single-column load plus one pass over [V Q_s] (d x (s + 1) m)
 *      and one over V (d x s m), on a copy of the basis split once into FP32 head and
 *      tail arrays, in compensated FP32-pair arithmetic (about 2^-44 relative; FP64
 *      FMAs would bound these products by the FP64 pipe).
 * The iterate after j deflated steps minimises the A_mu-norm error over
 * span(V) + K_j(P A_mu, r_0), P = I - A_mu V (V^T A_mu V)^{-1} V^T.
 *   A      BK_DENSE, BK_GRAM, BK_CSR or BK_RBF; FP64 or FP32 values (promoted; FP32 dense
 *          and Gram single-column products use the compensated FP32-pair kernels)
 *   s_lock locked block steps, 1..16; (s_lock + 1)(1 + sketch) <= 768
 *   b, x   d doubles (host or device); x is output
 *   opts   sketch (>= 0; 0 gives CG with s_lock locked Lanczos vectors), seed, tol (stop
 *          when the recurrence residual meets tol ||b|| and the FP64 residual recomputed
 *          from the stored values confirms it; checked every check_every iterations),
 *          max_loads (cap on s_lock + 1 + iterations, counting block loads as one)
 *   info   loads (s_lock block loads, the load for r_0, one per iteration),
 *          refinements (columns of the locked basis, s_lock m), residual_loads
 *          (recomputed residual checks), rel_residual (recomputed)
 * Returns BK_NOT_CONVERGED at the load cap (x holds the last iterate), BK_BREAKDOWN if
 * T_s + mu I is not positive definite or p^T A_mu p or r^T r stopped being positive,
 * BK_ERR_UNSUPPORTED if (s_lock + 1)(1 + sketch) > 768. */
bk_status bk_solve_shrink(bk_ctx* ctx, const bk_operator* A, double mu, const double* b, double* x, int32_t s_lock,
                          const bk_opts* opts, bk_info* info);

/* Many independent systems (A_i + mu_i I) x_i = b_i of uneven size, i < n, solved
 * together (bk_solve on each, batched): systems are grouped by padded block width and
 * every step of the block-CG recurrence (Def. BCG) runs as one launch over all systems
 * of a group, each system owning thread blocks in proportion to d_i^2 m_i; a chunk of
 * check_every steps is replayed as a CUDA graph and systems that have converged skip
 * their work. FP64 refinement restarts as in bk_solve, with the same stopping rules
 * per system (a pass that lost its recurrence is undone and stops that system; two
 * passes that reduce its residual less than twofold stop it). With FP32 blocks, the
 * systems stopped that way are solved again from x = 0 in FP64 blocks, in one nested
 * batch (their info->fp64_fallback = 1; loads and passes add up).
 *   A      n dense operators, all FP32 or all FP64 values (BK_DENSE only). With FP32
 *          blocks, a width group whose matrices all have 16-byte aligned rows (device
 *          base 16-byte aligned, ld a multiple of 4) runs its block products on the
 *          tensor cores (TF32 with split operands, FP32 accuracy); otherwise on FFMA.
 *   mu     n shifts (host array); b, x: n pointers to d_i doubles (host or device)
 *   opts   as bk_solve; sketch = -1 takes the block width per system from the table that
 *          bk_autotune filled in this context (nearest size bucket floor(log2 d); 16
 *          when the table is empty)
 *   info   n records (may be NULL); ms_total is the whole batch
 * Returns BK_NOT_CONVERGED if any system missed tol. */
bk_status bk_solve_batched(bk_ctx* ctx, int32_t n, const bk_operator* A, const double* mu, const double* const* b,
                           double* const* x, const bk_opts* opts, bk_info* info);

/* Chooses the sketch size per size bucket (floor(log2 d)) from timed calibration
 * solves and stores the table in the context; bk_solve_batched uses it when
 * opts->sketch = -1. A candidate whose block width the kernels are not built for
 * (bk_solve_batched: BK_ERR_UNSUPPORTED) is skipped. For the winning sketch the
 * bucket's block-product kernel and tile shape are chosen too: the default (the
 * tensor-core product, 128-row tiles, TMA ring, split TF32, for FP32 blocks at widths
 * it is built for; else the CUDA-core product with 16-row x 64-column tiles through
 * shared memory) is timed against the other choices (the CUDA-core product with 16-row
 * and with 32-row tiles) and the fastest is kept. The calibration systems of each
 * bucket are solved together with bk_solve_batched, repeated in one batch until it
 * streams about 1 GB of matrix per
 * block product (at most 64 copies), so the timing reflects throughput inside a large
 * batch; each candidate is timed as the best of three solves after a warm one, and
 * the fastest candidate that converges on every system wins. Calibrate on systems
 * drawn independently of the ones to be solved. chosen (n ints, may be NULL) receives
 * the pick per system. Host memory for the copies' x vectors is allocated here. */
bk_status bk_autotune(bk_ctx* ctx, int32_t n, const bk_operator* A, const double* mu, const double* const* b,
                      const int32_t* candidates, int32_t ncand, const bk_opts* opts, int32_t* chosen);

/* The autotune table of a context as a text file (one line per size bucket:
 * floor(log2 d), sketch, product kernel 1 = tensor-core, 0 = CUDA-core with 16-row
 * tiles, 2 = CUDA-core with 32-row tiles), so that a calibration can be reused by
 * later contexts and processes. bk_autotune_load replaces
 * the context's table with the file's; it returns BK_ERR_ARG (table unchanged) for a
 * file it cannot open or a malformed line. Host-only calls. */
bk_status bk_autotune_save(const bk_ctx* ctx, const char* path);
bk_status bk_autotune_load(bk_ctx* ctx, const char* path);

/* Quadrature for the square root (Sec. 1, Eq. sqrt_rational; Sec. 5 Def. blansq):
 * nodes z_j^2 and weights w_j, j < n, with
 *     sqrt(lambda) ~= sum_j w_j lambda / (lambda + z_j^2)   for lambda in [lo, hi],
 * from the substitution z = sqrt(lo) sc(u | 1 - lo/hi), which maps [0, inf) onto
 * [0, K(1 - lo/hi)] with dz / sqrt((lo + z^2)(hi + z^2)) = du / sqrt(hi) (the identity of
 * Eq. ellipticK_eval), and the midpoint rule in u. The error decays geometrically in
 * n: about 1e-12 relative at n = 32 for hi/lo = 1e8. Host computation (no device use):
 * K by the arithmetic-geometric mean, sn/cn/dn by the descending recursion of
 * Abramowitz & Stegun 16.4. z2, w: n doubles each (host). 0 < lo <= hi. */
bk_status bk_sqrt_quadrature(double lo, double hi, int32_t n, double* z2, double* w);

/* Y = A X + mu X for L columns in FP64 (one "matrix-load" of Sec. 1.2 at the accuracy of
 * the FP64 refinement residual). X and Y are d x L column-major with leading dimensions
 * ldx, ldy >= d, host or device (host arrays are staged through the context workspace;
 * the call synchronises the context stream before it returns). A may be BK_DENSE,
 * BK_CSR, BK_GRAM (d = cols) or BK_RBF. The products are FP64-accurate: FP64 values
 * through FP64 products; FP32-stored dense and Gram-form values, promoted, through
 * compensated FP32-pair products (about 2^-44 relative to sum |a_ik x_k|, 16-byte
 * aligned rows with ld a multiple of 4; FP64 products otherwise); BK_RBF entries formed
 * on the fly as described for BK_RBF. Returns BK_ERR_ARG for a null pointer, L < 1, a
 * leading dimension below d or a non-finite mu, and the operator's checks as in
 * bk_solve / bk_sample. */
bk_status bk_apply(bk_ctx* ctx, const bk_operator* A, double mu, int32_t L, const double* X, int64_t ldx,
                   double* Y, int64_t ldy);

/* Y = A X + mu X in FP64 for a dense FP32-stored A (BK_DENSE, dtype BK_F32) or a Gram-
 * form A = Z^T Z (BK_GRAM, FP32 or FP64 Z: Y = Z^T (Z X) + mu X, both products split;
 * host or device arrays as in bk_apply), on the BF16 tensor cores by an error-free
 * splitting in the manner of Ozaki, Ogita and Oishi (2012): the product of the
 * BK_PREC_OZAKI loads and of the BK_PREC_BF16 refinement residuals. The paper prescribes no product algorithm; this is a GB300
 * implementation of its FP64-accurate matrix-load (Sec. 1.2, Sec. 5).
 * Each row of A and each column of X is cut into blocks of 512 consecutive elements;
 * a block whose largest magnitude is below 2^e is written as 2^e sum_i a_i 2^-(6+7i)
 * with 7 integer digits |a_i| <= 64 (exact in BF16), which keeps every value to
 * 2^-49 of 2^e. The digit products with i + j <= 6 are accumulated per block on the
 * tensor cores, where every partial sum is an integer below 2^24 and so exact; the
 * blocks are added in unevaluated FP32 pairs. Error of entry i of Y: at most about
 * 2^-45 sum_k 2^eA(i,k) 2^eX(k), where 2^eA(i,k) and 2^eX(k) bound the blocks that
 * a_ik and x_k fall in; this equals 2^-45 sum_k |a_ik x_k| up to the spread of the
 * magnitudes within a block (a factor 4 when they lie within a factor 2 of its
 * largest), not for blocks of very uneven magnitudes. The digits of A (7 d^2 BF16
 * values, 14 d^2 bytes; for Z, of Z and Z^T, 28 n d bytes; in the context workspace)
 * are made at every call; the drivers make them once per call.
 * Y and X have leading dimensions ldy, ldx >= d and L columns (L <= 4096). Returns
 * BK_ERR_UNSUPPORTED for other operators, BK_TIMEOUT if a pipeline wait gave up. */
bk_status bk_apply_ozaki(bk_ctx* ctx, const bk_operator* A, double mu, int32_t L, const double* X, int64_t ldx,
                         double* Y, int64_t ldy);

/* One block product with its Gram matrix (one "matrix-load", Sec. 1.2):
 *   Y = A P + mu P  and  G = P^T Y  (m x m, FP64, row-major).
 * P and Y are d x m blocks in the panel layout above (leading dimension ld), element type `dtype`
 * (BK_F64 or BK_F32; for BK_F32 the operator values are rounded to FP32 first if
 * they are FP64). 1 <= m <= 64. G accumulates FP32 products in FP32 over row tiles
 * and in FP64 across tiles when dtype is BK_F32. */
bk_status bk_block_apply(bk_ctx* ctx, const bk_operator* A, double mu, int32_t dtype, int64_t m,
                         const void* P, void* Y, int64_t ld, double* G);

/* G = X^T Y for d x m blocks X, Y in the panel layout (leading dimension ld, element
 * type dtype); G is m x m FP64 row-major. */
bk_status bk_gram(bk_ctx* ctx, int32_t dtype, int64_t d, int64_t m, const void* X, const void* Y,
                  int64_t ld, double* G);

/* X = G^{-1} S for a symmetric positive definite m x m G (the small factor/solve of
 * each block-CG step): Cholesky of D^{-1/2} G D^{-1/2} (D = diag G) with diagonal
 * pivoting, one warp per column of S. G, S, X are m x m FP64 row-major. Returns
 * BK_BREAKDOWN if G is numerically rank deficient (a scaled pivot below 1e-14) or has
 * a non-positive diagonal entry. 1 <= m <= 64. */
bk_status bk_chol_solve(bk_ctx* ctx, int64_t m, const double* G, const double* S, double* X);

/* Standard normals k = offset .. offset+n-1 of Philox4x32-10 stream `stream` with
 * key `seed`, by Box-Muller, as defined for the sketch Omega:
 *   block c = k / 2; counter (c mod 2^32, c / 2^32, stream, 0); key (seed mod 2^32,
 *   seed / 2^32); u1 = ((x0>>5) 2^26 + (x1>>6) + 1/2) 2^-53, u2 likewise from x2, x3;
 *   value = sqrt(-2 ln u1) cos(2 pi u2) for even k, sin for odd k.
 * Omega (d x l) is entry k = j d + i of stream 3. out has n doubles. */
bk_status bk_gaussian(bk_ctx* ctx, uint64_t seed, uint32_t stream, int64_t n, int64_t offset,
                      double* out);

/* bk_block_apply without any device allocation. The paper has no counterpart: this
 * entry point exists for callers that cannot let a library allocate device memory,
 * such as a host framework that owns every device allocation through its own pool and
 * budget (a library cudaMalloc would be invisible to it), or a latency-sensitive caller
 * that cannot afford the device-wide synchronisation a cudaMalloc or cudaFree implies.
 *
 * It computes the same Y = A P + mu P and G = P^T Y as bk_block_apply and checks its
 * arguments by the same rules, but takes no context and allocates nothing. CSR
 * operators and FP64 dense operators run the same kernels and launch shape as
 * bk_block_apply. FP32 dense operators always run the CUDA-core dense kernel here,
 * while bk_block_apply may take the tensor-core product for them (it needs a scratch
 * copy of P), so the two round differently within the FP32 tolerance.
 *   - every array (A's arrays, P, Y, G) must be device memory of the current device
 *     (BK_ERR_ARG otherwise, also for memory of another GPU): there is no staging copy;
 *   - A->dtype must equal dtype (BK_ERR_UNSUPPORTED otherwise): there is no converted
 *     copy of the values;
 *   - the Gram partials use a fixed scratch array of 4 MiB (2^19 doubles) compiled into
 *     the library as a __device__ variable. Each device that loads the library holds it
 *     until the process exits. A call whose partials would not fit (more CTAs times
 *     Gram entries than 2^19) returns BK_ERR_TOO_LARGE; on GB300 every supported size
 *     fits.
 * The first call on a device does a one-time set-up: it looks up the scratch address
 * (cudaGetSymbolAddress) with that device current. Make that first call before any
 * stream capture. All calls share the scratch, so calls whose kernels overlap on the
 * GPU (different streams or host threads, same device) race on it and must be
 * serialised by the caller. Each call rewrites every partial it reads, so no clearing
 * is needed. Work is enqueued on `cuda_stream` (a cudaStream_t, NULL for the legacy
 * default stream), and the call synchronises that stream before it returns.
 * 1 <= m <= 36. */
bk_status bk_block_apply_static(const bk_operator* A, double mu, int32_t dtype, int64_t m, const void* P,
                                void* Y, int64_t ld, double* G, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* BK_H */
