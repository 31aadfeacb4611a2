// Per-system descriptor of the batched block-CG (k_batch.cu, bk_batch_api.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bk_common.cuh"

namespace bk {

struct BSys {
  int64_t d, lda, ld;       // order, row stride of A, panel leading dimension of the blocks
  int m;                    // block width (<= the group's padded width)
  int cta0, ncta;           // thread-block range of this system in the block kernels
  int index;                // position in the caller's batch (Omega key offset)
  int active;               // runs an inner solve in the current refinement pass
  int max_loads;            // cap for the inner solve
  double tol_abs;           // inner target on ||R e_1|| = ||c||
  double rscale, rnorm;     // 1 / ||r|| and ||r|| of the current refinement residual
  double mu;
  const void* A;            // values in the block kernels' value type
  const void* A64;          // values as stored (FP64 residual)
  void *P, *Q, *Y;          // panel blocks (directions, residual basis, A_mu P)
  double *xin, *x64, *r64;  // inner iterate, solution, FP64 residual
  const double* b;
  double *Gp, *Sp;          // per-CTA Gram partials (entries x npG, entries x ncta)
  int npG;                  // partials of G: ncta, or the row tiles of the tensor-core product
  float* pt;                // P^T head/tail for the tensor-core product (or null)
  double* cvec;             // c = C e_1 (R = Q C), FP64
  void *gi_t, *xc_t;        // G^+ (mp x mp) and G^+ c (mp) in the block precision
  void *ti_t, *t_t;         // (T^+)^T and T (mp x mp, row-major) in the block precision
  DevState* st;
};

// Tensor-core block product for a group whose systems all qualify (FP32 values,
// 16-byte aligned rows): CTA i computes row tile tile_row[i] of system tile_sys[i];
// maps holds two CUtensorMaps per system (A, then P^T head/tail), 64-byte aligned.
struct BatchTc {
  const int* tile_sys = nullptr;
  const int* tile_row = nullptr;
  int ntiles = 0;
  const void* maps = nullptr;
  long long wait_cycles = 0;  // limit of each pipeline wait in SM clocks (0: the default)
};
cudaError_t launch_batch_dense_tc(int mp, BSys* sys, const int* cta_sys, int ncta, const BatchTc& tc,
                                  cudaStream_t st);
// Host: the two tensor maps of one system (A: d x d, row pitch lda; P^T: 2N x d, pitch
// round_up(d, 32)) written to out[0], out[1].
cudaError_t tc_make_maps(int mp, int64_t d, const float* A, int64_t lda, const float* pt, void* out);

// One block-CG step for every system of a group with padded width mp (tc: the group's
// tensor-core product, or null for the FFMA product, whose row tiles are tile_rows = 16
// or 32 rows per thread block).
cudaError_t launch_batch_step(int is_f64, int vals_f64, int mp, BSys* sys, int nsys, const int* cta_sys, int ncta,
                              double rank_tol, const BatchTc* tc, int tile_rows, cudaStream_t st);
// Start blocks of the active systems (Q = [r/||r||, Omega/sqrt(d)] normalised, P = Q,
// c = T e_1); resets their control blocks.
cudaError_t launch_batch_start(int is_f64, int mp, BSys* sys, int nsys, const int* cta_sys, int ncta, uint64_t seed,
                               double rank_tol, cudaStream_t st);
cudaError_t launch_batch_axpy(BSys* sys, const int* cta_sys, int ncta, cudaStream_t st);
cudaError_t launch_batch_resid(int vals_f64, BSys* sys, const int* cta_sys, int ncta, double* rnorm_parts,
                               cudaStream_t st);

}  // namespace bk
