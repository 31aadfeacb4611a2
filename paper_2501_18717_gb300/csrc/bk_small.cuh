// One-thread-block FP64 Cholesky factorisation with dropped dependent columns, shared by
// the single-system and batched small solves.
//
// On this part an FP64 instruction has a 64-cycle latency, a single warp issues at most
// one FP64 instruction per 64 cycles, and a square root or division is a dependent
// chain of several hundred cycles, so the factorisation is organised around its
// dependency chain: no pivot search (comparisons are FP64 instructions too), one thread
// forms 1/sqrt(pivot) by Newton steps, and the trailing update is spread over the warps
// of the block (the SM sub-partitions).
#pragma once

#include <cuda_runtime.h>

namespace bk {

constexpr int kSmallMax = 64;
constexpr int kLds = kSmallMax + 1;

struct SmallShared {
  double W[kSmallMax * kLds];
  double z[kSmallMax];
  double dscale[kSmallMax];
  double invd[kSmallMax];  // 1 / L[k][k]
  int perm[kSmallMax];
};


// 1/sqrt(x) for a positive normal FP64 x: an FP32 estimate of the argument brought
// into [1, 4) by an exact power-of-two scaling, then two Newton steps in FP64
// (r <- r (3 - x r^2) / 2 converges quadratically: about 1e-7 -> 1e-14 -> rounding).
__device__ __forceinline__ double rsqrt_newton(double x) {
  const int e = ((__double2hiint(x) >> 20) & 0x7ff) - 1023;
  const int h = e >> 1;  // floor(e / 2)
  const double xs = x * __hiloint2double((1023 - 2 * h) << 20, 0);
  double r = (double)rsqrtf((float)xs) * __hiloint2double((1023 - h) << 20, 0);
  r = r * fma(-0.5 * x, r * r, 1.5);
  r = r * fma(-0.5 * x, r * r, 1.5);
  return r;
}

// Cholesky of the unit-diagonal scaled matrix in the given column order; a pivot at
// or below rank_tol marks column k as numerically in the span of the kept columns
// before it: its row and column are dropped (invd[k] = 0) and the factorisation
// continues. A zero diagonal entry (a zero column of the block whose Gram this is) is
// dropped the same way. Returns the number of kept columns, or -1 for a negative or
// non-finite entry. On return the lower triangle of W holds the factor L of the scaled
// matrix (column k zero for a dropped k, row k as computed before the drop), z[i] =
// 1/sqrt(M_ii) (1 for a zero diagonal), dscale[i] = sqrt(M_ii) (0 for a zero diagonal)
// and invd[k] = 1 / L[k][k] (0 for dropped columns); M = (L^T D^{1/2})^T (L^T D^{1/2})
// on the kept columns, D = diag(dscale)^2.
template <int NTH>
__device__ int block_cholesky_skip(SmallShared& sh, int m, double rank_tol) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = NTH / 32;
  double* W = sh.W;
  __shared__ int s_bad, s_rank;
  if (tid == 0) {
    s_bad = 0;
    s_rank = 0;
  }
  __syncthreads();
  for (int i = tid; i < m; i += NTH) {
    const double g = W[i * kLds + i];
    const bool bad = g < 0.0 || !isfinite(g);
    if (bad) s_bad = 1;
    const bool pos = !bad && g > 0.0;
    const double r = pos ? rsqrt_newton(g) : 1.0;  // D^{-1/2}
    sh.z[i] = r;
    sh.dscale[i] = pos ? g * r : 0.0;  // sqrt(g)
  }
  __syncthreads();
  if (s_bad) return -1;
  for (int idx = tid; idx < m * m; idx += NTH) {
    const int r = idx / m, c = idx - r * m;
    W[r * kLds + c] *= sh.z[r] * sh.z[c];
  }
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    if (tid == 0) {
      const double x = W[k * kLds + k];
      const bool keep = x > rank_tol;
      double r = 0.0;
      if (keep) {
        r = rsqrt_newton(x);
        s_rank += 1;
      }
      W[k * kLds + k] = keep ? x * r : 0.0;
      sh.invd[k] = r;
      sh.perm[k] = keep;
    }
    __syncthreads();
    const double inv = sh.invd[k];  // 0 drops the column: L[:,k] = 0, no trailing update
    for (int i = k + 1 + tid; i < m; i += NTH) W[i * kLds + k] *= inv;
    __syncthreads();
    if (inv != 0.0) {
      for (int i = k + 1 + warp; i < m; i += NW) {
        const double lik = W[i * kLds + k];
        for (int j = k + 1 + lane; j <= i; j += 32) W[i * kLds + j] = fma(-lik, W[j * kLds + k], W[i * kLds + j]);
      }
    }
    __syncthreads();
  }
  return s_rank;
}

}  // namespace bk
