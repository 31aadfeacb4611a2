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

constexpr int kSmallMax = 68;  // widest padded block
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

// 1/x for a positive FP64 pivot. On this part the FP64 conversions and fused
// multiply-adds are long-latency instructions on the critical path of every column,
// so the estimate is formed with integer operations: x's exponent and top 20 mantissa
// bits as an FP32 value, its FP32 reciprocal, and that widened back to FP64 (exact).
// The estimate's relative error e0 is below 2^-19. One third-order Newton step,
// r (1 + e + e^2) with e = 1 - x r, leaves e0^3 < 2^-57 plus rounding: three dependent
// fused multiply-adds. Pivots outside the FP32 exponent range take an FP64 division.
__device__ __forceinline__ double recip_pivot(double x) {
  const int hi = __double2hiint(x);
  const int e = ((hi >> 20) & 0x7ff) - 1023;
  if (e < -125 || e > 125) return 1.0 / x;
  const float xf = __uint_as_float(((unsigned)(e + 127) << 23) | ((unsigned)(hi & 0xfffff) << 3));
  const unsigned rb = __float_as_uint(__frcp_rn(xf));
  const int re = (int)((rb >> 23) & 0xff) - 127;
  const double r = __hiloint2double((int)((rb & 0x80000000u) | ((unsigned)(re + 1023) << 20) | ((rb & 0x7fffffu) >> 3)),
                                    (int)((rb & 7u) << 29));
  const double ee = fma(-x, r, 1.0);
  return fma(r, fma(ee, ee, ee), r);
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
  const int tid = threadIdx.x;
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
  // Right-looking, one block barrier per column, on the pivots x_k themselves: the
  // trailing update is W[i][j] -= W[i][k] W[j][k] / x_k, which needs only 1 / x_k; the
  // square roots (L[k][k] and 1 / L[k][k]) and the scaling of the columns follow in
  // one parallel pass at the end. The pivot thread (lane 0 of the last warp) updates
  // the next diagonal entry and forms its reciprocal; the other pairs (i, j),
  // k < j <= i, of the trailing triangle are spread over the other threads, so the
  // pivot chain does not wait on a warp that also carries update work.
  constexpr int PW = NTH - 32;
  static_assert(PW % 8 == 0 && PW >= 8, "update threads form a TI x 8 grid");
  auto pivot = [&](int k, double x) {  // keep column k if its pivot x is above rank_tol
    const double r = recip_pivot(x);      // formed beside the test, not after it
    const bool keep = x > rank_tol;
    sh.invd[k] = keep ? r : 0.0;  // 1 / x_k during the factorisation
    sh.perm[k] = keep;
  };
  if (tid == PW) pivot(0, W[0]);
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    const double rx = sh.invd[k];  // 0 drops the column: no trailing update
    const int n = m - 1 - k;       // rows below k
    if (n > 0) {
      if (tid < PW) {
        if (rx != 0.0) {
          // the trailing triangle k < j <= i < m over a fixed TI x 8 thread grid: rows
          // k + 1 + ti + TI a, columns k + 1 + tj + 8 b (no index decoding per entry)
          constexpr int TJ = 8, TI = PW / TJ;
          const int ti = tid / TJ, tj = tid % TJ;
          for (int i = k + 1 + ti; i < m; i += TI) {
            const double lik = -W[i * kLds + k] * rx;
            for (int j = k + 1 + tj; j <= i; j += TJ)
              if (j != i || i != k + 1) W[i * kLds + j] = fma(lik, W[j * kLds + k], W[i * kLds + j]);
          }
        }
      } else if (tid == PW) {
        const int i = k + 1;
        double x = W[i * kLds + i];
        if (rx != 0.0) {
          x = fma(-W[i * kLds + k] * rx, W[i * kLds + k], x);
          W[i * kLds + i] = x;
        }
        pivot(i, x);
      }
    }
    __syncthreads();
  }
  {  // the number of kept columns (an integer sum: the order of the adds is immaterial)
    int kept = 0;
    for (int k = tid; k < m; k += NTH) kept += sh.perm[k];
    if (kept) atomicAdd(&s_rank, kept);
  }
  __syncthreads();
  for (int k = tid; k < m; k += NTH) {  // L[k][k] = sqrt(x_k), invd[k] = 1 / L[k][k]
    const double x = W[k * kLds + k];
    const double r = sh.perm[k] ? rsqrt_newton(x) : 0.0;
    W[k * kLds + k] = sh.perm[k] ? x * r : 0.0;
    sh.invd[k] = r;
  }
  __syncthreads();
  for (int idx = tid; idx < m * m; idx += NTH) {  // L[i][k] = W[i][k] / L[k][k], i > k
    const int i = idx / m, k = idx - i * m;
    if (i > k) W[i * kLds + k] *= sh.invd[k];
  }
  __syncthreads();
  return s_rank;
}

}  // namespace bk
