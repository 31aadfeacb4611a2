// Kernels of the block-Lanczos drivers (ridge path and Gaussian sampling):
//   k_ci_*          Cholesky with dropped dependent columns and the inverse factor of an
//                   m x m FP64 Gram (m <= 256), for the CholQR orthogonalisation of a block:
//                   scaling, panel factorisations and trailing updates, inverse, R
//   k_band_*        the banded block-tridiagonal T_t (Sec. 3.2, Thm. cost): assembly
//                   from the Lanczos blocks, shifted Cholesky solves for many shifts in
//                   one launch (one CTA per shift), and the banded product T_t Y
//   small helpers   FP32/FP64 block copies, scaled column sums, residual norms
#include <algorithm>

#include "bk_common.cuh"

namespace bk {
namespace {

// 1/sqrt(x), x > 0 normal: FP32 estimate of an exactly rescaled argument, two Newton
// steps in FP64 (quadratic convergence).
__device__ __forceinline__ double rsqrt_nr(double x) {
  const int e = ((__double2hiint(x) >> 20) & 0x7ff) - 1023;
  const int h = e >> 1;
  const double xs = x * __hiloint2double((1023 - 2 * h) << 20, 0);
  double r = (double)rsqrtf((float)xs) * __hiloint2double((1023 - h) << 20, 0);
  r = r * fma(-0.5 * x, r * r, 1.5);
  r = r * fma(-0.5 * x, r * r, 1.5);
  return r;
}


// One CTA. G (m x m, row-major, FP64) = W^T W of a block W. Writes
//   R     (m x m, row-major, upper): W = Q R on the kept columns (R rows of dropped
//         columns are zero; their entries above the diagonal record the dependence)
//   Rinv  (m x m, row-major, upper): Q = W Rinv, zero rows/columns for dropped columns
//   keep  (m ints): 1 for kept columns
// with the factorisation done on D^{-1/2} G D^{-1/2} (D = diag G), dropping a column
// whose scaled pivot is <= rank_tol. work: m * m doubles of scratch (global).
// Returns the number of kept columns in *rank.
// CholQR factor and inverse (m <= 256) in parallel pieces: the scaled Gram, then per
// panel of kCiNB columns a one-CTA panel factorisation in shared memory and a many-CTA
// update of the trailing lower triangle in 4 x 4 register tiles, then the inverse
// factor one warp per column and the upper factor R. The matrix lives in `work` (m x m
// row-major, lower triangle used); rs (D^{-1/2}) and invd (1 / L[k][k], 0 for dropped
// columns) in `scratch` (2 m doubles).
constexpr int kCiNB = 32;

__device__ __forceinline__ double ci_rs(double g) { return (g > 0.0 && isfinite(g)) ? rsqrt_nr(g) : 0.0; }

__global__ void k_ci_scale(int m, const double* __restrict__ G, double* L, double* rs, int* rank) {
  const int64_t mm = (int64_t)m * m;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < mm;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / m), c = (int)(idx - (int64_t)r * m);
    L[idx] = G[idx] * ci_rs(G[(int64_t)r * m + r]) * ci_rs(G[(int64_t)c * m + c]);
    if (idx < m) rs[idx] = ci_rs(G[idx * m + idx]);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *rank = 0;
}

// Columns c0 .. c0 + nb - 1 (rows c0 .. m - 1) of the scaled matrix, column-major in
// shared memory: a pivot at or below rank_tol, or a zero diagonal of G, drops its column
// (zero column, invd 0, keep 0), which then changes nothing below.
__global__ void __launch_bounds__(256) k_ci_panel(int m, int c0, double* L, const double* __restrict__ rs,
                                                  double rank_tol, double* invd, int* keep, int* rank) {
  extern __shared__ __align__(16) double pan[];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int nb = min(kCiNB, m - c0), rows = m - c0, PR = ((m + 3) & ~3) + 4;
  __shared__ double s_inv;
  for (int idx = tid; idx < kCiNB * PR; idx += nth) {
    const int q = idx / PR, r = idx - q * PR;
    pan[idx] = (q < nb && r < rows && r >= q) ? L[(int64_t)(c0 + r) * m + c0 + q] : 0.0;
  }
  __syncthreads();
  for (int q = 0; q < nb; ++q) {
    double* col = pan + q * PR;
    if (tid == 0) {
      const double x = col[q];
      const bool kp = rs[c0 + q] > 0.0 && x > rank_tol;
      const double r = kp ? rsqrt_nr(x) : 0.0;
      col[q] = kp ? x * r : 0.0;
      invd[c0 + q] = r;
      keep[c0 + q] = kp;
      if (kp) atomicAdd(rank, 1);
      s_inv = r;
    }
    __syncthreads();
    const double inv = s_inv;
    for (int r = q + 1 + tid; r < rows; r += nth) col[r] *= inv;
    __syncthreads();
    if (inv != 0.0 && q + 1 < nb) {
      const int nk = nb - 1 - q;
      for (int idx = tid; idx < nk * rows; idx += nth) {
        const int k = q + 1 + idx / rows, r = idx - (idx / rows) * rows;
        if (r >= k) pan[k * PR + r] = fma(-col[r], col[k], pan[k * PR + r]);
      }
      __syncthreads();
    }
  }
  for (int idx = tid; idx < kCiNB * PR; idx += nth) {
    const int q = idx / PR, r = idx - q * PR;
    if (q < nb && r < rows && r >= q) L[(int64_t)(c0 + r) * m + c0 + q] = pan[idx];
  }
}

// L[i][j] -= sum_q L[i][c0 + q] L[j][c0 + q] for c0 + nb <= j <= i < m, a 4 x 4 tile per thread
__global__ void __launch_bounds__(256) k_ci_syrk(int m, int c0, int nb, double* L) {
  const int w0 = c0 + nb, wn = m - w0;
  const int t4 = (wn + 3) / 4, ntiles = t4 * (t4 + 1) / 2;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
    int ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while (ti * (ti + 1) / 2 > t) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    const int tc = t - ti * (ti + 1) / 2;
    const int ib = w0 + 4 * ti, cb = w0 + 4 * tc;
    double acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
    for (int q = 0; q < nb; ++q) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = ib + u < m ? L[(int64_t)(ib + u) * m + c0 + q] : 0.0;
        b[u] = cb + u < m ? L[(int64_t)(cb + u) * m + c0 + q] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int i = ib + u, j = cb + v;
        if (i < m && j <= i) L[(int64_t)i * m + j] -= acc[u][v];
      }
  }
}

// Row c of Rinv = D^{-1/2} L^{-T}: rs[c] (L^{-1})[j][c], j >= c, from column c of L^{-1}
// by forward substitution over the kept indices (a warp per column, lanes over the dot
// products; dropped indices stay zero).
__global__ void __launch_bounds__(256) k_ci_inv(int m, const double* __restrict__ L, const double* __restrict__ rs,
                                                const double* __restrict__ invd, const int* __restrict__ keep,
                                                double* Rinv) {
  __shared__ double ys[8][256];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * 8 + w;
  if (c >= m) return;
  double* y = ys[w];
  for (int j = lane; j < m; j += 32) y[j] = 0.0;
  __syncwarp();
  if (keep[c]) {
    for (int j = c; j < m; ++j) {
      if (!keep[j]) continue;  // uniform across the warp
      double s = 0.0;
      for (int l = c + lane; l < j; l += 32) s = fma(L[(int64_t)j * m + l], y[l], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const double val = ((j == c ? 1.0 : 0.0) - s) * invd[j];
      __syncwarp();
      if (lane == 0) y[j] = val;
      __syncwarp();
    }
  }
  for (int j = lane; j < m; j += 32) Rinv[(int64_t)c * m + j] = (j >= c) ? rs[c] * y[j] : 0.0;
}

// R = L^T D^{1/2}: R[i][j] = L[j][i] / rs[j] for j >= i on the kept columns
__global__ void k_ci_r(int m, const double* __restrict__ L, const double* __restrict__ rs,
                       const int* __restrict__ keep, double* R) {
  const int64_t mm = (int64_t)m * m;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < mm;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / m), j = (int)(idx - (int64_t)i * m);
    R[idx] = (j >= i && keep[i] && rs[j] > 0.0) ? L[(int64_t)j * m + i] / rs[j] : 0.0;
  }
}

// Band storage of the symmetric block-tridiagonal T (half-bandwidth bw, row stride ldb
// >= the largest n used): band[r * ldb + c] = T(c + r, c) for 0 <= r <= bw.
// Adds the m x m diagonal block A (row-major) at block k and the subdiagonal block B
// (rows of block k+1, columns of block k) when B is non-null.
__global__ void k_band_put(int ldb, int bw, int m, int k, const double* __restrict__ A, const double* __restrict__ B,
                           double* band) {
  const int c0 = k * m;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < m * m; idx += gridDim.x * blockDim.x) {
    const int i = idx / m, j = idx - i * m;
    if (i >= j) band[(size_t)(i - j) * ldb + c0 + j] = 0.5 * (A[i * m + j] + A[j * m + i]);
    if (B) {
      // T(c0 + m + i, c0 + j) = B[i][j]; B is upper triangular, so r = m + i - j <= m
      const int r = m + i - j;
      if (r <= bw && c0 + j < ldb) band[(size_t)r * ldb + c0 + j] = B[i * m + j];
    }
  }
}

// M (2m x m, column-major, block precision) = [B_{k-1}^T; A_k] for the three-term
// recurrence W -= [Q_{k-1} Q_k] M; B (upper triangular) and A row-major m x m FP64.
// first: the top half is zero (no Q_{k-1}).
template <typename T>
__global__ void k_three_term(int m, int first, const double* __restrict__ A, const double* __restrict__ B, T* M) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 2 * m * m; idx += gridDim.x * blockDim.x) {
    const int j = idx / (2 * m), r = idx - j * 2 * m;
    double v;
    if (r < m)
      v = first ? 0.0 : B[j * m + r];  // (B^T)(r, j) = B(j, r)
    else
      v = A[(r - m) * m + j];
    M[idx] = (T)v;
  }
}

// Shifted banded Cholesky solves (T + mu_j I) Z_j = E_j, E_j = the nrhs columns of rhs
// starting at column rhs_col[j] (rhs: n x ncol column-major, ld n). Two kernels:
//   k_band_factor (bw > 112, blocked) / k_band_factor_smem (bw <= 112): one CTA per
//     shift j factors T + mu_j I (band storage, bw subdiagonals) into work: L x
//     (bw + 2) x n doubles (the factor and the reciprocal diagonal). A diagonal entry that is exactly zero (a dropped Lanczos direction) is
//     replaced by 1 so the dropped direction decouples. A pivot that is not positive
//     drops its direction the same way (its solution component is zero) and sets
//     flags[j] = 1: T + mu_j I was not positive definite.
//   k_band_subst: CTAs (j, s) run the forward and backward substitutions for their
//     slice of the right-hand sides, so that many right-hand sides spread over many SMs.
// Z_j is n x nrhs column-major at Z + j * n * nrhs. Cost O(n bw^2) per shift to factor,
// O(n bw nrhs) to substitute (Thm. cost).
// Wide bands (bw > 112): blocked right-looking factorisation. A panel of kBandNB
// columns (rows c0 .. c0 + kBandNB + bw - 1, column-major in shared memory) is factored
// column by column; its update of the window that follows, a rank-kBandNB symmetric
// update of the band entries (i, c), c0 + kBandNB <= c <= i, runs in 4 x 4 register tiles
// over the panel, so each band entry is read and written once per panel instead of once
// per column (the column-by-column update in global memory was latency bound at
// bw = 256). Same storage, pivots and dropped directions as k_band_factor_smem.
constexpr int kBandNB = 32;
__global__ void __launch_bounds__(256) k_band_factor(int n, int bw, const double* __restrict__ band, int ldb,
                                                     const double* __restrict__ mus, double* work, int* flags) {
  extern __shared__ __align__(16) double pan[];  // [kBandNB][PR], column q at pan + q PR
  const int j = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
  // panel rows: the band's rows padded to a multiple of 4, plus one spare 4-row tile for
  // the window tiles that start at the 4-aligned row below the window (all zeros)
  const int PR = ((kBandNB + bw + 3) & ~3) + 4;
  double* Lb = work + (size_t)j * (bw + 2) * n;
  double* invL = Lb + (size_t)(bw + 1) * n;
  const double mu = mus[j];
  __shared__ double s_inv;
  __shared__ int s_bad;
  for (size_t idx = tid; idx < (size_t)(bw + 1) * n; idx += nth) {
    const int r = (int)(idx / n), c = (int)(idx % n);
    // entries that reach past the end of T_t (rows >= n) are not part of it
    double v = (c + r < n) ? band[(size_t)r * ldb + c] : 0.0;
    if (r == 0) v = (v == 0.0) ? 1.0 : v + mu;
    Lb[idx] = v;
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += kBandNB) {
    const int nb = min(kBandNB, n - c0);
    const int rows = min(nb + bw, n - c0);  // panel rows c0 .. c0 + rows - 1
    // panel in: pan[q][r] = L(c0 + r, c0 + q) inside the band, 0 elsewhere
    for (int idx = tid; idx < kBandNB * PR; idx += nth) {
      const int q = idx / PR, r = idx - q * PR, off = r - q;
      pan[idx] = (q < nb && r < rows && off >= 0 && off <= bw) ? Lb[(size_t)off * n + c0 + q] : 0.0;
    }
    __syncthreads();
    for (int q = 0; q < nb; ++q) {
      double* col = pan + q * PR;
      if (tid == 0) {
        const double x = col[q];
        if (!(x > 0.0)) {  // not positive: drop this direction (unit pivot, zero column)
          s_bad = 1;
          s_inv = 0.0;
          col[q] = 1.0;
        } else {
          const double r = rsqrt_nr(x);
          col[q] = x * r;
          s_inv = r;
        }
        invL[c0 + q] = s_inv;
      }
      __syncthreads();
      const double inv = s_inv;
      for (int r = q + 1 + tid; r < rows; r += nth) col[r] *= inv;
      __syncthreads();
      if (inv != 0.0 && q + 1 < nb) {
        // the panel's later columns k: L(r, k) -= L(r, q) L(k, q), r >= k
        const int nk = nb - 1 - q;
        for (int idx = tid; idx < nk * rows; idx += nth) {
          const int k = q + 1 + idx / rows, r = idx - (idx / rows) * rows;
          if (r >= k) pan[k * PR + r] = fma(-col[r], col[k], pan[k * PR + r]);
        }
        __syncthreads();
      }
    }
    // panel out
    for (int idx = tid; idx < kBandNB * PR; idx += nth) {
      const int q = idx / PR, r = idx - q * PR, off = r - q;
      if (q < nb && r < rows && off >= 0 && off <= bw) Lb[(size_t)off * n + c0 + q] = pan[idx];
    }
    // window update: band entries (i, c), nb <= c - c0 <= i - c0 < rows, minus the
    // panel's rank-nb product; 4 x 4 tiles of the lower triangle, a thread per tile
    // tiles start at the 4-aligned row wb <= nb (aligned 16-byte loads); entries above
    // the window (rows < nb) are skipped
    const int wb = nb & ~3, wn = rows - wb;
    if (rows > nb) {
      const int t4 = (wn + 3) / 4;
      const int ntiles = t4 * (t4 + 1) / 2;
      for (int t = tid; t < ntiles; t += nth) {
        int ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
        while (ti * (ti + 1) / 2 > t) --ti;
        while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
        const int tc = t - ti * (ti + 1) / 2;
        const int ib = wb + 4 * ti, cb = wb + 4 * tc;  // panel rows of the tile (< PR - 3)
        double acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
        for (int q = 0; q < nb; ++q) {
          const double2* pa = reinterpret_cast<const double2*>(pan + q * PR + ib);
          const double2* pc = reinterpret_cast<const double2*>(pan + q * PR + cb);
          const double2 a01 = pa[0], a23 = pa[1], c01 = pc[0], c23 = pc[1];
          const double a[4] = {a01.x, a01.y, a23.x, a23.y}, cc[4] = {c01.x, c01.y, c23.x, c23.y};
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], cc[v], acc[u][v]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const int ri = ib + u, rc = cb + v;
            if (rc >= nb && ri < rows && ri >= rc && ri - rc <= bw) {
              double* e = Lb + (size_t)(ri - rc) * n + c0 + rc;
              *e -= acc[u][v];
            }
          }
      }
    }
    __syncthreads();
  }
  if (tid == 0) flags[j] = s_bad;
}

// The same factorisation with the active window in shared memory, for bw <= 112: the
// columns c .. c + bw are the only ones column c's step reads or updates, so a ring of
// bw + 1 columns (slot c mod (bw + 1), entry r = L(c + r, c)) holds them; a finished
// column goes to `work` and the band's next column takes its slot. Global memory then
// sees each entry once instead of once per trailing update.
__global__ void __launch_bounds__(256) k_band_factor_smem(int n, int bw, const double* __restrict__ band, int ldb,
                                                          const double* __restrict__ mus, double* work, int* flags) {
  extern __shared__ double win[];
  const int j = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nth >> 5;
  const int W = bw + 1;
  double* Lb = work + (size_t)j * (bw + 2) * n;
  double* invL = Lb + (size_t)(bw + 1) * n;
  const double mu = mus[j];
  __shared__ double s_inv;
  __shared__ int s_bad;
  auto band_entry = [&](int c, int r) {
    double v = (c + r < n) ? band[(size_t)r * ldb + c] : 0.0;
    if (r == 0) v = (v == 0.0) ? 1.0 : v + mu;
    return v;
  };
  const int first = min(n, W);
  for (int idx = tid; idx < first * W; idx += nth) {
    const int c = idx / W, r = idx - c * W;
    win[c * W + r] = band_entry(c, r);
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int c = 0; c < n; ++c) {
    double* col = win + (c % W) * W;
    // the band's column c + W, fetched now so that its latency overlaps this step
    const bool next = c + W < n;
    const double pre = (next && tid < W) ? band_entry(c + W, tid) : 0.0;
    if (tid == 0) {
      const double x = col[0];
      if (!(x > 0.0)) {  // not positive: drop this direction (see k_band_factor)
        s_bad = 1;
        s_inv = 0.0;
        col[0] = 1.0;
      } else {
        const double r = rsqrt_nr(x);
        col[0] = x * r;
        s_inv = r;
      }
      invL[c] = s_inv;
    }
    __syncthreads();
    const double inv = s_inv;
    const int w = min(bw, n - 1 - c);
    for (int r = 1 + tid; r <= w; r += nth) col[r] *= inv;
    __syncthreads();
    if (inv != 0.0) {
      for (int a = 1 + warp; a <= w; a += nw) {
        const double la = col[a];
        for (int b = 1 + lane; b <= a; b += 32) {
          double* t = win + ((c + b) % W) * W + (a - b);
          *t = fma(-la, col[b], *t);
        }
      }
      __syncthreads();
    }
    // column c is final: out to the factor, and the band's column c + W into its slot
    if (tid < W) {
      Lb[(size_t)tid * n + c] = (tid <= w) ? col[tid] : 0.0;
      if (next) col[tid] = pre;
    }
    __syncthreads();
  }
  if (tid == 0) flags[j] = s_bad;
}

__global__ void __launch_bounds__(256) k_band_subst(int n, int bw, const double* __restrict__ rhs,
                                                    const int* __restrict__ rhs_col, int nrhs, int per_cta,
                                                    const double* __restrict__ work, double* Z,
                                                    const int* __restrict__ flags) {
  const int j = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
  const int q0 = blockIdx.y * per_cta;
  const int q1 = min(nrhs, q0 + per_cta);
  if (q0 >= q1) return;
  const int nq = q1 - q0;
  const double* Lb = work + (size_t)j * (bw + 2) * n;
  const double* invL = Lb + (size_t)(bw + 1) * n;
  double* z = Z + (size_t)j * n * nrhs + (size_t)q0 * n;
  const double* e = rhs + (size_t)(rhs_col[j] + q0) * n;
  for (size_t idx = tid; idx < (size_t)n * nq; idx += nth) z[idx] = e[idx];
  __syncthreads();
  // forward L y = e, column-oriented: y_c *= 1/L_cc, then y_{c+r} -= L(c+r, c) y_c
  for (int c = 0; c < n; ++c) {
    const double inv = invL[c];
    for (int q = tid; q < nq; q += nth) z[(size_t)q * n + c] *= inv;
    __syncthreads();
    const int w = min(bw, n - 1 - c);
    for (int idx = tid; idx < w * nq; idx += nth) {
      const int r = 1 + idx % w, q = idx / w;
      z[(size_t)q * n + c + r] = fma(-Lb[(size_t)r * n + c], z[(size_t)q * n + c], z[(size_t)q * n + c + r]);
    }
    __syncthreads();
  }
  // backward L^T z = y, column-oriented: z_c *= 1/L_cc, then z_{c-r} -= L(c, c-r) z_c
  for (int c = n - 1; c >= 0; --c) {
    const double inv = invL[c];
    for (int q = tid; q < nq; q += nth) z[(size_t)q * n + c] *= inv;
    __syncthreads();
    const int w = min(bw, c);
    for (int idx = tid; idx < w * nq; idx += nth) {
      const int r = 1 + idx % w, q = idx / w;
      z[(size_t)q * n + c - r] = fma(-Lb[(size_t)r * n + c - r], z[(size_t)q * n + c], z[(size_t)q * n + c - r]);
    }
    __syncthreads();
  }
}

// out (n x nc, column-major) = (T + shift I) Y for the banded symmetric T.
__global__ void k_band_mult(int n, int bw, const double* __restrict__ band, int ldb, double shift,
                            const double* __restrict__ Y, int nc, double* out) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)n * nc;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n), q = (int)(idx / n);
    double s = shift * Y[(size_t)q * n + i];
    const int lo = max(0, i - bw), hi = min(n - 1, i + bw);
    for (int k = lo; k <= hi; ++k) {
      const double t = (k <= i) ? band[(size_t)(i - k) * ldb + k] : band[(size_t)(k - i) * ldb + i];
      s = fma(t, Y[(size_t)q * n + k], s);
    }
    out[idx] = s;
  }
}

// Y (n x nc) = sum_j c_j Z_j for L stacked n x nc blocks.
__global__ void k_combine_shifts(int n, int nc, int L, const double* __restrict__ Z, const double* __restrict__ c,
                                 double* Y) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)n * nc;
       idx += (size_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < L; ++j) s = fma(c[j], Z[(size_t)j * n * nc + idx], s);
    Y[idx] = s;
  }
}

// ||B z_last|| per shift: z_last = rows n-m..n-1 of Z_j (column q), B (m x m row-major).
__global__ void k_lanczos_res(int n, int m, int L, int nrhs, const double* __restrict__ Blast,
                              const double* __restrict__ Z, double* out) {
  // one warp per (shift, rhs)
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= L * nrhs) return;
  const int j = w / nrhs, q = w % nrhs;
  const double* zl = Z + (size_t)j * n * nrhs + (size_t)q * n + (n - m);
  double ss = 0.0;
  for (int i = lane; i < m; i += 32) {
    double s = 0.0;
    for (int k = 0; k < m; ++k) s = fma(Blast[i * m + k], zl[k], s);
    ss = fma(s, s, ss);
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if (lane == 0) out[w] = sqrt(ss);
}

// Column c of a d x m block (column-major, ld) times scale[c]; FP32 or FP64.
template <typename T>
__global__ void k_scale_cols(int64_t d, int m, int64_t ld, const double* __restrict__ scale, T* X) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < d * m;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = idx / d, i = idx - c * d;
    X[c * ld + i] = (T)((double)X[c * ld + i] * scale[c]);
  }
}

template <typename TI, typename TO>
__global__ void k_copy_cols(int64_t d, int m, const TI* __restrict__ in, int64_t ldi, TO* out, int64_t ldo) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < d * m;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = idx / d, i = idx - c * d;
    out[c * ldo + i] = (TO)in[c * ldi + i];
  }
}

// R = B 1^T - (A X + X diag(mu)) given AX (d x L, FP64): column norms squared partials.
__global__ void k_shift_residual(int64_t d, int L, const double* __restrict__ b, const double* __restrict__ AX,
                                 const double* __restrict__ X, int64_t ld, const double* __restrict__ mus,
                                 double* R, double* norms2) {
  // one CTA per column
  const int j = blockIdx.x;
  __shared__ double red[32];
  double ss = 0.0;
  for (int64_t i = threadIdx.x; i < d; i += blockDim.x) {
    const double r = b[i] - (AX[j * ld + i] + mus[j] * X[j * ld + i]);
    R[j * ld + i] = r;
    ss = fma(r, r, ss);
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) norms2[j] = s;
  }
}

// rhs (n x mb, column-major, ld n) = E_1 R_0: rhs(i, q) = R0[i][q] for i < mb, else 0.
__global__ void k_e1r0(int n, int mb, const double* __restrict__ R0, double* rhs) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)n * mb;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n), q = (int)(idx / n);
    rhs[idx] = (i < mb) ? R0[i * mb + q] : 0.0;
  }
}

// Gershgorin bound max_i sum_k |T(i, k)| of the leading n x n part of the band (one CTA).
__global__ void k_band_gersh(int n, int bw, const double* __restrict__ band, int ldb, double* out) {
  __shared__ double red[32];
  double mx = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    const int lo = max(0, i - bw), hi = min(n - 1, i + bw);
    for (int k = lo; k <= hi; ++k) s += fabs((k <= i) ? band[(size_t)(i - k) * ldb + k] : band[(size_t)(k - i) * ldb + i]);
    mx = fmax(mx, s);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) *out = v;
  }
}

inline int cgrid(int64_t work, int th) {
  int64_t g = (work + th - 1) / th;
  if (g < 1) g = 1;
  if (g > 152 * 16) g = 152 * 16;
  return (int)g;
}

}  // namespace

cudaError_t launch_band_gersh(int n, int bw, const double* band, int ldb, double* out, cudaStream_t st) {
  k_band_gersh<<<1, 1024, 0, st>>>(n, bw, band, ldb, out);
  return cudaGetLastError();
}

cudaError_t launch_e1r0(int n, int mb, const double* R0, double* rhs, cudaStream_t st) {
  k_e1r0<<<cgrid((int64_t)n * mb, 256), 256, 0, st>>>(n, mb, R0, rhs);
  return cudaGetLastError();
}

cudaError_t launch_chol_inv(int m, const double* G, double rank_tol, double* work, double* R, double* Rinv,
                            int* keep, int* rank, double* scratch, cudaStream_t st) {
  if (m < 1 || m > 256) return cudaErrorInvalidValue;
  double* rs = scratch;
  double* invd = scratch + m;
  const int gmm = (int)std::min<int64_t>(((int64_t)m * m + 255) / 256, 1024);
  k_ci_scale<<<gmm, 256, 0, st>>>(m, G, work, rs, rank);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)kCiNB * (((m + 3) & ~3) + 4) * 8;
  if ((e = cudaFuncSetAttribute(k_ci_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  for (int c0 = 0; c0 < m; c0 += kCiNB) {
    const int nb = std::min(kCiNB, m - c0);
    k_ci_panel<<<1, 256, smem, st>>>(m, c0, work, rs, rank_tol, invd, keep, rank);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (c0 + nb < m) {
      const int t4 = (m - c0 - nb + 3) / 4, ntiles = t4 * (t4 + 1) / 2;
      k_ci_syrk<<<(ntiles + 255) / 256, 256, 0, st>>>(m, c0, nb, work);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  k_ci_inv<<<(m + 7) / 8, 256, 0, st>>>(m, work, rs, invd, keep, Rinv);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_ci_r<<<gmm, 256, 0, st>>>(m, work, rs, keep, R);
  return cudaGetLastError();
}

cudaError_t launch_three_term(int is_f64, int m, int first, const double* A, const double* B, void* M,
                              cudaStream_t st) {
  const int g = (2 * m * m + 255) / 256;
  if (is_f64)
    k_three_term<double><<<g, 256, 0, st>>>(m, first, A, B, (double*)M);
  else
    k_three_term<float><<<g, 256, 0, st>>>(m, first, A, B, (float*)M);
  return cudaGetLastError();
}

cudaError_t launch_band_put(int ldb, int bw, int m, int k, const double* A, const double* B, double* band,
                            cudaStream_t st) {
  k_band_put<<<cgrid((int64_t)m * m, 256), 256, 0, st>>>(ldb, bw, m, k, A, B, band);
  return cudaGetLastError();
}

cudaError_t launch_band_solve(int n, int bw, const double* band, int ldb, int L, const double* mus,
                              const double* rhs, const int* rhs_col, int nrhs, double* work, double* Z, int* flags,
                              cudaStream_t st) {
  if (L <= 0) return cudaSuccess;
  cudaError_t e;
  if (bw <= 112) {
    const size_t smem = (size_t)(bw + 1) * (bw + 1) * 8;
    if ((e = cudaFuncSetAttribute(k_band_factor_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
      return e;
    k_band_factor_smem<<<L, 256, smem, st>>>(n, bw, band, ldb, mus, work, flags);
  } else {
    const size_t smem = (size_t)kBandNB * (((kBandNB + bw + 3) & ~3) + 4) * 8;
    if ((e = cudaFuncSetAttribute(k_band_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
      return e;
    k_band_factor<<<L, 256, smem, st>>>(n, bw, band, ldb, mus, work, flags);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // right-hand-side slices: about two CTAs per SM in total, at least 8 columns each
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int slices = std::max(1, std::min((2 * sms + L - 1) / L, nrhs / 8));
  const int per = (nrhs + slices - 1) / slices;
  slices = (nrhs + per - 1) / per;
  k_band_subst<<<dim3(L, slices), 256, 0, st>>>(n, bw, rhs, rhs_col, nrhs, per, work, Z, flags);
  return cudaGetLastError();
}

cudaError_t launch_band_mult(int n, int bw, const double* band, int ldb, double shift, const double* Y, int nc,
                             double* out, cudaStream_t st) {
  k_band_mult<<<cgrid((int64_t)n * nc, 256), 256, 0, st>>>(n, bw, band, ldb, shift, Y, nc, out);
  return cudaGetLastError();
}

cudaError_t launch_combine_shifts(int n, int nc, int L, const double* Z, const double* c, double* Y,
                                  cudaStream_t st) {
  k_combine_shifts<<<cgrid((int64_t)n * nc, 256), 256, 0, st>>>(n, nc, L, Z, c, Y);
  return cudaGetLastError();
}

cudaError_t launch_lanczos_res(int n, int m, int L, int nrhs, const double* Blast, const double* Z, double* out,
                               cudaStream_t st) {
  int warps = L * nrhs;
  k_lanczos_res<<<(warps * 32 + 255) / 256, 256, 0, st>>>(n, m, L, nrhs, Blast, Z, out);
  return cudaGetLastError();
}

cudaError_t launch_scale_cols(int is_f64, int64_t d, int m, int64_t ld, const double* scale, void* X,
                              cudaStream_t st) {
  if (is_f64)
    k_scale_cols<double><<<cgrid(d * m, 256), 256, 0, st>>>(d, m, ld, scale, (double*)X);
  else
    k_scale_cols<float><<<cgrid(d * m, 256), 256, 0, st>>>(d, m, ld, scale, (float*)X);
  return cudaGetLastError();
}

cudaError_t launch_copy_cols(int in_f64, int out_f64, int64_t d, int m, const void* in, int64_t ldi, void* out,
                             int64_t ldo, cudaStream_t st) {
  int g = cgrid(d * m, 256);
  if (in_f64 && out_f64)
    k_copy_cols<double, double><<<g, 256, 0, st>>>(d, m, (const double*)in, ldi, (double*)out, ldo);
  else if (in_f64)
    k_copy_cols<double, float><<<g, 256, 0, st>>>(d, m, (const double*)in, ldi, (float*)out, ldo);
  else if (out_f64)
    k_copy_cols<float, double><<<g, 256, 0, st>>>(d, m, (const float*)in, ldi, (double*)out, ldo);
  else
    k_copy_cols<float, float><<<g, 256, 0, st>>>(d, m, (const float*)in, ldi, (float*)out, ldo);
  return cudaGetLastError();
}

cudaError_t launch_shift_residual(int64_t d, int L, const double* b, const double* AX, const double* X, int64_t ld,
                                  const double* mus, double* R, double* norms2, cudaStream_t st) {
  k_shift_residual<<<L, 256, 0, st>>>(d, L, b, AX, X, ld, mus, R, norms2);
  return cudaGetLastError();
}

}  // namespace bk
