// Block-CG step kernels other than the block product: Gram partial reduction, the
// small FP64 Cholesky solves, the fused residual and direction updates, the start
// block and small helpers.
//
// One block-CG step (Def. BCG; the recurrence of O'Leary cited in Sec. 3):
//   Y = A_mu P ; G = P^T Y                       (k_csr_spmm_gram / k_dense_gram)
//   alpha = G^{-1} S                             (k_small_alpha)
//   R -= Y alpha ; S' = R^T R                    (k_update_r)
//   beta = S^{-1} S'                             (k_small_beta, with the residual test)
//   x += P alpha[:,0] ; P = R + P beta ; S = S'  (k_update_p)
#include "bk_common.cuh"
#include "bk_tile.cuh"

namespace bk {
namespace {

constexpr int kUpdThreads = 128;

__device__ __forceinline__ bool is_done(const DevState* s) { return s && (s->done_a | s->done_b); }

// ------------------------------------------------------------------ Gram of blocks
template <typename T, int MP, int TM>
__global__ void __launch_bounds__(TM) k_gram(int64_t d, const T* __restrict__ X, const T* __restrict__ Y,
                                            int64_t ld, int m, double* parts, int nparts) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sX = reinterpret_cast<T*>(smem_raw);
  T* sY = sX + TM * MP;
  GramAcc<T, MP> g;
  g.init();
  int64_t ntiles = (d + TM - 1) / TM;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int64_t i = tile * TM + threadIdx.x;
    T vx[MP], vy[MP];
#pragma unroll
    for (int q = 0; q < MP / 4; ++q) {
      bool ok = (i < d) && (4 * q < m);
      if (ok) {
        ldg4(panel_row(X, ld, q, i), vx + 4 * q);
        ldg4(panel_row(Y, ld, q, i), vy + 4 * q);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) vx[4 * q + u] = vy[4 * q + u] = (T)0;
      }
    }
    store_row<MP>(sX, threadIdx.x, vx);
    store_row<MP>(sY, threadIdx.x, vy);
    __syncthreads();
    g.tile(sX, sY, TM);
    __syncthreads();
  }
  gram_finish<T, MP>(g, reinterpret_cast<double*>(smem_raw), parts, nparts, blockIdx.x);
}

// ------------------------------------------------------------------ partial reduction
// One warp per partial entry; lanes stride over partials, then a fixed shuffle tree.
template <int MP>
__global__ void k_reduce_gram(int m, const double* __restrict__ parts, int nparts, double* out,
                              const DevState* state) {
  if (is_done(state)) return;
  using S = GramShape<MP>;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= S::NE) return;
  const double* p = parts + (size_t)warp * nparts;
  double s = 0.0;
  for (int k = lane; k < nparts; k += 32) s += p[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    int t = warp >> 4, e = warp & 15;
    int tt = t, r = 0;
    while (tt >= S::NB - r) {
      tt -= S::NB - r;
      ++r;
    }
    int row = 4 * r + (e >> 2), col = 4 * (r + tt) + (e & 3);
    // keep the upper triangle (row <= col) and mirror it
    if (row <= col && col < m) {
      out[row * m + col] = s;
      out[col * m + row] = s;
    }
  }
}

// ------------------------------------------------------------------ small solves
// The m x m systems G alpha = S and S beta = S' of each step are solved by a Cholesky
// factorisation of the unit-diagonal scaled matrix D^{-1/2} M D^{-1/2}, one CTA per
// right-hand-side column (every CTA factors the same matrix in the same order, so all
// agree on which columns are kept). A column whose pivot falls below rank_tol is
// numerically in the span of the columns before it; it is dropped and the solution
// is taken on the kept columns only (zero rows elsewhere). For G = P^T A_mu P this
// keeps X += P alpha the Galerkin update over span(P) when the block has become rank
// deficient (Sec. 3.2: blocks can lose rank even in exact arithmetic).
constexpr int kSmallMax = 64;
constexpr int kLds = kSmallMax + 1;

struct SmallShared {
  double W[kSmallMax * kLds];
  double z[kSmallMax];
  double dscale[kSmallMax];
  double invd[kSmallMax];  // 1 / L[k][k]
  int perm[kSmallMax];
};

constexpr int kSmallThreads = 128;

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

// On this part an FP64 instruction has a 64-cycle latency, a single warp issues at
// most one FP64 instruction per 64 cycles, and a square root or division is a
// dependent chain of several hundred cycles, so the factorisation is organised around
// its dependency chain: no pivot search (comparisons are FP64 instructions too), one
// thread forms 1/sqrt(pivot) by Newton steps, and the trailing update is spread over
// four warps (four SM sub-partitions).
//
// Cholesky of the unit-diagonal scaled matrix in the given column order; a pivot at
// or below rank_tol marks column k as numerically in the span of the kept columns
// before it: its row and column are dropped (flag keep[k] = 0) and the factorisation
// continues. Returns the number of kept columns, or -1 for a non-positive or
// non-finite diagonal entry. On return the lower triangle of W holds L on the kept
// rows/columns (zeros elsewhere) and invd[k] = 1 / L[k][k] (0 for dropped columns).
__device__ int block_cholesky_skip(SmallShared& sh, int m, double rank_tol) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kSmallThreads / 32;
  double* W = sh.W;
  __shared__ int s_bad, s_rank;
  if (tid == 0) {
    s_bad = 0;
    s_rank = 0;
  }
  __syncthreads();
  for (int i = tid; i < m; i += kSmallThreads) {
    const double g = W[i * kLds + i];
    const bool bad = !(g > 0.0) || !isfinite(g);
    if (bad) s_bad = 1;
    const double r = bad ? 1.0 : rsqrt_newton(g);  // D^{-1/2}
    sh.z[i] = r;
    sh.dscale[i] = bad ? 1.0 : g * r;  // sqrt(g)
  }
  __syncthreads();
  if (s_bad) return -1;
  for (int idx = tid; idx < m * m; idx += kSmallThreads) {
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
    for (int i = k + 1 + tid; i < m; i += kSmallThreads) W[i * kLds + k] *= inv;
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

// z <- L^+ applied twice (L^{-T} L^{-1} on the kept columns, zero on dropped ones),
// warp 0; invd holds 1 / L[k][k] (0 for dropped columns).
__device__ void chol_apply_warp0(const double* L, const double* invd, double* z, int m) {
  if ((threadIdx.x >> 5) == 0) {
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < m; ++k) {
      __syncwarp();
      const double zk = z[k] * invd[k];
      __syncwarp();
      if (lane == 0) z[k] = zk;
      for (int i = k + 1 + lane; i < m; i += 32) z[i] = fma(-L[i * kLds + k], zk, z[i]);
    }
    for (int k = m - 1; k >= 0; --k) {
      __syncwarp();
      const double zk = z[k] * invd[k];
      __syncwarp();
      if (lane == 0) z[k] = zk;
      for (int i = lane; i < k; i += 32) z[i] = fma(-L[k * kLds + i], zk, z[i]);
    }
    __syncwarp();
  }
  __syncthreads();
}

// CTA j: column j of X = M^+ RHS on the kept columns (zero rows on dropped ones); the
// result is left in sh.z[0:m]. Returns the number of kept columns (-1: invalid diagonal).
__device__ int small_solve_column(const double* M, const double* RHS, int m, int j, double rank_tol,
                                  SmallShared& sh) {
  const int tid = threadIdx.x;
  for (int idx = tid; idx < m * m; idx += kSmallThreads) {
    const int r = idx / m, c = idx - r * m;
    sh.W[r * kLds + c] = M[idx];
  }
  __syncthreads();
  const int rank = block_cholesky_skip(sh, m, rank_tol);
  if (rank <= 0) return rank;
  // the scaled system: (D^{-1/2} M D^{-1/2}) (D^{1/2} x) = D^{-1/2} rhs, D^{-1/2} = 1/dscale
  __shared__ double y[kSmallMax];
  __shared__ double rs[kSmallMax];
  for (int i = tid; i < m; i += kSmallThreads) {
    rs[i] = sh.z[i];  // D^{-1/2} from the scaling step
    y[i] = RHS[i * m + j] * rs[i];
  }
  __syncthreads();
  chol_apply_warp0(sh.W, sh.invd, y, m);
  for (int i = tid; i < m; i += kSmallThreads) sh.z[i] = y[i] * rs[i];
  __syncthreads();
  return rank;
}

template <typename T>
__device__ void write_column(const double* z, int m, int mp, int j, double* X, T* Xt) {
  for (int i = threadIdx.x; i < mp; i += kSmallThreads) {
    double v = (i < m) ? z[i] : 0.0;
    if (i < m) X[i * m + j] = v;
    Xt[i * mp + j] = (T)v;
  }
}

template <typename T>
__device__ void zero_pad_columns(int m, int mp, T* Xt) {
  // columns m..mp-1 of the padded copy (CTA 0 only)
  for (int idx = threadIdx.x; idx < mp * mp; idx += kSmallThreads) {
    int c = idx % mp;
    if (c >= m) Xt[idx] = (T)0;
  }
}

template <typename T>
__global__ void k_small_alpha(int m, int mp, const double* G, const double* S, double* X, T* Xt,
                              double rank_tol, DevState* state) {
  __shared__ SmallShared sh;
  bool cta0 = blockIdx.x == 0;
  if (is_done(state)) {
    if (cta0 && threadIdx.x == 0) state->pending_x = 0;
    return;
  }
  int j = blockIdx.x;
  int rank = small_solve_column(G, S, m, j, rank_tol, sh);
  if (rank > 0) write_column<T>(sh.z, m, mp, j, X, Xt);
  if (cta0) {
    zero_pad_columns<T>(m, mp, Xt);
    if (threadIdx.x == 0) {
      state->loads += 1;
      if (rank <= 0) {
        state->pending_x = 0;
        state->done_a = 1;
        state->status = ST_BREAKDOWN;
      } else {
        // a rank-deficient block still gives a valid Galerkin step; the inner solve
        // ends after it and the caller restarts from the new residual
        state->pending_x = 1;
        if (rank < m) {
          state->done_a = 1;
          state->status = ST_DEFLATED;
        }
      }
    }
  }
}

template <typename T>
__global__ void k_small_beta(int m, int mp, const double* Sold, const double* Snew, double* X, T* Xt,
                             double rank_tol, DevState* state) {
  __shared__ SmallShared sh;
  bool cta0 = blockIdx.x == 0;
  if (is_done(state)) return;
  double res = sqrt(fmax(Snew[0], 0.0));
  bool conv = res <= state->tol_abs;
  bool cap = state->loads >= state->max_loads;
  if (conv || cap) {
    if (cta0 && threadIdx.x == 0) {
      state->res = res;
      state->done_b = 1;
      state->status = conv ? ST_CONVERGED : ST_LOADCAP;
    }
    return;
  }
  int j = blockIdx.x;
  int rank = small_solve_column(Sold, Snew, m, j, rank_tol, sh);
  if (rank == m) write_column<T>(sh.z, m, mp, j, X, Xt);
  if (cta0) {
    zero_pad_columns<T>(m, mp, Xt);
    if (threadIdx.x == 0) {
      state->res = res;
      if (rank != m) {
        state->done_b = 1;
        state->status = rank < 0 ? ST_BREAKDOWN : ST_DEFLATED;
      }
    }
  }
}

__global__ void k_chol_solve(int m, const double* G, const double* S, double* X, double rank_tol, int* flag) {
  __shared__ SmallShared sh;
  int j = blockIdx.x;
  int rank = small_solve_column(G, S, m, j, rank_tol, sh);
  if (rank != m) {
    if (threadIdx.x == 0) atomicExch(flag, 1);
    return;
  }
  for (int i = threadIdx.x; i < m; i += kSmallThreads) X[i * m + j] = sh.z[i];
}

// ------------------------------------------------------------------ updates
// R -= Y alpha, then the Gram partial of the new R. Thread per row; the whole R and Y
// rows are loaded up front (2 MP independent loads per thread in flight), alpha is
// read from shared memory as 16-byte broadcasts.
template <typename T, int MP, int TM>
__global__ void __launch_bounds__(TM, sizeof(T) == 4 ? 4 : 2)
    k_update_r(int64_t d, int m, const T* __restrict__ Y, T* __restrict__ R, int64_t ld,
               const T* __restrict__ alpha_t, double* parts, int nparts, const DevState* state) {
  if (is_done(state)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sA = reinterpret_cast<T*>(smem_raw);  // MP x MP
  T* sX = sA + MP * MP;                     // TM x MP tile of the new R
  for (int idx = threadIdx.x; idx < MP * MP; idx += blockDim.x) sA[idx] = alpha_t[idx];
  __syncthreads();
  GramAcc<T, MP> g;
  g.init();
  int64_t ntiles = (d + TM - 1) / TM;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t i = tile * TM + threadIdx.x;
    const bool ok = i < d;
    asm volatile("" ::: "memory");  // no hoisting of the alpha reads across tiles
    T acc[MP], y[MP];
#pragma unroll
    for (int q = 0; q < MP / 4; ++q) {
      if (ok && 4 * q < m) {
        ld4(panel_row(R, ld, q, i), acc + 4 * q);
        ldg4(panel_row(Y, ld, q, i), y + 4 * q);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[4 * q + u] = y[4 * q + u] = (T)0;
      }
    }
#pragma unroll
    for (int k = 0; k < MP; ++k) {
      const T* a = sA + k * MP;
#pragma unroll
      for (int c = 0; c < MP; ++c) acc[c] = fma(-y[k], a[c], acc[c]);
    }
    if (ok) {
#pragma unroll
      for (int q = 0; q < MP / 4; ++q)
        if (4 * q < m) st4(panel_row(R, ld, q, i), acc + 4 * q);
    }
    store_row<MP>(sX, threadIdx.x, acc);
    __syncthreads();
    g.tile(sX, sX, TM);
    __syncthreads();
  }
  // sred aliases the tile area after the alpha block
  gram_finish<T, MP>(g, reinterpret_cast<double*>(smem_raw + ((MP * MP * sizeof(T) + 15) / 16) * 16), parts,
                     nparts, blockIdx.x);
}

// x += P alpha[:,0]; unless the solve just ended, P = R + P beta; CTA 0 copies Snew
// into Sold. Thread per row, both rows loaded up front.
template <typename T, int MP>
__global__ void __launch_bounds__(kUpdThreads, sizeof(T) == 4 ? 3 : 2)
    k_update_p(int64_t d, int m, const T* __restrict__ R, T* P, int64_t ld, const T* __restrict__ alpha_t,
               const T* __restrict__ beta_t, double* x, const double* Snew, double* Sold, const DevState* state) {
  if (state && !state->pending_x) return;
  const bool upd = !(state && (state->done_a | state->done_b));
  __shared__ __align__(16) T sB[MP * MP];
  __shared__ __align__(16) T sa0[MP];
  for (int idx = threadIdx.x; idx < MP * MP; idx += blockDim.x) sB[idx] = beta_t[idx];
  for (int idx = threadIdx.x; idx < MP; idx += blockDim.x) sa0[idx] = alpha_t[idx * MP];
  if (upd && blockIdx.x == 0 && Sold)
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) Sold[idx] = Snew[idx];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
    asm volatile("" ::: "memory");  // no hoisting of the beta reads across rows
    T p[MP], acc[MP];
#pragma unroll
    for (int q = 0; q < MP / 4; ++q) {
      if (4 * q < m) {
        ld4(panel_row(P, ld, q, i), p + 4 * q);
        if (upd) ldg4(panel_row(R, ld, q, i), acc + 4 * q);
        else {
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[4 * q + u] = (T)0;
        }
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) p[4 * q + u] = acc[4 * q + u] = (T)0;
      }
    }
    T xs = 0;
#pragma unroll
    for (int k = 0; k < MP; ++k) xs = fma(p[k], sa0[k], xs);
    x[i] += (double)xs;
    if (upd) {
#pragma unroll
      for (int k = 0; k < MP; ++k) {
        const T* b = sB + k * MP;
#pragma unroll
        for (int c = 0; c < MP; ++c) acc[c] = fma(p[k], b[c], acc[c]);
      }
#pragma unroll
      for (int q = 0; q < MP / 4; ++q)
        if (4 * q < m) st4(panel_row(P, ld, q, i), acc + 4 * q);
    }
  }
}

// ------------------------------------------------------------------ start block, helpers
// R = P = [r * scale, Omega] on panels: the Omega buffer is a full panel block whose
// column 0 and padding columns are zero.
template <typename T>
__global__ void k_start_block(int64_t d, int m, int64_t ld, const double* r, double scale, const T* omega,
                              T* R, T* P, double* x) {
  const int nq = (m + 3) >> 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
    for (int q = 0; q < nq; ++q) {
      T v[4];
      ldg4(panel_row(omega, ld, q, i), v);
      if (q == 0) v[0] = (T)(r[i] * scale);
      st4(panel_row(R, ld, q, i), v);
      st4(panel_row(P, ld, q, i), v);
    }
    x[i] = 0.0;
  }
}

__global__ void k_init_state(DevState* s, int max_loads, double tol_abs) {
  s->done_a = 0;
  s->done_b = 0;
  s->pending_x = 0;
  s->loads = 0;
  s->status = ST_RUNNING;
  s->max_loads = max_loads;
  s->tol_abs = tol_abs;
  s->res = 1.0;
}

__global__ void k_axpy(int64_t d, double a, const double* y, double* x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fma(a, y[i], x[i]);
}

__global__ void k_to_f32(int64_t n, const double* in, float* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

__global__ void k_to_f64(int64_t n, const float* in, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

// ||v||^2 partials, one per CTA, deterministic order.
__global__ void k_norm2_parts(int64_t d, const double* v, double* parts) {
  __shared__ double red[32];
  double ss = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x)
    ss = fma(v[i], v[i], ss);
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = ss;
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    double s = (l < nw) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (l == 0) parts[blockIdx.x] = s;
  }
}

__global__ void k_dense_to_f32(int64_t d, const double* in, int64_t lda, float* out, int64_t lda32) {
  int64_t n = d * d;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = k / d, c = k - r * d;
    out[r * lda32 + c] = (float)in[r * lda + c];
  }
}

int sm_count(int device) {
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n <= 0) n = 152;
  return n;
}

inline int capped_grid(int64_t work, int threads, int cap) {
  int64_t g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

template <typename T, int MP>
cudaError_t gram_impl(int64_t d, const void* X, const void* Y, int64_t ld, int m, double* parts, int nparts,
                      cudaStream_t st) {
  constexpr int TM = sizeof(T) == 4 ? 256 : 128;
  size_t smem = gram_smem_bytes<T, MP>(TM, TM);
  auto kern = k_gram<T, MP, TM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<nparts, TM, smem, st>>>(d, (const T*)X, (const T*)Y, ld, m, parts, nparts);
  return cudaGetLastError();
}

template <typename T, int MP>
cudaError_t update_r_impl(int64_t d, int m, const void* Y, void* R, int64_t ld, const void* alpha_t, double* parts,
                          int nparts, const DevState* state, cudaStream_t st) {
  constexpr int TM = 128;
  size_t head = ((MP * MP * sizeof(T) + 15) / 16) * 16;
  size_t smem = head + gram_smem_bytes<T, MP>(TM, TM);
  auto kern = k_update_r<T, MP, TM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<nparts, TM, smem, st>>>(d, m, (const T*)Y, (T*)R, ld, (const T*)alpha_t, parts, nparts, state);
  return cudaGetLastError();
}

template <typename T, int MP>
cudaError_t update_p_impl(int64_t d, int m, const void* R, void* P, int64_t ld, const void* alpha_t,
                          const void* beta_t, double* x, const double* Snew, double* Sold, const DevState* state,
                          cudaStream_t st, int device) {
  int grid = capped_grid(d, kUpdThreads, sm_count(device) * (sizeof(T) == 4 ? 4 : 2) * 4);
  k_update_p<T, MP><<<grid, kUpdThreads, 0, st>>>(d, m, (const T*)R, (T*)P, ld, (const T*)alpha_t,
                                                  (const T*)beta_t, x, Snew, Sold, state);
  return cudaGetLastError();
}

#define BK_DISPATCH_MP(mp, F, ...)                  \
  switch (mp) {                                     \
    case 4: return F<4>(__VA_ARGS__);               \
    case 8: return F<8>(__VA_ARGS__);               \
    case 16: return F<16>(__VA_ARGS__);             \
    case 24: return F<24>(__VA_ARGS__);             \
    case 36: return F<36>(__VA_ARGS__);             \
    default: return cudaErrorInvalidValue;          \
  }

template <int MP>
cudaError_t gram_d(int64_t d, const void* X, const void* Y, int64_t ld, int m, double* parts, int nparts,
                   cudaStream_t st) {
  return gram_impl<double, MP>(d, X, Y, ld, m, parts, nparts, st);
}
template <int MP>
cudaError_t gram_f(int64_t d, const void* X, const void* Y, int64_t ld, int m, double* parts, int nparts,
                   cudaStream_t st) {
  return gram_impl<float, MP>(d, X, Y, ld, m, parts, nparts, st);
}
template <int MP>
cudaError_t reduce_mp(int m, const double* parts, int nparts, double* out, const DevState* state, cudaStream_t st) {
  int warps = GramShape<MP>::NE;
  int threads = 256;
  int grid = (warps * 32 + threads - 1) / threads;
  k_reduce_gram<MP><<<grid, threads, 0, st>>>(m, parts, nparts, out, state);
  return cudaGetLastError();
}
template <int MP>
cudaError_t upd_r_d(int64_t d, int m, const void* Y, void* R, int64_t ld, const void* a, double* parts, int np,
                    const DevState* s, cudaStream_t st) {
  return update_r_impl<double, MP>(d, m, Y, R, ld, a, parts, np, s, st);
}
template <int MP>
cudaError_t upd_r_f(int64_t d, int m, const void* Y, void* R, int64_t ld, const void* a, double* parts, int np,
                    const DevState* s, cudaStream_t st) {
  return update_r_impl<float, MP>(d, m, Y, R, ld, a, parts, np, s, st);
}
template <int MP>
cudaError_t upd_p_d(int64_t d, int m, const void* R, void* P, int64_t ld, const void* a, const void* b, double* x,
                    const double* Sn, double* So, const DevState* s, cudaStream_t st, int dev) {
  return update_p_impl<double, MP>(d, m, R, P, ld, a, b, x, Sn, So, s, st, dev);
}
template <int MP>
cudaError_t upd_p_f(int64_t d, int m, const void* R, void* P, int64_t ld, const void* a, const void* b, double* x,
                    const double* Sn, double* So, const DevState* s, cudaStream_t st, int dev) {
  return update_p_impl<float, MP>(d, m, R, P, ld, a, b, x, Sn, So, s, st, dev);
}

}  // namespace

// ------------------------------------------------------------------ launchers
int gram_grid(int is_f64, int mp, int64_t d, int device) {
  int tm = is_f64 ? 128 : 256;
  int64_t ntiles = (d + tm - 1) / tm;
  int cap = sm_count(device) * 2;
  return (int)(ntiles < cap ? (ntiles < 1 ? 1 : ntiles) : cap);
}
int update_r_grid(int is_f64, int mp, int64_t d, int device) {
  int64_t ntiles = (d + 127) / 128;
  int cap = sm_count(device) * (is_f64 ? 2 : 4);
  return (int)(ntiles < cap ? (ntiles < 1 ? 1 : ntiles) : cap);
}

cudaError_t launch_gram(int is_f64, int mp, int64_t d, const void* X, const void* Y, int64_t ld, int m,
                        double* parts, int nparts, cudaStream_t st) {
  if (is_f64) {
    BK_DISPATCH_MP(mp, gram_d, d, X, Y, ld, m, parts, nparts, st);
  } else {
    BK_DISPATCH_MP(mp, gram_f, d, X, Y, ld, m, parts, nparts, st);
  }
}

cudaError_t launch_reduce_gram(int mp, int m, const double* parts, int nparts, double* out, const DevState* state,
                               cudaStream_t st) {
  BK_DISPATCH_MP(mp, reduce_mp, m, parts, nparts, out, state, st);
}

cudaError_t launch_small_alpha(int is_f64, int mp, int m, const double* G, const double* S, double* X, void* Xt,
                               double rank_tol, DevState* state, cudaStream_t st) {
  if (m < 1 || m > kSmallMax || mp < m) return cudaErrorInvalidValue;
  if (is_f64)
    k_small_alpha<double><<<m, kSmallThreads, 0, st>>>(m, mp, G, S, X, (double*)Xt, rank_tol, state);
  else
    k_small_alpha<float><<<m, kSmallThreads, 0, st>>>(m, mp, G, S, X, (float*)Xt, rank_tol, state);
  return cudaGetLastError();
}

cudaError_t launch_small_beta(int is_f64, int mp, int m, const double* Sold, const double* Snew, double* X, void* Xt,
                              double rank_tol, DevState* state, cudaStream_t st) {
  if (m < 1 || m > kSmallMax || mp < m) return cudaErrorInvalidValue;
  if (is_f64)
    k_small_beta<double><<<m, kSmallThreads, 0, st>>>(m, mp, Sold, Snew, X, (double*)Xt, rank_tol, state);
  else
    k_small_beta<float><<<m, kSmallThreads, 0, st>>>(m, mp, Sold, Snew, X, (float*)Xt, rank_tol, state);
  return cudaGetLastError();
}

cudaError_t launch_chol_solve(int m, const double* G, const double* S, double* X, int* flag, cudaStream_t st) {
  if (m < 1 || m > kSmallMax) return cudaErrorInvalidValue;
  k_chol_solve<<<m, kSmallThreads, 0, st>>>(m, G, S, X, 1e-14, flag);
  return cudaGetLastError();
}

cudaError_t launch_update_r(int is_f64, int mp, int64_t d, int m, const void* Y, void* R, int64_t ld,
                            const void* alpha_t, double* parts, int nparts, const DevState* state,
                            cudaStream_t st) {
  if (is_f64) {
    BK_DISPATCH_MP(mp, upd_r_d, d, m, Y, R, ld, alpha_t, parts, nparts, state, st);
  } else {
    BK_DISPATCH_MP(mp, upd_r_f, d, m, Y, R, ld, alpha_t, parts, nparts, state, st);
  }
}

cudaError_t launch_update_p(int is_f64, int mp, int64_t d, int m, const void* R, void* P, int64_t ld,
                            const void* alpha_t, const void* beta_t, double* x, const double* Snew, double* Sold,
                            const DevState* state, cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (is_f64) {
    BK_DISPATCH_MP(mp, upd_p_d, d, m, R, P, ld, alpha_t, beta_t, x, Snew, Sold, state, st, dev);
  } else {
    BK_DISPATCH_MP(mp, upd_p_f, d, m, R, P, ld, alpha_t, beta_t, x, Snew, Sold, state, st, dev);
  }
}

cudaError_t launch_start_block(int is_f64, int64_t d, int m, int64_t ld, const double* r, double scale,
                               const void* omega, void* R, void* P, double* x, cudaStream_t st) {
  int grid = capped_grid(d, 256, 152 * 8);
  if (is_f64)
    k_start_block<double><<<grid, 256, 0, st>>>(d, m, ld, r, scale, (const double*)omega, (double*)R, (double*)P, x);
  else
    k_start_block<float><<<grid, 256, 0, st>>>(d, m, ld, r, scale, (const float*)omega, (float*)R, (float*)P, x);
  return cudaGetLastError();
}

cudaError_t launch_init_state(DevState* state, int max_loads, double tol_abs, cudaStream_t st) {
  k_init_state<<<1, 1, 0, st>>>(state, max_loads, tol_abs);
  return cudaGetLastError();
}

cudaError_t launch_axpy(int64_t d, double a, const double* y, double* x, cudaStream_t st) {
  k_axpy<<<capped_grid(d, 256, 152 * 8), 256, 0, st>>>(d, a, y, x);
  return cudaGetLastError();
}

cudaError_t launch_to_f32(int64_t n, const double* in, float* out, cudaStream_t st) {
  k_to_f32<<<capped_grid(n, 256, 152 * 16), 256, 0, st>>>(n, in, out);
  return cudaGetLastError();
}

cudaError_t launch_to_f64(int64_t n, const float* in, double* out, cudaStream_t st) {
  k_to_f64<<<capped_grid(n, 256, 152 * 16), 256, 0, st>>>(n, in, out);
  return cudaGetLastError();
}

cudaError_t launch_norm2_parts(int64_t d, const double* v, double* parts, int nparts, cudaStream_t st) {
  k_norm2_parts<<<nparts, 256, 0, st>>>(d, v, parts);
  return cudaGetLastError();
}

cudaError_t launch_dense_to_f32(int64_t d, const double* in, int64_t lda, float* out, int64_t lda32,
                                cudaStream_t st) {
  k_dense_to_f32<<<capped_grid(d * d, 256, 152 * 16), 256, 0, st>>>(d, in, lda, out, lda32);
  return cudaGetLastError();
}

}  // namespace bk
