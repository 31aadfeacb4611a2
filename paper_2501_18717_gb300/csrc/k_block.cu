// Block-CG step kernels other than the block product: Gram partial reduction, the
// small FP64 Cholesky solves, the fused residual and direction updates, the start
// block and small helpers.
//
// One block-CG step in the orthonormal-residual form (block CG with a QR-factored
// residual, Dubrulle 2001): the residual block is kept as R = Q C with Q of (nearly)
// orthonormal columns, and only c = C e_1 is carried (the column-0 system is the one
// solved; Def. BCG, bcg^(1)). With P the search directions:
//   Y = A_mu P ; G = P^T Y                       (k_csr_spmm_gram / k_dense_gram)
//   Gi = G^+ ; xc = G^+ c                        (k_small_alpha)
//   W = Q - Y Gi ; S = W^T W                     (k_update_r; FP32: k_update_r_pf)
//   S = T^T T (T upper) ; c <- T c ; test ||c||  (k_small_beta)
//   x += P xc ; Q = W T^{-1} ; P = Q + P T^T     (k_update_p; FP32: k_update_p_async)
// In exact arithmetic this gives the iterates of O'Leary's recurrence (the one the
// paper cites in Sec. 3): both are the Galerkin iterates over the block Krylov space.
// It differs in rounding: P is built from an orthonormal basis instead of residual
// columns whose norms drift apart as they converge, which keeps the small systems well
// conditioned. In FP32 blocks the O'Leary form stops converging on spectra with
// kappa ~ 1e5 while this form converges.
#include "bk_common.cuh"
#include "bk_small.cuh"
#include "bk_tile.cuh"
#include "bk_update.cuh"

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
  GramAcc<T, MP, gram_bpt<MP, TM>()> g;
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
// The m x m systems of each step are solved through a Cholesky factorisation of the
// unit-diagonal scaled matrix D^{-1/2} M D^{-1/2} (block_cholesky_skip), one CTA per
// output column: every CTA factors the same matrix in the same order, so all agree on
// which columns are kept. A column whose pivot falls below rank_tol is numerically in
// the span of the columns before it; it is dropped (zero rows and columns in the
// results), which for G = P^T A_mu P keeps x += P G^+ c the Galerkin update over
// span(P) when the block has become rank deficient (Sec. 3.2: blocks can lose rank even
// in exact arithmetic), and for S = W^T W leaves the dropped direction out of the new
// basis. A dropped column of Q (and so of P) stays zero from then on: its Gram rows
// are zero and a zero diagonal is dropped again.
constexpr int kSmallThreads = 128;

// Forward (L^+) and backward (L^{-T} on the kept columns) substitution on z in place,
// warp 0; invd holds 1 / L[k][k] (0 for dropped columns).
__device__ void chol_forward_warp0(const double* L, const double* invd, double* z, int m) {
  if ((threadIdx.x >> 5) == 0) {
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < m; ++k) {
      __syncwarp();
      const double zk = z[k] * invd[k];
      __syncwarp();
      if (lane == 0) z[k] = zk;
      for (int i = k + 1 + lane; i < m; i += 32) z[i] = fma(-L[i * kLds + k], zk, z[i]);
    }
    __syncwarp();
  }
  __syncthreads();
}
__device__ void chol_backward_warp0(const double* L, const double* invd, double* z, int m) {
  if ((threadIdx.x >> 5) == 0) {
    const int lane = threadIdx.x & 31;
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

__device__ int load_and_factor(const double* M, int m, double rank_tol, SmallShared& sh) {
  for (int idx = threadIdx.x; idx < m * m; idx += kSmallThreads) {
    const int r = idx / m, c = idx - r * m;
    sh.W[r * kLds + c] = M[idx];
  }
  __syncthreads();
  return block_cholesky_skip<kSmallThreads>(sh, m, rank_tol);
}

// CTA j < m: column j of Gi = G^+ (row-major mp x mp copy in the block precision);
// CTA m: xc = G^+ c. CTA 0 owns the control block: one more load, and the x update
// of this step is pending unless G is unusable.
template <typename T>
__global__ void k_small_alpha(int m, int mp, const double* G, const double* cvec, T* gi_t, T* xc_t,
                              double rank_tol, DevState* state) {
  __shared__ SmallShared sh;
  __shared__ double y[kSmallMax];
  const bool cta0 = blockIdx.x == 0;
  if (is_done(state)) {
    if (cta0 && threadIdx.x == 0) state->pending_x = 0;
    return;
  }
  const int j = blockIdx.x;
  const int rank = load_and_factor(G, m, rank_tol, sh);
  if (rank > 0) {
    for (int i = threadIdx.x; i < m; i += kSmallThreads) {
      const double rhs = j < m ? (i == j ? 1.0 : 0.0) : cvec[i];
      y[i] = rhs * sh.z[i];
    }
    __syncthreads();
    chol_forward_warp0(sh.W, sh.invd, y, m);
    chol_backward_warp0(sh.W, sh.invd, y, m);
    for (int i = threadIdx.x; i < mp; i += kSmallThreads) {
      const T v = (T)(i < m ? y[i] * sh.z[i] : 0.0);
      if (j < m)
        gi_t[i * mp + j] = v;
      else
        xc_t[i] = v;
    }
  }
  if (cta0) {
    const int pad = mp - m;
    if (pad > 0)
      for (int idx = threadIdx.x; idx < mp * pad; idx += kSmallThreads) gi_t[(idx / pad) * mp + m + idx % pad] = (T)0;
    if (threadIdx.x == 0) {
      state->loads += 1;
      state->first = 0;
      if (rank <= 0) {
        state->pending_x = 0;
        state->done_a = 1;
        state->status = ST_BREAKDOWN;
      } else {
        state->pending_x = 1;
      }
    }
  }
}

// S = W^T W = T^T T with T = L^T D^{1/2} upper triangular (on the kept columns).
// CTA j writes column j of Ti = T^+ (ti_t[i * mp + j]) and column j of T as row j of
// T^T (t_t[j * mp + i] = T(i, j) = L(j, i) dscale[j], i <= j), both mp x mp row-major in
// the block precision. CTA 0 also forms c <- T c, the residual ||c|| = ||R e_1|| and the
// stopping decision. The columns are written even when the solve stops here (no later
// kernel reads them then), so only CTA 0 reads c and no CTA reads what another writes.
template <typename T>
__global__ void k_small_beta(int m, int mp, const double* S, double* cvec, T* ti_t, T* t_t, double rank_tol,
                             DevState* state) {
  __shared__ SmallShared sh;
  __shared__ double y[kSmallMax];
  __shared__ double cn[kSmallMax];
  if (is_done(state)) return;
  const int j = blockIdx.x;
  const int rank = load_and_factor(S, m, rank_tol, sh);
  if (rank >= 0) {
    for (int i = threadIdx.x; i < m; i += kSmallThreads) y[i] = (i == j) ? 1.0 : 0.0;
    __syncthreads();
    chol_backward_warp0(sh.W, sh.invd, y, m);
    for (int i = threadIdx.x; i < mp; i += kSmallThreads) {
      ti_t[i * mp + j] = (T)(i < m ? y[i] * sh.z[i] : 0.0);
      t_t[j * mp + i] = (T)(i <= j ? sh.W[j * kLds + i] * sh.dscale[j] : 0.0);
    }
  }
  if (j != 0) return;
  const int pad = mp - m;
  for (int idx = threadIdx.x; idx < mp * pad; idx += kSmallThreads) {
    ti_t[(size_t)(idx / pad) * mp + m + idx % pad] = (T)0;  // columns m..mp-1
    t_t[(size_t)(m + idx / mp) * mp + idx % mp] = (T)0;     // rows m..mp-1
  }
  if (rank < 0) {
    if (threadIdx.x == 0) {
      state->done_b = 1;
      state->status = ST_BREAKDOWN;
    }
    return;
  }
  for (int i = threadIdx.x; i < m; i += kSmallThreads) {
    double s = 0.0;
    for (int k = i; k < m; ++k) s = fma(sh.W[k * kLds + i] * sh.dscale[k], cvec[k], s);
    cn[i] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += kSmallThreads) cvec[i] = cn[i];
  if (threadIdx.x == 0) {
    state->kept = rank;
    double ss = 0.0;
    for (int i = 0; i < m; ++i) ss = fma(cn[i], cn[i], ss);
    const double res = sqrt(ss);
    state->res = res;
    const bool conv = res <= state->tol_abs;
    if (conv || state->loads >= state->max_loads) {
      state->done_b = 1;
      state->status = conv ? ST_CONVERGED : ST_LOADCAP;
    } else if (!(res <= kDivergedRes)) {
      state->done_b = 1;
      state->status = ST_BREAKDOWN;
    }
  }
}

// Stand-alone X = G^+ S column by column (no control block); flag set on a dropped
// column or an unusable G.
__global__ void k_chol_solve(int m, const double* G, const double* S, double* X, double rank_tol, int* flag) {
  __shared__ SmallShared sh;
  __shared__ double y[kSmallMax];
  const int j = blockIdx.x;
  const int rank = load_and_factor(G, m, rank_tol, sh);
  if (rank != m) {
    if (threadIdx.x == 0) atomicExch(flag, 1);
    return;
  }
  for (int i = threadIdx.x; i < m; i += kSmallThreads) y[i] = S[i * m + j] * sh.z[i];
  __syncthreads();
  chol_forward_warp0(sh.W, sh.invd, y, m);
  chol_backward_warp0(sh.W, sh.invd, y, m);
  for (int i = threadIdx.x; i < m; i += kSmallThreads) X[i * m + j] = y[i] * sh.z[i];
}

// ------------------------------------------------------------------ updates
// R -= Y alpha, then the Gram partial of the new R. A tile of 128 rows is split over
// 32 x CG threads: thread (rg, cg) owns rows rg + 32 u (u < 4) and the CPT = MP / CG
// columns of column group cg. The Y tile is staged in shared memory column by column,
// so each k costs four row values and CPT / 4 broadcast 16-byte alpha chunks for 4 CPT
// FMAs (at width 36: 7 shared loads per 48 FMAs; one row per thread needed 9 per 36,
// which left the kernel bound by the shared-memory pipe). Width 68 (17 chunks of 4)
// takes 17 column groups of 4 columns (544 threads).
template <int MP>
struct UpdRShape {
  static constexpr int CG = (MP % 12 == 0) ? MP / 12 : ((MP % 8 == 0) ? MP / 8 : MP / 4);
  static constexpr int CPT = MP / CG;
  static constexpr int TH = 32 * CG;
  static constexpr int TM = 128;
};

template <typename T, int MP>
struct UpdRSmem {
  static constexpr int LDY = UpdRShape<MP>::TM + (sizeof(T) == 4 ? 4 : 2);
  static constexpr size_t A_B = ((size_t)MP * MP * sizeof(T) + 15) / 16 * 16;
  static constexpr size_t Y_B = ((size_t)MP * LDY * sizeof(T) + 15) / 16 * 16;
  static constexpr size_t X_B = (size_t)UpdRShape<MP>::TM * MP * sizeof(T);
  static constexpr size_t RED_B = (size_t)gram_phases<MP>(UpdRShape<MP>::TH) * GramShape<MP>::NE * 8;
  static constexpr size_t TOTAL = A_B + (Y_B + X_B > RED_B ? Y_B + X_B : RED_B);
};

template <typename T, int MP>
__global__ void __launch_bounds__(UpdRShape<MP>::TH)
    k_update_r(int64_t d, int m, const T* __restrict__ Y, T* __restrict__ R, int64_t ld,
               const T* __restrict__ alpha_t, double* parts, int nparts, const DevState* state) {
  if (is_done(state)) return;
  using U = UpdRShape<MP>;
  using SM = UpdRSmem<T, MP>;
  constexpr int TM = U::TM, CPT = U::CPT, LDY = SM::LDY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sA = reinterpret_cast<T*>(smem_raw);               // MP x MP: row k = alpha(k, :)
  T* sY = reinterpret_cast<T*>(smem_raw + SM::A_B);      // MP x LDY: column k of the Y tile
  T* sX = reinterpret_cast<T*>(smem_raw + SM::A_B + SM::Y_B);  // TM x MP: new R rows
  for (int idx = threadIdx.x; idx < MP * MP; idx += blockDim.x) sA[idx] = alpha_t[idx];
  const int rg = threadIdx.x & 31, cg = threadIdx.x >> 5, c0 = cg * CPT;
  GramAcc<T, MP, gram_bpt<MP, U::TH>()> g;
  g.init();
  __syncthreads();
  const int64_t ntiles = (d + TM - 1) / TM;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t i0 = tile * TM;
    T acc[4][CPT];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t i = i0 + rg + 32 * u;
#pragma unroll
      for (int pi = 0; pi < CPT / 4; ++pi) {
        const int q = c0 / 4 + pi;
        T y4[4];
        if (i < d && 4 * q < m) {
          ld4(panel_row(R, ld, q, i), acc[u] + 4 * pi);
          ldg4(panel_row(Y, ld, q, i), y4);
        } else {
#pragma unroll
          for (int w = 0; w < 4; ++w) acc[u][4 * pi + w] = y4[w] = (T)0;
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) sY[(4 * q + w) * LDY + rg + 32 * u] = y4[w];
      }
    }
    __syncthreads();
    // columns m..MP-1 of Y are zero: the product stops at m
#pragma unroll 4
    for (int k = 0; k < m; ++k) {
      T yk[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) yk[u] = sY[k * LDY + rg + 32 * u];
      T a[CPT];
#pragma unroll
      for (int j4 = 0; j4 < CPT / 4; ++j4) {
        if constexpr (sizeof(T) == 4) {
          const float4 v = *reinterpret_cast<const float4*>(sA + k * MP + c0 + 4 * j4);
          a[4 * j4] = v.x;
          a[4 * j4 + 1] = v.y;
          a[4 * j4 + 2] = v.z;
          a[4 * j4 + 3] = v.w;
        } else {
          const double2 v0 = *reinterpret_cast<const double2*>(sA + k * MP + c0 + 4 * j4);
          const double2 v1 = *reinterpret_cast<const double2*>(sA + k * MP + c0 + 4 * j4 + 2);
          a[4 * j4] = v0.x;
          a[4 * j4 + 1] = v0.y;
          a[4 * j4 + 2] = v1.x;
          a[4 * j4 + 3] = v1.y;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int j = 0; j < CPT; ++j) acc[u][j] = fma(-yk[u], a[j], acc[u][j]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int row = rg + 32 * u;
      const int64_t i = i0 + row;
#pragma unroll
      for (int pi = 0; pi < CPT / 4; ++pi) {
        const int q = c0 / 4 + pi;
        if (i < d && 4 * q < m) st4(panel_row(R, ld, q, i), acc[u] + 4 * pi);
        T v4[4] = {acc[u][4 * pi], acc[u][4 * pi + 1], acc[u][4 * pi + 2], acc[u][4 * pi + 3]};
        store4<MP>(sX, row, q, v4);
      }
    }
    __syncthreads();
    gram_tile<TM, U::TH>(g, sX, sX);
    __syncthreads();
  }
  // the phase buffer of the Gram reduction aliases the tiles after alpha
  gram_finish<T, MP>(g, reinterpret_cast<double*>(smem_raw + SM::A_B), parts, nparts, blockIdx.x);
}

// FP32 residual update at widths up to 36 with the next tile in flight: the Y tile is
// kept in shared memory in the panel layout (row r of panel q as one 16-byte slot),
// copied there by cp.async (no registers held), and each thread's rows of R go straight
// into its accumulators. Both are issued for tile n + 1 right after the W rows of tile
// n are stored, so the Gram of tile n covers their latency (the accumulators are dead
// during it). The product, its order and the Gram are those of k_update_r.
template <int MP>
struct UpdRPf {
  static constexpr size_t A_B = ((size_t)MP * MP * 4 + 15) / 16 * 16;
  static constexpr size_t Y_B = (size_t)(MP / 4) * UpdRShape<MP>::TM * 16;
  static constexpr size_t X_B = (size_t)UpdRShape<MP>::TM * MP * 4;
  static constexpr size_t RED_B = (size_t)gram_phases<MP>(UpdRShape<MP>::TH) * GramShape<MP>::NE * 8;
  static constexpr size_t TOTAL = A_B + (Y_B + X_B > RED_B ? Y_B + X_B : RED_B);
};

template <int MP>
__global__ void __launch_bounds__(UpdRShape<MP>::TH)
    k_update_r_pf(int64_t d, int m, const float* __restrict__ Y, float* __restrict__ R, int64_t ld,
                  const float* __restrict__ alpha_t, double* parts, int nparts, const DevState* state) {
  if (is_done(state)) return;
  using U = UpdRShape<MP>;
  using SM = UpdRPf<MP>;
  constexpr int TM = U::TM, CPT = U::CPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sA = reinterpret_cast<float*>(smem_raw);                        // MP x MP: row k = alpha(k, :)
  float4* sYp = reinterpret_cast<float4*>(smem_raw + SM::A_B);           // panel q, row r at q * TM + r
  float* sX = reinterpret_cast<float*>(smem_raw + SM::A_B + SM::Y_B);    // TM x MP: new R rows
  for (int idx = threadIdx.x; idx < MP * MP; idx += blockDim.x) sA[idx] = alpha_t[idx];
  const int rg = threadIdx.x & 31, cg = threadIdx.x >> 5, c0 = cg * CPT;
  GramAcc<float, MP, gram_bpt<MP, U::TH>()> g;
  g.init();
  const int64_t ntiles = (d + TM - 1) / TM;
  float acc[4][CPT];
  auto issue = [&](int64_t tile) {
    const int64_t i0 = tile * TM;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t i = i0 + rg + 32 * u;
      const bool ok = i < d;
      const int64_t ii = ok ? i : 0;
#pragma unroll
      for (int pi = 0; pi < CPT / 4; ++pi) {
        const int q = c0 / 4 + pi;
        if (4 * q < m) {  // Y rows past d land as zeros
          upd_cp16(sYp + q * TM + rg + 32 * u, panel_row(Y, ld, q, ii), ok ? 16 : 0);
          if (ok)
            ld4(panel_row(R, ld, q, i), acc[u] + 4 * pi);
          else {
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[u][4 * pi + w] = 0.f;
          }
        } else {
#pragma unroll
          for (int w = 0; w < 4; ++w) acc[u][4 * pi + w] = 0.f;
        }
      }
    }
    upd_cp_commit();
  };
  if (blockIdx.x < ntiles) issue(blockIdx.x);
  const int nq = (m + 3) >> 2;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t i0 = tile * TM;
    upd_cp_wait0();
    __syncthreads();  // the Y tile (and alpha) visible; every thread's previous Gram is done
    // k over the full panels (no branch), then the live columns of the last panel:
    // columns m..MP-1 of Y are zero, so the product stops at m
    auto step = [&](int k, const float (&yk)[4]) {
      float a[CPT];
#pragma unroll
      for (int j4 = 0; j4 < CPT / 4; ++j4) {
        const float4 v = *reinterpret_cast<const float4*>(sA + k * MP + c0 + 4 * j4);
        a[4 * j4] = v.x;
        a[4 * j4 + 1] = v.y;
        a[4 * j4 + 2] = v.z;
        a[4 * j4 + 3] = v.w;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int j = 0; j < CPT; ++j) acc[u][j] = fmaf(-yk[u], a[j], acc[u][j]);
    };
    auto panel = [&](int q, float (&y4)[4][4]) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 v = sYp[q * TM + rg + 32 * u];
        y4[0][u] = v.x;
        y4[1][u] = v.y;
        y4[2][u] = v.z;
        y4[3][u] = v.w;
      }
    };
    const int qf = m >> 2;
#pragma unroll 2
    for (int q = 0; q < qf; ++q) {
      float y4[4][4];
      panel(q, y4);
#pragma unroll
      for (int w = 0; w < 4; ++w) step(4 * q + w, y4[w]);
    }
    if (qf < nq) {
      float y4[4][4];
      panel(qf, y4);
#pragma unroll
      for (int w = 0; w < 4; ++w)
        if (4 * qf + w < m) step(4 * qf + w, y4[w]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int row = rg + 32 * u;
      const int64_t i = i0 + row;
#pragma unroll
      for (int pi = 0; pi < CPT / 4; ++pi) {
        const int q = c0 / 4 + pi;
        if (i < d && 4 * q < m) st4(panel_row(R, ld, q, i), acc[u] + 4 * pi);
        float v4[4] = {acc[u][4 * pi], acc[u][4 * pi + 1], acc[u][4 * pi + 2], acc[u][4 * pi + 3]};
        store4<MP>(sX, row, q, v4);
      }
    }
    __syncthreads();  // sX complete; every thread is done reading the Y tile
    if (tile + gridDim.x < ntiles) issue(tile + gridDim.x);
    gram_tile<TM, U::TH>(g, sX, sX);
  }
  __syncthreads();
  // the phase buffer of the Gram reduction aliases the tiles after alpha
  gram_finish<float, MP>(g, reinterpret_cast<double*>(smem_raw + SM::A_B), parts, nparts, blockIdx.x);
}

// x += P xc; unless the solve just ended, Q = W T^{-1} (W is held in Q) and
// P = Q + P T^T (P = Q on the first call of an inner solve, which only normalises the
// start block); the row loop is update_pq_rows.
// (No residency hint at width 36: with one the compiler spills the row arrays.)
template <typename T, int MP>
__global__ void __launch_bounds__(kUpdThreads, MP < 36 ? (sizeof(T) == 4 ? 3 : 2) : 0)
    k_update_p(int64_t d, int m, T* Q, T* P, int64_t ld, const T* __restrict__ xc_t, const T* __restrict__ ti_t,
               const T* __restrict__ t_t, double* x, const DevState* state) {
  const bool do_x = state->pending_x;
  const bool upd = !(state->done_a | state->done_b);
  if (!do_x && !upd) return;
  const bool first = state->first;
  // above width 36 the two tables are in dynamic shared memory (two FP64 68 x 68
  // tables exceed the 48 KB of static shared memory)
  constexpr bool kDyn = MP > 36;
  __shared__ __align__(16) T sTi_s[kDyn ? 1 : MP * MP];
  __shared__ __align__(16) T sTT_s[kDyn ? 1 : MP * MP];
  __shared__ __align__(16) T sxc[MP];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sTi = kDyn ? reinterpret_cast<T*>(smem_raw) : sTi_s;
  T* sTT = kDyn ? reinterpret_cast<T*>(smem_raw) + MP * MP : sTT_s;
  for (int idx = threadIdx.x; idx < MP * MP; idx += blockDim.x) {
    sTi[idx] = ti_t[idx];
    sTT[idx] = first ? (T)0 : t_t[idx];
  }
  for (int idx = threadIdx.x; idx < MP; idx += blockDim.x) sxc[idx] = do_x ? xc_t[idx] : (T)0;
  __syncthreads();
  update_pq_rows<T, MP>(blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x, d, m, Q, P,
                        ld, sTi, sTT, sxc, do_x, upd, x);
}

// FP32 direction update at widths up to 36 with each thread's next row in flight
// (update_pq_rows_async: a two-stage cp.async ring of 16-byte panel slots in dynamic
// shared memory, 72 KB at width 36); persistent grid of two CTAs per SM.
template <int MP>
__global__ void __launch_bounds__(kUpdThreads, 2)
    k_update_p_async(int64_t d, int m, float* Q, float* P, int64_t ld, const float* __restrict__ xc_t,
                     const float* __restrict__ ti_t, const float* __restrict__ t_t, double* x,
                     const DevState* state) {
  const bool do_x = state->pending_x;
  const bool upd = !(state->done_a | state->done_b);
  if (!do_x && !upd) return;
  const bool first = state->first;
  __shared__ __align__(16) float sTi[MP * MP];
  __shared__ __align__(16) float sTT[MP * MP];
  __shared__ __align__(16) float sxc[MP];
  extern __shared__ __align__(16) float4 ring[];
  for (int idx = threadIdx.x; idx < MP * MP; idx += blockDim.x) {
    sTi[idx] = ti_t[idx];
    sTT[idx] = first ? 0.f : t_t[idx];
  }
  for (int idx = threadIdx.x; idx < MP; idx += blockDim.x) sxc[idx] = do_x ? xc_t[idx] : 0.f;
  __syncthreads();
  update_pq_rows_async<MP>(blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x, d, m, Q,
                           P, ld, sTi, sTT, sxc, do_x, upd, x, ring);
}

// ------------------------------------------------------------------ start block, helpers
// Q = [r * scale, Omega] on panels (the Omega buffer is a full panel block whose column
// 0 and padding columns are zero), x = 0. P is formed by the first k_update_p.
template <typename T>
__global__ void k_start_block(int64_t d, int m, int64_t ld, const double* r, double scale, const T* omega, T* Q,
                              double* x) {
  const int nq = (m + 3) >> 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
    for (int q = 0; q < nq; ++q) {
      T v[4];
      ldg4(panel_row(omega, ld, q, i), v);
      if (q == 0) v[0] = (T)(r[i] * scale);
      st4(panel_row(Q, ld, q, i), v);
    }
    x[i] = 0.0;
  }
}

// New inner solve: c = e_1 (the start block's column 0 has norm 1), first = 1.
__global__ void k_init_state(DevState* s, int max_loads, double tol_abs, double* cvec, int m) {
  for (int i = threadIdx.x; i < m; i += blockDim.x) cvec[i] = i == 0 ? 1.0 : 0.0;
  if (threadIdx.x == 0) {
    s->done_a = 0;
    s->done_b = 0;
    s->pending_x = 0;
    s->first = 1;
    s->loads = 0;
    s->status = ST_RUNNING;
    s->max_loads = max_loads;
    s->timeout = 0;
    s->kept = m;
    s->tol_abs = tol_abs;
    s->res = 1.0;
  }
}

__global__ void k_axpy(int64_t d, double a, const double* y, double* x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fma(a, y[i], x[i]);
}

__global__ void k_axpy_out(int64_t d, double a, const double* y, const double* x, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = fma(a, y[i], x[i]);
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
  if constexpr (sizeof(T) == 4 && MP <= 36) {
    const size_t smem = UpdRPf<MP>::TOTAL;
    auto kern = k_update_r_pf<MP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<nparts, UpdRShape<MP>::TH, smem, st>>>(d, m, (const float*)Y, (float*)R, ld, (const float*)alpha_t,
                                                  parts, nparts, state);
    return cudaGetLastError();
  }
  const size_t smem = UpdRSmem<T, MP>::TOTAL;
  auto kern = k_update_r<T, MP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<nparts, UpdRShape<MP>::TH, smem, st>>>(d, m, (const T*)Y, (T*)R, ld, (const T*)alpha_t, parts, nparts,
                                                state);
  return cudaGetLastError();
}

template <typename T, int MP>
cudaError_t update_p_impl(int64_t d, int m, void* Q, void* P, int64_t ld, const void* xc_t, const void* ti_t,
                          const void* t_t, double* x, const DevState* state, cudaStream_t st, int device) {
  if constexpr (sizeof(T) == 4 && MP <= 36) {
    const size_t ring = (size_t)2 * 2 * (MP / 4) * kUpdThreads * 16;
    auto k = k_update_p_async<MP>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring);
    if (e != cudaSuccess) return e;
    const int grid = capped_grid(d, kUpdThreads, sm_count(device) * 2);
    k<<<grid, kUpdThreads, ring, st>>>(d, m, (float*)Q, (float*)P, ld, (const float*)xc_t, (const float*)ti_t,
                                       (const float*)t_t, x, state);
    return cudaGetLastError();
  } else {
    int grid = capped_grid(d, kUpdThreads, sm_count(device) * (sizeof(T) == 4 ? 4 : 2) * 4);
    const size_t smem = MP > 36 ? 2 * (size_t)MP * MP * sizeof(T) : 0;
    if (smem) {
      cudaError_t e = cudaFuncSetAttribute(k_update_p<T, MP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    k_update_p<T, MP><<<grid, kUpdThreads, smem, st>>>(d, m, (T*)Q, (T*)P, ld, (const T*)xc_t, (const T*)ti_t,
                                                    (const T*)t_t, x, state);
    return cudaGetLastError();
  }
}

#define BK_DISPATCH_MP(mp, F, ...)                  \
  switch (mp) {                                     \
    case 4: return F<4>(__VA_ARGS__);               \
    case 8: return F<8>(__VA_ARGS__);               \
    case 16: return F<16>(__VA_ARGS__);             \
    case 24: return F<24>(__VA_ARGS__);             \
    case 36: return F<36>(__VA_ARGS__);             \
    case 68: return F<68>(__VA_ARGS__);             \
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
cudaError_t upd_p_d(int64_t d, int m, void* Q, void* P, int64_t ld, const void* xc, const void* ti, const void* t,
                    double* x, const DevState* s, cudaStream_t st, int dev) {
  return update_p_impl<double, MP>(d, m, Q, P, ld, xc, ti, t, x, s, st, dev);
}
template <int MP>
cudaError_t upd_p_f(int64_t d, int m, void* Q, void* P, int64_t ld, const void* xc, const void* ti, const void* t,
                    double* x, const DevState* s, cudaStream_t st, int dev) {
  return update_p_impl<float, MP>(d, m, Q, P, ld, xc, ti, t, x, s, st, dev);
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

cudaError_t launch_small_alpha(int is_f64, int mp, int m, const double* G, const double* cvec, void* gi_t,
                               void* xc_t, double rank_tol, DevState* state, cudaStream_t st) {
  if (m < 1 || m > kSmallMax || mp < m) return cudaErrorInvalidValue;
  if (is_f64)
    k_small_alpha<double><<<m + 1, kSmallThreads, 0, st>>>(m, mp, G, cvec, (double*)gi_t, (double*)xc_t, rank_tol,
                                                           state);
  else
    k_small_alpha<float><<<m + 1, kSmallThreads, 0, st>>>(m, mp, G, cvec, (float*)gi_t, (float*)xc_t, rank_tol,
                                                          state);
  return cudaGetLastError();
}

cudaError_t launch_small_beta(int is_f64, int mp, int m, const double* S, double* cvec, void* ti_t, void* t_t,
                              double rank_tol, DevState* state, cudaStream_t st) {
  if (m < 1 || m > kSmallMax || mp < m) return cudaErrorInvalidValue;
  if (is_f64)
    k_small_beta<double><<<m, kSmallThreads, 0, st>>>(m, mp, S, cvec, (double*)ti_t, (double*)t_t, rank_tol, state);
  else
    k_small_beta<float><<<m, kSmallThreads, 0, st>>>(m, mp, S, cvec, (float*)ti_t, (float*)t_t, rank_tol, state);
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

cudaError_t launch_update_p(int is_f64, int mp, int64_t d, int m, void* Q, void* P, int64_t ld, const void* xc_t,
                            const void* ti_t, const void* t_t, double* x, const DevState* state, cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (is_f64) {
    BK_DISPATCH_MP(mp, upd_p_d, d, m, Q, P, ld, xc_t, ti_t, t_t, x, state, st, dev);
  } else {
    BK_DISPATCH_MP(mp, upd_p_f, d, m, Q, P, ld, xc_t, ti_t, t_t, x, state, st, dev);
  }
}

cudaError_t launch_start_block(int is_f64, int64_t d, int m, int64_t ld, const double* r, double scale,
                               const void* omega, void* Q, double* x, cudaStream_t st) {
  int grid = capped_grid(d, 256, 152 * 8);
  if (is_f64)
    k_start_block<double><<<grid, 256, 0, st>>>(d, m, ld, r, scale, (const double*)omega, (double*)Q, x);
  else
    k_start_block<float><<<grid, 256, 0, st>>>(d, m, ld, r, scale, (const float*)omega, (float*)Q, x);
  return cudaGetLastError();
}

cudaError_t launch_init_state(DevState* state, int max_loads, double tol_abs, double* cvec, int m, cudaStream_t st) {
  k_init_state<<<1, 64, 0, st>>>(state, max_loads, tol_abs, cvec, m);
  return cudaGetLastError();
}

cudaError_t launch_axpy(int64_t d, double a, const double* y, double* x, cudaStream_t st) {
  k_axpy<<<capped_grid(d, 256, 152 * 8), 256, 0, st>>>(d, a, y, x);
  return cudaGetLastError();
}

cudaError_t launch_axpy_out(int64_t d, double a, const double* y, const double* x, double* out, cudaStream_t st) {
  k_axpy_out<<<capped_grid(d, 256, 152 * 8), 256, 0, st>>>(d, a, y, x, out);
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
