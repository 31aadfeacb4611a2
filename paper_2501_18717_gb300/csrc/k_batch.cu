// Batched block-CG: many independent dense SPD systems of uneven size advance together,
// one launch per step kernel for the whole batch. Every system owns a contiguous range
// of thread blocks (sized by its share of the work) in the block kernels and one thread
// block in the small solves, so partial Grams and control state stay per system and
// every sum is formed in a fixed order. The steps are those of bk_solve (Def. BCG in
// the orthonormal-residual form, R = Q C with c = C e_1): Y = A_mu P with G = P^T Y;
// Gi = G^+, xc = G^+ c; W = Q - Y Gi with S = W^T W; S = T^T T, c <- T c;
// x += P xc, Q = W T^{-1}, P = Q + P T^T.
#include "bk_batch.cuh"
#include "bk_common.cuh"
#include "bk_rng.cuh"
#include "bk_small.cuh"
#include "bk_tile.cuh"
#include "bk_update.cuh"

namespace bk {
namespace {

__device__ __forceinline__ bool sys_done(const BSys& s) { return s.st->done_a | s.st->done_b; }

// ---------------------------------------------------------------- block product
// Row tiles of TMD rows; thread (r, cg) owns row r and columns cg, cg + CG, ...
template <typename T, typename VA, int MP, int TMD, int KC, int NTH>
__global__ void __launch_bounds__(NTH) k_bop(const BSys* __restrict__ sys, const int* __restrict__ cta_sys) {
  const BSys S = sys[cta_sys[blockIdx.x]];
  if (sys_done(S)) return;
  const int j = blockIdx.x - S.cta0;
  constexpr int CG = NTH / TMD;
  constexpr int NC = (MP + CG - 1) / CG;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sA = reinterpret_cast<T*>(smem_raw);
  T* sP = sA + TMD * (KC + 1);
  T* sX = sP + KC * MP;
  T* sY = sX + TMD * MP;
  const VA* A = static_cast<const VA*>(S.A);
  const T* P = static_cast<const T*>(S.P);
  T* Y = static_cast<T*>(S.Y);
  const int64_t d = S.d, lda = S.lda, ld = S.ld;
  const T mu = (T)S.mu;
  GramAcc<T, MP, gram_bpt<MP, NTH>()> g;
  g.init();
  const int r = threadIdx.x / CG, cg = threadIdx.x % CG;
  const int nq = (S.m + 3) >> 2;
  const int64_t ntiles = (d + TMD - 1) / TMD;
  for (int64_t tile = j; tile < ntiles; tile += S.ncta) {
    const int64_t row0 = tile * TMD;
    T acc[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) acc[q] = (T)0;
    for (int64_t k0 = 0; k0 < d; k0 += KC) {
      for (int idx = threadIdx.x; idx < TMD * KC; idx += NTH) {
        const int rr = idx / KC, kk = idx - rr * KC;
        const int64_t gr = row0 + rr, gk = k0 + kk;
        sA[rr * (KC + 1) + kk] = (gr < d && gk < d) ? (T)A[gr * lda + gk] : (T)0;
      }
      for (int idx = threadIdx.x; idx < KC * (MP / 4); idx += NTH) {
        const int q = idx / KC, kk = idx - q * KC;
        const int64_t gk = k0 + kk;
        T pv[4] = {0, 0, 0, 0};
        if (gk < d && q < nq) ldg4(P + ((int64_t)q * ld + gk) * 4, pv);
#pragma unroll
        for (int u = 0; u < 4; ++u) sP[kk * MP + 4 * q + u] = pv[u];
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < KC; ++kk) {
        const T a = sA[r * (KC + 1) + kk];
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          const int c = cg + q * CG;
          if (c < MP) acc[q] = fma(a, sP[kk * MP + c], acc[q]);
        }
      }
      __syncthreads();
    }
    const int64_t gi = row0 + r;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const int c = cg + q * CG;
      if (c < MP) {
        const bool live = gi < d && (c >> 2) < nq;
        const int64_t off = (((int64_t)(c >> 2) * ld + gi) << 2) + (c & 3);
        const T pv = live ? P[off] : (T)0;
        const T yv = live ? fma(mu, pv, acc[q]) : (T)0;
        if (live) Y[off] = yv;
        sX[r * MP + c] = pv;
        sY[r * MP + c] = yv;
      }
    }
    __syncthreads();
    gram_tile<TMD, NTH>(g, sX, sY);
    __syncthreads();
  }
  gram_finish<T, MP>(g, reinterpret_cast<double*>(smem_raw), S.Gp, S.ncta, j);
}

// ---------------------------------------------------------------- residual update + Gram
template <typename T, int MP, int TM>
__global__ void __launch_bounds__(TM) k_bupd_r(const BSys* __restrict__ sys, const int* __restrict__ cta_sys) {
  const BSys S = sys[cta_sys[blockIdx.x]];
  if (sys_done(S)) return;
  const int j = blockIdx.x - S.cta0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sA = reinterpret_cast<T*>(smem_raw);
  T* sX = sA + MP * MP;
  const T* at = static_cast<const T*>(S.gi_t);
  for (int idx = threadIdx.x; idx < MP * MP; idx += blockDim.x) sA[idx] = at[idx];
  __syncthreads();
  const T* Y = static_cast<const T*>(S.Y);
  T* R = static_cast<T*>(S.Q);  // W = Q - Y Gi overwrites Q
  const int64_t d = S.d, ld = S.ld;
  const int m = S.m;
  GramAcc<T, MP, gram_bpt<MP, TM>()> g;
  g.init();
  const int64_t ntiles = (d + TM - 1) / TM;
  for (int64_t tile = j; tile < ntiles; tile += S.ncta) {
    const int64_t i = tile * TM + threadIdx.x;
    const bool ok = i < d;
    asm volatile("" ::: "memory");
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
    gram_tile<TM, TM>(g, sX, sX);
    __syncthreads();
  }
  gram_finish<T, MP>(g, reinterpret_cast<double*>(smem_raw + ((MP * MP * sizeof(T) + 15) / 16) * 16), S.Sp,
                     S.ncta, j);
}

// ---------------------------------------------------------------- Gram of Q (start)
template <typename T, int MP, int TM>
__global__ void __launch_bounds__(TM) k_bgram_r(const BSys* __restrict__ sys, const int* __restrict__ cta_sys) {
  const BSys S = sys[cta_sys[blockIdx.x]];
  if (S.active == 0) return;
  const int j = blockIdx.x - S.cta0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sX = reinterpret_cast<T*>(smem_raw);
  const T* R = static_cast<const T*>(S.Q);
  const int64_t d = S.d, ld = S.ld;
  GramAcc<T, MP, gram_bpt<MP, TM>()> g;
  g.init();
  const int64_t ntiles = (d + TM - 1) / TM;
  for (int64_t tile = j; tile < ntiles; tile += S.ncta) {
    const int64_t i = tile * TM + threadIdx.x;
    T v[MP];
#pragma unroll
    for (int q = 0; q < MP / 4; ++q) {
      if (i < d && 4 * q < S.m)
        ldg4(panel_row(R, ld, q, i), v + 4 * q);
      else {
#pragma unroll
        for (int u = 0; u < 4; ++u) v[4 * q + u] = (T)0;
      }
    }
    store_row<MP>(sX, threadIdx.x, v);
    __syncthreads();
    gram_tile<TM, TM>(g, sX, sX);
    __syncthreads();
  }
  gram_finish<T, MP>(g, reinterpret_cast<double*>(smem_raw), S.Sp, S.ncta, j);
}

// ---------------------------------------------------------------- direction update
// x += P xc; unless the inner solve stopped, Q = W T^{-1} and P = Q + P T^T (P = Q on
// the start call); the row loop is update_pq_rows.
template <typename T, int MP>
constexpr size_t bupd_p_smem() {
  return MP > 36 ? 2 * (size_t)MP * MP * sizeof(T) : 0;
}

template <typename T, int MP, int NTH>
__global__ void __launch_bounds__(NTH) k_bupd_p(const BSys* __restrict__ sys, const int* __restrict__ cta_sys) {
  const BSys S = sys[cta_sys[blockIdx.x]];
  const bool do_x = S.st->pending_x;
  const bool upd = !(S.st->done_a | S.st->done_b);
  if (!do_x && !upd) return;
  const bool first = S.st->first;
  const int j = blockIdx.x - S.cta0;
  // above width 36 the two tables are in dynamic shared memory (two FP64 68 x 68
  // tables exceed the 48 KB of static shared memory)
  constexpr bool kDyn = MP > 36;
  __shared__ __align__(16) T sTi_s[kDyn ? 1 : MP * MP];
  __shared__ __align__(16) T sTT_s[kDyn ? 1 : MP * MP];
  __shared__ __align__(16) T sxc[MP];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sTi = kDyn ? reinterpret_cast<T*>(smem_raw) : sTi_s;
  T* sTT = kDyn ? reinterpret_cast<T*>(smem_raw) + MP * MP : sTT_s;
  const T* ti = static_cast<const T*>(S.ti_t);
  const T* tt = static_cast<const T*>(S.t_t);
  const T* xc = static_cast<const T*>(S.xc_t);
  for (int idx = threadIdx.x; idx < MP * MP; idx += NTH) {
    sTi[idx] = ti[idx];
    sTT[idx] = first ? (T)0 : tt[idx];
  }
  for (int idx = threadIdx.x; idx < MP; idx += NTH) sxc[idx] = do_x ? xc[idx] : (T)0;
  __syncthreads();
  const int m = S.m;
  T* Q = static_cast<T*>(S.Q);
  T* P = static_cast<T*>(S.P);
  const int64_t d = S.d, ld = S.ld;
  update_pq_rows<T, MP>((int64_t)j * NTH + threadIdx.x, (int64_t)S.ncta * NTH, d, m, Q, P, ld, sTi, sTT, sxc, do_x,
                        upd, S.xin);
}

// ---------------------------------------------------------------- small solves
constexpr int kBSmall = 128;

// Sum of the per-CTA Gram partials (fixed order) into a full symmetric m x m matrix in
// shared memory (stride kLds).
template <int MP>
__device__ void reduce_parts(const double* parts, int nparts, int m, double* W) {
  using GS = GramShape<MP>;
  for (int e = threadIdx.x; e < GS::NE; e += blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) s += parts[(size_t)e * nparts + p];
    const int t = e >> 4, q = e & 15;
    int tt = t, r = 0;
    while (tt >= GS::NB - r) {
      tt -= GS::NB - r;
      ++r;
    }
    const int row = 4 * r + (q >> 2), col = 4 * (r + tt) + (q & 3);
    if (row <= col && col < m) {
      W[row * kLds + col] = s;
      W[col * kLds + row] = s;
    }
  }
}

// Z (m x nc, row-major, shared) <- D^{-1/2} L^{-T} [L^{-1}] D^{-1/2} Z on the kept
// columns of the factorisation in sh: with forward = true the pseudo-inverse M^+ of the
// factored matrix applied to Z; with forward = false, Z <- (T^+) Z for T = L^T D^{1/2}
// (only the backward substitution, and no input scaling). The threads of the block
// share the columns of each substitution step.
__device__ void apply_factor(const SmallShared& sh, int m, int nc, double* Z, bool forward) {
  const int tid = threadIdx.x;
  if (forward) {
    for (int idx = tid; idx < m * nc; idx += kBSmall) Z[idx] *= sh.z[idx / nc];
    __syncthreads();
    for (int k = 0; k < m; ++k) {
      const double inv = sh.invd[k];
      for (int q = tid; q < nc; q += kBSmall) Z[k * nc + q] *= inv;
      __syncthreads();
      for (int idx = tid; idx < (m - k - 1) * nc; idx += kBSmall) {
        const int i = k + 1 + idx / nc, q = idx % nc;
        Z[i * nc + q] = fma(-sh.W[i * kLds + k], Z[k * nc + q], Z[i * nc + q]);
      }
      __syncthreads();
    }
  }
  for (int k = m - 1; k >= 0; --k) {
    const double inv = sh.invd[k];
    for (int q = tid; q < nc; q += kBSmall) Z[k * nc + q] *= inv;
    __syncthreads();
    for (int idx = tid; idx < k * nc; idx += kBSmall) {
      const int i = idx / nc, q = idx % nc;
      Z[i * nc + q] = fma(-sh.W[k * kLds + i], Z[k * nc + q], Z[i * nc + q]);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < m * nc; idx += kBSmall) Z[idx] *= sh.z[idx / nc];
  __syncthreads();
}

// mode 0 (alpha): Gi = G^+ and xc = G^+ c (G reduced from Gp); one more load.
// mode 1 (beta): S = W^T W (reduced from Sp) = T^T T; T^+ and T^T (row-major) for the
// direction update, c <- T c and the stopping decision on ||c||. The start of an inner solve is a
// mode-1 call on S = Q^T Q with c = e_1.
// Zs (MP x (MP + 1)) and cn (MP) are in dynamic shared memory (bsmall_smem bytes).
template <int MP>
constexpr size_t bsmall_smem() {
  return (size_t)(MP * (MP + 1) + MP) * sizeof(double);
}

template <typename T, int MP>
__global__ void __launch_bounds__(kBSmall) k_bsmall(BSys* __restrict__ sys, int mode, double rank_tol) {
  BSys& S = sys[blockIdx.x];
  __shared__ SmallShared sh;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Zs = reinterpret_cast<double*>(smem_raw);
  double* cn = Zs + MP * (MP + 1);
  const int m = S.m;
  DevState* st = S.st;
  if (st->done_a | st->done_b) {
    if (mode == 0 && threadIdx.x == 0) st->pending_x = 0;
    return;
  }
  reduce_parts<MP>(mode == 0 ? S.Gp : S.Sp, mode == 0 ? S.npG : S.ncta, m, sh.W);
  __syncthreads();
  const int rank = block_cholesky_skip<kBSmall>(sh, m, rank_tol);
  if (mode == 0) {
    if (rank > 0) {
      const int nc = m + 1;  // columns of I, then c
      for (int idx = threadIdx.x; idx < m * nc; idx += kBSmall) {
        const int i = idx / nc, q = idx % nc;
        Zs[idx] = q < m ? (i == q ? 1.0 : 0.0) : S.cvec[i];
      }
      __syncthreads();
      apply_factor(sh, m, nc, Zs, true);
      T* gi = static_cast<T*>(S.gi_t);
      T* xc = static_cast<T*>(S.xc_t);
      for (int idx = threadIdx.x; idx < MP * MP; idx += kBSmall) {
        const int i = idx / MP, q = idx % MP;
        gi[idx] = (T)((i < m && q < m) ? Zs[i * nc + q] : 0.0);
      }
      for (int i = threadIdx.x; i < MP; i += kBSmall) xc[i] = (T)(i < m ? Zs[i * nc + m] : 0.0);
    }
    if (threadIdx.x == 0) {
      st->loads += 1;
      st->first = 0;
      if (rank <= 0) {
        st->pending_x = 0;
        st->done_a = 1;
        st->status = ST_BREAKDOWN;
      } else {
        st->pending_x = 1;
      }
    }
    return;
  }
  // mode 1
  if (rank < 0) {
    if (threadIdx.x == 0) {
      st->done_b = 1;
      st->status = ST_BREAKDOWN;
    }
    return;
  }
  for (int idx = threadIdx.x; idx < m * m; idx += kBSmall) Zs[idx] = (idx / m == idx % m) ? 1.0 : 0.0;
  for (int i = threadIdx.x; i < m; i += kBSmall) {
    double s = 0.0;
    for (int k = i; k < m; ++k) s = fma(sh.W[k * kLds + i] * sh.dscale[k], S.cvec[k], s);
    cn[i] = s;
  }
  __syncthreads();
  apply_factor(sh, m, m, Zs, false);  // Zs = T^+
  T* ti = static_cast<T*>(S.ti_t);
  T* tt = static_cast<T*>(S.t_t);
  for (int idx = threadIdx.x; idx < MP * MP; idx += kBSmall) {
    const int r = idx / MP, c = idx % MP;  // row r of T^+ and of T^T
    const bool in = r < m && c < m;
    ti[idx] = (T)(in ? Zs[r * m + c] : 0.0);
    tt[idx] = (T)((in && c <= r) ? sh.W[r * kLds + c] * sh.dscale[r] : 0.0);
  }
  for (int i = threadIdx.x; i < m; i += kBSmall) S.cvec[i] = cn[i];
  if (threadIdx.x == 0) {
    st->kept = rank;
    double ss = 0.0;
    for (int i = 0; i < m; ++i) ss = fma(cn[i], cn[i], ss);
    const double res = sqrt(ss);
    st->res = res;
    const bool conv = res <= st->tol_abs;
    if (conv || st->loads >= st->max_loads) {
      st->done_b = 1;
      st->status = conv ? ST_CONVERGED : ST_LOADCAP;
    } else if (!(res <= kDivergedRes)) {
      st->done_b = 1;
      st->status = ST_BREAKDOWN;
    }
  }
}

// ---------------------------------------------------------------- start block
// Active systems: Q = [r / ||r||, Omega / sqrt(d)] (Omega from Philox stream 3 with key
// seed + system index), x = 0, c = e_1, control block reset for a new inner solve.
template <typename T>
__global__ void k_bstart(BSys* __restrict__ sys, const int* __restrict__ cta_sys, uint64_t seed) {
  BSys& S = sys[cta_sys[blockIdx.x]];
  const int j = blockIdx.x - S.cta0;
  if (j == 0) {
    for (int i = threadIdx.x; i < S.m; i += blockDim.x) S.cvec[i] = i == 0 ? 1.0 : 0.0;
    if (threadIdx.x == 0) {
      DevState* st = S.st;
      st->done_a = S.active ? 0 : 1;
      st->done_b = 0;
      st->pending_x = 0;
      st->first = 1;
      st->loads = 0;
      st->status = S.active ? ST_RUNNING : ST_CONVERGED;
      st->max_loads = S.max_loads;
      st->timeout = 0;
      st->kept = S.m;
      st->tol_abs = S.tol_abs;
      st->res = 1.0;
    }
  }
  if (!S.active) return;
  const int64_t d = S.d, ld = S.ld;
  const int m = S.m, nq = (m + 3) >> 2;
  const double scale0 = S.rscale, scale = rsqrt((double)d);
  T* Q = static_cast<T*>(S.Q);
  const uint64_t key = seed + (uint64_t)S.index;
  for (int64_t i = (int64_t)j * blockDim.x + threadIdx.x; i < d; i += (int64_t)S.ncta * blockDim.x) {
    for (int q = 0; q < nq; ++q) {
      T v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = 4 * q + u;
        double val = 0.0;
        if (c == 0)
          val = S.r64[i] * scale0;
        else if (c < m)
          val = normal_at(key, 3u, (uint64_t)(c - 1) * d + i) * scale;
        v[u] = (T)val;
      }
      st4(panel_row(Q, ld, q, i), v);
    }
    S.xin[i] = 0.0;
  }
}

// ---------------------------------------------------------------- refinement
// x64 += ||r|| xin for systems that just ran an inner solve.
__global__ void k_baxpy(BSys* __restrict__ sys, const int* __restrict__ cta_sys) {
  const BSys S = sys[cta_sys[blockIdx.x]];
  if (!S.active) return;
  const int j = blockIdx.x - S.cta0;
  for (int64_t i = (int64_t)j * blockDim.x + threadIdx.x; i < S.d; i += (int64_t)S.ncta * blockDim.x)
    S.x64[i] = fma(S.rnorm, S.xin[i], S.x64[i]);
}

// r = b - (A x + mu x) in FP64 from the stored values (warp per row); per-CTA partial of
// ||r||^2 in rnorm_parts[blockIdx.x] (every system, also the converged ones).
template <typename V>
__global__ void __launch_bounds__(256) k_bresid(BSys* __restrict__ sys, const int* __restrict__ cta_sys,
                                               double* rnorm_parts) {
  const BSys S = sys[cta_sys[blockIdx.x]];
  const int j = blockIdx.x - S.cta0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const V* A = static_cast<const V*>(S.A64);
  __shared__ double red[8];
  double ss = 0.0;
  for (int64_t i = (int64_t)j * nw + warp; i < S.d; i += (int64_t)S.ncta * nw) {
    const V* row = A + i * S.lda;
    double s = 0.0;
    for (int64_t k = lane; k < S.d; k += 32) s = fma((double)row[k], S.x64[k], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const double ri = S.b[i] - (s + S.mu * S.x64[i]);
    if (lane == 0) {
      S.r64[i] = ri;
      ss = fma(ri, ri, ss);
    }
  }
  if (lane == 0) red[warp] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    rnorm_parts[blockIdx.x] = t;
  }
}

template <typename T, int MP, int TMD>
size_t bop_smem() {
  constexpr int KC = 64, NTH = 128;
  size_t main = (size_t)(TMD * (KC + 1) + KC * MP + 2 * TMD * MP) * sizeof(T);
  size_t red = (size_t)gram_phases<MP>(NTH) * GramShape<MP>::NE * sizeof(double);
  return main > red ? main : red;
}

// Dynamic shared memory limits of the small solve and the direction update (the small
// solve's static and dynamic parts together exceed 48 KB).
template <typename T, int MP>
cudaError_t small_attrs() {
  cudaError_t e =
      cudaFuncSetAttribute(k_bsmall<T, MP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsmall_smem<MP>());
  if (e == cudaSuccess && bupd_p_smem<T, MP>())
    e = cudaFuncSetAttribute(k_bupd_p<T, MP, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bupd_p_smem<T, MP>());
  return e;
}

template <typename T, typename VA, int MP, int TMD>
cudaError_t bop_launch(BSys* sys, const int* cta_sys, int ncta, cudaStream_t st) {
  auto k = k_bop<T, VA, MP, TMD, 64, 128>;
  const size_t sm = bop_smem<T, MP, TMD>();
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k<<<ncta, 128, sm, st>>>(sys, cta_sys);
  return cudaGetLastError();
}

template <typename T, typename VA, int MP>
cudaError_t step_impl(BSys* sys, int nsys, const int* cta_sys, int ncta, double rank_tol, const BatchTc* tc,
                      int tile_rows, cudaStream_t st) {
  cudaError_t e;
  if ((e = small_attrs<T, MP>()) != cudaSuccess) return e;
  if (tc)
    e = launch_batch_dense_tc(MP, sys, cta_sys, ncta, *tc, st);
  else if (tile_rows == 32)
    e = bop_launch<T, VA, MP, 32>(sys, cta_sys, ncta, st);
  else
    e = bop_launch<T, VA, MP, 16>(sys, cta_sys, ncta, st);
  if (e != cudaSuccess) return e;
  k_bsmall<T, MP><<<nsys, kBSmall, bsmall_smem<MP>(), st>>>(sys, 0, rank_tol);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    auto k = k_bupd_r<T, MP, 128>;
    size_t sm = ((MP * MP * sizeof(T) + 15) / 16) * 16 + gram_smem_bytes<T, MP>(128, 128);
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess) return e;
    k<<<ncta, 128, sm, st>>>(sys, cta_sys);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_bsmall<T, MP><<<nsys, kBSmall, bsmall_smem<MP>(), st>>>(sys, 1, rank_tol);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_bupd_p<T, MP, 128><<<ncta, 128, bupd_p_smem<T, MP>(), st>>>(sys, cta_sys);
  return cudaGetLastError();
}

template <typename T, int MP>
cudaError_t start_impl(BSys* sys, int nsys, const int* cta_sys, int ncta, uint64_t seed, double rank_tol,
                       cudaStream_t st) {
  cudaError_t e;
  if ((e = small_attrs<T, MP>()) != cudaSuccess) return e;
  k_bstart<T><<<ncta, 128, 0, st>>>(sys, cta_sys, seed);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  auto k = k_bgram_r<T, MP, 128>;
  size_t sm = gram_smem_bytes<T, MP>(128, 128);
  if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess) return e;
  k<<<ncta, 128, sm, st>>>(sys, cta_sys);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_bsmall<T, MP><<<nsys, kBSmall, bsmall_smem<MP>(), st>>>(sys, 1, rank_tol);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_bupd_p<T, MP, 128><<<ncta, 128, bupd_p_smem<T, MP>(), st>>>(sys, cta_sys);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_batch_step(int is_f64, int vals_f64, int mp, BSys* sys, int nsys, const int* cta_sys, int ncta,
                              double rank_tol, const BatchTc* tc, int tile_rows, cudaStream_t st) {
  if (!is_f64 && vals_f64) return cudaErrorInvalidValue;  // FP32 blocks take FP32 values
  if (tc && is_f64) return cudaErrorInvalidValue;          // the tensor-core product is FP32
  if (tile_rows != 16 && tile_rows != 32) return cudaErrorInvalidValue;
#define BK_B(MPV)                                                                                        \
  case MPV:                                                                                              \
    return is_f64 ? (vals_f64 ? step_impl<double, double, MPV>(sys, nsys, cta_sys, ncta, rank_tol, nullptr, \
                                                               tile_rows, st)                            \
                              : step_impl<double, float, MPV>(sys, nsys, cta_sys, ncta, rank_tol, nullptr,  \
                                                              tile_rows, st))                             \
                  : step_impl<float, float, MPV>(sys, nsys, cta_sys, ncta, rank_tol, tc, tile_rows, st);
  switch (mp) {
    BK_B(4)
    BK_B(8)
    BK_B(16)
    BK_B(24)
    BK_B(36)
    BK_B(68)
    default: return cudaErrorInvalidValue;
  }
#undef BK_B
}

cudaError_t launch_batch_start(int is_f64, int mp, BSys* sys, int nsys, const int* cta_sys, int ncta, uint64_t seed,
                               double rank_tol, cudaStream_t st) {
#define BK_B(MPV)                                                                           \
  case MPV:                                                                                 \
    return is_f64 ? start_impl<double, MPV>(sys, nsys, cta_sys, ncta, seed, rank_tol, st)   \
                  : start_impl<float, MPV>(sys, nsys, cta_sys, ncta, seed, rank_tol, st);
  switch (mp) {
    BK_B(4)
    BK_B(8)
    BK_B(16)
    BK_B(24)
    BK_B(36)
    BK_B(68)
    default: return cudaErrorInvalidValue;
  }
#undef BK_B
}

cudaError_t launch_batch_axpy(BSys* sys, const int* cta_sys, int ncta, cudaStream_t st) {
  k_baxpy<<<ncta, 256, 0, st>>>(sys, cta_sys);
  return cudaGetLastError();
}

cudaError_t launch_batch_resid(int vals_f64, BSys* sys, const int* cta_sys, int ncta, double* rnorm_parts,
                               cudaStream_t st) {
  if (vals_f64)
    k_bresid<double><<<ncta, 256, 0, st>>>(sys, cta_sys, rnorm_parts);
  else
    k_bresid<float><<<ncta, 256, 0, st>>>(sys, cta_sys, rnorm_parts);
  return cudaGetLastError();
}

}  // namespace bk
