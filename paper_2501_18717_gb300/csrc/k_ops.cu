// Block products with A_mu = A + mu I ("matrix-loads", Sec. 1.2) and the FP64 residual.
//
// k_csr_spmm_gram: Y = A P + mu P for CSR A, reading each matrix row once for all m
//   columns (thread per row, the row's nonzeros held in registers), with G = P^T Y
//   formed in the same pass from the row tile staged in shared memory (bk_tile.cuh).
//   Blocks are stored in panels of four columns (bk_tile.cuh): one gather of row j of
//   a panel is a single 16-byte load, and for stencil-like sparsity neighbouring rows
//   touch neighbouring rows of P, so a warp's gathers are contiguous.
// k_dense_gram: the same for a dense row-major A (tiled over K in shared memory).
// k_*_residual: r = b - A_mu x in FP64 from the stored values, with ||r||^2 partials.
#include "bk_common.cuh"
#include "bk_tile.cuh"

namespace bk {
namespace {

__device__ __forceinline__ bool is_done(const DevState* s) { return s && (s->done_a | s->done_b); }

int sm_count_ops(int device) {
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n <= 0) n = 152;
  return n;
}

// ------------------------------------------------------------------ CSR
// Thread per row; the grid strides over row tiles, so for a stencil the tiles whose
// rows a tile gathers are being read at the same time by other CTAs and are served
// from L2. The row's nonzeros (up to KMAX, more are read in a tail loop) are held in
// registers; the panels are walked QU at a time, and all loads of a group
// (the row's own panel rows and nnz 16-byte gathers per panel) are issued before any
// of them is used, so up to QU (KMAX + 1) loads per thread are in flight (FP32: 3 CTAs
// per SM at up to 168 registers, no spill; with the next tile's row data read during
// the Gram this measured 3 % faster than 4 CTAs at 128 registers with a spill). Each panel
// row of the result goes to Y and, as one 16-byte store, to the row-major shared tile
// used by the fused Gram.
template <int MP>
__host__ __device__ constexpr int csr_group() { return (MP / 4) % 3 == 0 ? 3 : 2; }
template <typename T, int MP>
__host__ __device__ constexpr int csr_blocks() {
  return MP > 36 ? (sizeof(T) == 4 ? 2 : 1) : (sizeof(T) == 4 ? 3 : 2);
}

template <typename T, int MP, int TM, int KMAX>
__global__ void __launch_bounds__(TM, (csr_blocks<T, MP>()))
    k_csr_spmm_gram(int64_t d, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                    const T* __restrict__ vals, T mu, const T* __restrict__ P, T* __restrict__ Y, int64_t ld, int m,
                    double* parts, int nparts, const DevState* state) {
  constexpr int QU = csr_group<MP>();
  constexpr int NQ = MP / 4;
  if (is_done(state)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sX = reinterpret_cast<T*>(smem_raw);
  T* sY = sX + TM * MP;
  GramAcc<T, MP, gram_bpt<MP, TM>()> g;
  g.init();
  const int t = threadIdx.x;
  const int nq = (m + 3) >> 2;
  int64_t ntiles = (d + TM - 1) / TM;
  // The row's nonzeros for a tile. Those of the next tile are read before the Gram of
  // the current one, so the dependent rowptr -> colidx loads leave the tile's start.
  int k0 = 0, nz = 0;
  T v[KMAX];
  int off[KMAX];
  auto load_row = [&](int64_t tile) {
    const int64_t i = tile * TM + t;
    k0 = 0;
    nz = 0;
    if (i < d) {
      k0 = rowptr[i];
      nz = rowptr[i + 1] - k0;
    }
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      bool on = k < nz;
      v[k] = on ? vals[k0 + k] : (T)0;
      off[k] = on ? colidx[k0 + k] : 0;
    }
  };
  if (blockIdx.x < ntiles) load_row(blockIdx.x);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t i = tile * TM + t;
    const bool ok = i < d;
#pragma unroll 1
    for (int q0 = 0; q0 < NQ; q0 += QU) {
      T pv[QU][4], gv[QU][KMAX][4];
#pragma unroll
      for (int j = 0; j < QU; ++j) {  // every load of the group first
        const int q = q0 + j;
        const bool live = ok && q < NQ && q < nq;
        const T* pq = P + (int64_t)(q < NQ ? q : 0) * ld * 4;
        if (live)
          ldg4(pq + i * 4, pv[j]);
        else {
#pragma unroll
          for (int u = 0; u < 4; ++u) pv[j][u] = (T)0;
        }
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
          if (live && k < nz)
            ldg4(pq + (int64_t)off[k] * 4, gv[j][k]);
          else {
#pragma unroll
            for (int u = 0; u < 4; ++u) gv[j][k][u] = (T)0;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < QU; ++j) {
        const int q = q0 + j;
        if (q >= NQ) break;
        const bool live = ok && q < nq;
        T a[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = mu * pv[j][u];
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
#pragma unroll
          for (int u = 0; u < 4; ++u) a[u] = fma(v[k], gv[j][k][u], a[u]);
        if (live) {
          const T* pq = P + (int64_t)q * ld * 4;
          for (int k = KMAX; k < nz; ++k) {
            T gt[4];
            ldg4(pq + (int64_t)colidx[k0 + k] * 4, gt);
            const T vk = vals[k0 + k];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = fma(vk, gt[u], a[u]);
          }
          st4(Y + ((int64_t)q * ld + i) * 4, a);
        }
        store4<MP>(sX, t, q, pv[j]);
        store4<MP>(sY, t, q, a);
      }
    }
    __syncthreads();
    if (tile + gridDim.x < ntiles) load_row(tile + gridDim.x);
    gram_tile<TM, TM>(g, sX, sY);
    __syncthreads();
  }
  gram_finish<T, MP>(g, reinterpret_cast<double*>(smem_raw), parts, nparts, blockIdx.x);
}

// ------------------------------------------------------------------ dense
// CTA computes TMD rows x MP columns of Y. K is walked in chunks of KC: the A chunk
// (TMD x KC, coalesced along K) and the P chunk (KC x MP, coalesced along K per
// column) are staged in shared memory. Thread (r, cg) owns row r and the columns
// cg, cg + CG, ... (CG = threads / TMD).
template <typename T, int MP, int TMD, int KC, int NTH>
__global__ void __launch_bounds__(NTH) k_dense_gram(int64_t d, const T* __restrict__ A, int64_t lda, T mu,
                                                   const T* __restrict__ P, T* __restrict__ Y, int64_t ld, int m,
                                                   double* parts, int nparts, const DevState* state) {
  if (is_done(state)) return;
  constexpr int CG = NTH / TMD;
  constexpr int NC = (MP + CG - 1) / CG;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sA = reinterpret_cast<T*>(smem_raw);  // TMD x (KC + 1)
  T* sP = sA + TMD * (KC + 1);             // KC x MP
  T* sX = sP + KC * MP;                    // TMD x MP tiles for the Gram
  T* sY = sX + TMD * MP;
  GramAcc<T, MP, gram_bpt<MP, NTH>()> g;
  g.init();
  int r = threadIdx.x / CG, cg = threadIdx.x % CG;
  const int nq = (m + 3) >> 2;  // panels held in memory
  int64_t ntiles = (d + TMD - 1) / TMD;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int64_t row0 = tile * TMD;
    T acc[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) acc[q] = (T)0;
    for (int64_t k0 = 0; k0 < d; k0 += KC) {
      for (int idx = threadIdx.x; idx < TMD * KC; idx += NTH) {
        int rr = idx / KC, kk = idx - rr * KC;
        int64_t gr = row0 + rr, gk = k0 + kk;
        sA[rr * (KC + 1) + kk] = (gr < d && gk < d) ? A[gr * lda + gk] : (T)0;
      }
      for (int idx = threadIdx.x; idx < KC * (MP / 4); idx += NTH) {
        int q = idx / KC, kk = idx - q * KC;
        int64_t gk = k0 + kk;
        T pv[4] = {0, 0, 0, 0};
        if (gk < d && q < nq) ldg4(P + ((int64_t)q * ld + gk) * 4, pv);
#pragma unroll
        for (int u = 0; u < 4; ++u) sP[kk * MP + 4 * q + u] = pv[u];
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < KC; ++kk) {
        T a = sA[r * (KC + 1) + kk];
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          int c = cg + q * CG;
          if (c < MP) acc[q] = fma(a, sP[kk * MP + c], acc[q]);
        }
      }
      __syncthreads();
    }
    int64_t gi = row0 + r;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      int c = cg + q * CG;
      if (c < MP) {
        // only the panels of the m live columns exist in memory; the rest count as zero
        const bool live = gi < d && (c >> 2) < nq;
        const int64_t off = (((int64_t)(c >> 2) * ld + gi) << 2) + (c & 3);
        T pv = live ? P[off] : (T)0;
        T yv = live ? fma(mu, pv, acc[q]) : (T)0;
        if (live) Y[off] = yv;
        sX[r * MP + c] = pv;
        sY[r * MP + c] = yv;
      }
    }
    __syncthreads();
    g.tile(sX, sY, TMD);
    __syncthreads();
  }
  gram_finish<T, MP>(g, reinterpret_cast<double*>(smem_raw), parts, nparts, blockIdx.x);
}

// ------------------------------------------------------------------ FP64 residuals
constexpr int kResThreads = 256;

__device__ __forceinline__ void block_sum_to(double v, double* parts, double* red) {
  // deterministic CTA reduction: warp shuffle tree, then warp 0 over the warp sums
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    double s = (l < nw) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (l == 0) parts[blockIdx.x] = s;
  }
}

template <typename V>
__global__ void __launch_bounds__(kResThreads) k_csr_residual(int64_t d, const int* __restrict__ rowptr,
                                                             const int* __restrict__ colidx,
                                                             const V* __restrict__ vals, double mu,
                                                             const double* __restrict__ x,
                                                             const double* __restrict__ b, double* r,
                                                             double* norm_parts) {
  __shared__ double red[32];
  double ss = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
    double s = mu * x[i];
    int k0 = rowptr[i], k1 = rowptr[i + 1];
    for (int k = k0; k < k1; ++k) s = fma((double)vals[k], x[colidx[k]], s);
    double ri = b[i] - s;
    if (r) r[i] = ri;
    ss = fma(ri, ri, ss);
  }
  block_sum_to(ss, norm_parts, red);
}

template <typename V>
__global__ void __launch_bounds__(kResThreads) k_dense_residual(int64_t d, const V* __restrict__ A, int64_t lda,
                                                               double mu, const double* __restrict__ x,
                                                               const double* __restrict__ b, double* r,
                                                               double* norm_parts) {
  __shared__ double red[32];
  int lane = threadIdx.x & 31;
  int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double ss = 0.0;
  for (int64_t i = warp; i < d; i += nwarps) {
    double s = 0.0;
    const V* row = A + i * lda;
    for (int64_t k = lane; k < d; k += 32) s = fma((double)row[k], x[k], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    double ri = b[i] - (s + mu * x[i]);
    if (lane == 0) {
      if (r) r[i] = ri;
      ss = fma(ri, ri, ss);
    }
  }
  block_sum_to(ss, norm_parts, red);
}

// ------------------------------------------------------------------ dispatch helpers
template <typename T, int MP>
constexpr int csr_tm() {
  return 128;
}

template <typename T, int MP>
cudaError_t csr_impl(int64_t d, const int* rowptr, const int* colidx, const void* vals, double mu, const void* P,
                     void* Y, int64_t ld, int m, double* parts, int nparts, const DevState* state, cudaStream_t st) {
  constexpr int TM = csr_tm<T, MP>();
  size_t smem = gram_smem_bytes<T, MP>(TM, TM);
  auto kern = k_csr_spmm_gram<T, MP, TM, 7>;  // 7 nonzeros per row in registers (7-point stencils)
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<nparts, TM, smem, st>>>(d, rowptr, colidx, (const T*)vals, (T)mu, (const T*)P, (T*)Y, ld, m, parts, nparts,
                                 state);
  return cudaGetLastError();
}

template <typename T, int MP>
struct DenseCfg {
  static constexpr int TMD = 16, KC = 64, NTH = 128;
  static size_t smem() {
    size_t main = (size_t)(TMD * (KC + 1) + KC * MP + 2 * TMD * MP) * sizeof(T);
    size_t red = (size_t)gram_phases<MP>(NTH) * GramShape<MP>::NE * sizeof(double);
    return main > red ? main : red;
  }
};

template <typename T, int MP>
cudaError_t dense_impl(int64_t d, const void* A, int64_t lda, double mu, const void* P, void* Y, int64_t ld, int m,
                       double* parts, int nparts, const DevState* state, cudaStream_t st) {
  using C = DenseCfg<T, MP>;
  size_t smem = C::smem();
  auto kern = k_dense_gram<T, MP, C::TMD, C::KC, C::NTH>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<nparts, C::NTH, smem, st>>>(d, (const T*)A, lda, (T)mu, (const T*)P, (T*)Y, ld, m, parts, nparts, state);
  return cudaGetLastError();
}

#define BK_DISPATCH_MP2(mp, F, ...)        \
  switch (mp) {                            \
    case 4: return F<4>(__VA_ARGS__);      \
    case 8: return F<8>(__VA_ARGS__);      \
    case 16: return F<16>(__VA_ARGS__);    \
    case 24: return F<24>(__VA_ARGS__);    \
    case 36: return F<36>(__VA_ARGS__);    \
    case 68: return F<68>(__VA_ARGS__);    \
    default: return cudaErrorInvalidValue; \
  }

template <int MP>
cudaError_t csr_d(int64_t d, const int* rp, const int* ci, const void* v, double mu, const void* P, void* Y,
                  int64_t ld, int m, double* parts, int np, const DevState* s, cudaStream_t st) {
  return csr_impl<double, MP>(d, rp, ci, v, mu, P, Y, ld, m, parts, np, s, st);
}
template <int MP>
cudaError_t csr_f(int64_t d, const int* rp, const int* ci, const void* v, double mu, const void* P, void* Y,
                  int64_t ld, int m, double* parts, int np, const DevState* s, cudaStream_t st) {
  return csr_impl<float, MP>(d, rp, ci, v, mu, P, Y, ld, m, parts, np, s, st);
}
template <int MP>
cudaError_t dense_d(int64_t d, const void* A, int64_t lda, double mu, const void* P, void* Y, int64_t ld, int m,
                    double* parts, int np, const DevState* s, cudaStream_t st) {
  return dense_impl<double, MP>(d, A, lda, mu, P, Y, ld, m, parts, np, s, st);
}
template <int MP>
cudaError_t dense_f(int64_t d, const void* A, int64_t lda, double mu, const void* P, void* Y, int64_t ld, int m,
                    double* parts, int np, const DevState* s, cudaStream_t st) {
  return dense_impl<float, MP>(d, A, lda, mu, P, Y, ld, m, parts, np, s, st);
}

}  // namespace

int csr_spmm_gram_grid(int is_f64, int mp, int64_t d, int device) {
  int tm = 128;
  int64_t ntiles = (d + tm - 1) / tm;
  // resident CTAs per SM (the launch bounds of csr_blocks)
  int cap = sm_count_ops(device) * (mp > 36 ? (is_f64 ? 1 : 2) : (is_f64 ? 2 : 3));
  if (ntiles < 1) ntiles = 1;
  return (int)(ntiles < cap ? ntiles : cap);
}

int dense_gram_grid(int is_f64, int mp, int64_t d, int device) {
  int64_t ntiles = (d + 15) / 16;
  int cap = sm_count_ops(device) * 4;
  if (ntiles < 1) ntiles = 1;
  return (int)(ntiles < cap ? ntiles : cap);
}

cudaError_t launch_csr_spmm_gram(int is_f64, int mp, int64_t d, const int* rowptr, const int* colidx,
                                 const void* vals, double mu, const void* P, void* Y, int64_t ld, int m,
                                 double* parts, int nparts, const DevState* state, cudaStream_t st) {
  if (is_f64) {
    BK_DISPATCH_MP2(mp, csr_d, d, rowptr, colidx, vals, mu, P, Y, ld, m, parts, nparts, state, st);
  } else {
    BK_DISPATCH_MP2(mp, csr_f, d, rowptr, colidx, vals, mu, P, Y, ld, m, parts, nparts, state, st);
  }
}

cudaError_t launch_dense_gram(int is_f64, int mp, int64_t d, const void* A, int64_t lda, double mu, const void* P,
                              void* Y, int64_t ld, int m, double* parts, int nparts, const DevState* state,
                              cudaStream_t st) {
  if (is_f64) {
    BK_DISPATCH_MP2(mp, dense_d, d, A, lda, mu, P, Y, ld, m, parts, nparts, state, st);
  } else {
    BK_DISPATCH_MP2(mp, dense_f, d, A, lda, mu, P, Y, ld, m, parts, nparts, state, st);
  }
}

int residual_parts(int64_t d) {
  int64_t g = (d + kResThreads - 1) / kResThreads;
  if (g < 1) g = 1;
  if (g > 1024) g = 1024;
  return (int)g;
}

cudaError_t launch_csr_residual(int vals_f64, int64_t d, const int* rowptr, const int* colidx, const void* vals,
                                double mu, const double* x, const double* b, double* r, double* norm_parts,
                                int nparts, cudaStream_t st) {
  if (vals_f64)
    k_csr_residual<double><<<nparts, kResThreads, 0, st>>>(d, rowptr, colidx, (const double*)vals, mu, x, b, r,
                                                           norm_parts);
  else
    k_csr_residual<float><<<nparts, kResThreads, 0, st>>>(d, rowptr, colidx, (const float*)vals, mu, x, b, r,
                                                          norm_parts);
  return cudaGetLastError();
}

cudaError_t launch_dense_residual(int vals_f64, int64_t d, const void* A, int64_t lda, double mu, const double* x,
                                  const double* b, double* r, double* norm_parts, int nparts, cudaStream_t st) {
  if (vals_f64)
    k_dense_residual<double><<<nparts, kResThreads, 0, st>>>(d, (const double*)A, lda, mu, x, b, r, norm_parts);
  else
    k_dense_residual<float><<<nparts, kResThreads, 0, st>>>(d, (const float*)A, lda, mu, x, b, r, norm_parts);
  return cudaGetLastError();
}

}  // namespace bk
