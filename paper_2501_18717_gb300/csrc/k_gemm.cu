// Dense products for the block-Lanczos drivers (ridge path, sampling): the Gram-form
// operator Z^T (Z P), the dense operator for wide blocks, the reorthogonalisation
// products Q^T W and W - Q C, and the basis combination Q Z (Sec. 3.2, Thm. cost:
// O(d m^2 t^2) work for full reorthogonalisation, O(d m t) per shift for the combine).
//
// C = alpha * A * B + beta * C with general element strides, so one kernel serves
// row-major, column-major and transposed operands:
//   A(i, k) = A[i * sai + k * sak]   (M x K)
//   B(k, j) = B[k * sbk + j * sbj]   (K x N)
//   C(i, j) = C[i + j * ldc]         (M x N, column-major)
// Tiles of 64 x 64 outputs, K in steps of 16 staged in shared memory, 256 threads with
// 4 x 4 outputs each, accumulation in the element type of C (FP32 or FP64). A and B may
// each be FP32 or FP64; the tile loader reads along whichever stride is unit so the
// global loads coalesce.
#include <algorithm>

#include "bk_common.cuh"

namespace bk {
namespace {

constexpr int GBM = 64, GBN = 64, GBK = 16, GTH = 256;

template <typename TA, typename TB, typename TC>
__global__ void __launch_bounds__(GTH) k_gemm(int64_t M, int64_t N, int64_t K, TC alpha, const TA* __restrict__ A,
                                             int64_t sai, int64_t sak, const TB* __restrict__ B, int64_t sbk,
                                             int64_t sbj, TC beta, TC* __restrict__ C, int64_t ldc,
                                             int64_t kchunk, int64_t zstride) {
  // split-K: CTA z covers k in [z kchunk, (z + 1) kchunk) and writes its own C + z zstride
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = kbeg + kchunk < K ? kbeg + kchunk : K;
  C += (int64_t)blockIdx.z * zstride;
  __shared__ TC sA[GBK][GBM + 4];
  __shared__ TC sB[GBK][GBN + 4];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;  // 16 x 16 threads, 4 x 4 outputs each
  const int64_t i0 = (int64_t)blockIdx.x * GBM, j0 = (int64_t)blockIdx.y * GBN;
  TC acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = (TC)0;
  const bool a_rows_fast = (sai == 1);  // consecutive i contiguous
  const bool b_rows_fast = (sbk == 1);  // consecutive k contiguous
  for (int64_t k0 = kbeg; k0 < kend; k0 += GBK) {
    // A tile: GBM x GBK elements, 4 per thread
#pragma unroll
    for (int e = 0; e < (GBM * GBK) / GTH; ++e) {
      int idx = tid + e * GTH;
      int ii, kk;
      if (a_rows_fast) {
        ii = idx % GBM;
        kk = idx / GBM;
      } else {
        kk = idx % GBK;
        ii = idx / GBK;
      }
      int64_t gi = i0 + ii, gk = k0 + kk;
      sA[kk][ii] = (gi < M && gk < kend) ? (TC)A[gi * sai + gk * sak] : (TC)0;
    }
#pragma unroll
    for (int e = 0; e < (GBN * GBK) / GTH; ++e) {
      int idx = tid + e * GTH;
      int jj, kk;
      if (b_rows_fast) {
        kk = idx % GBK;
        jj = idx / GBK;
      } else {
        jj = idx % GBN;
        kk = idx / GBN;
      }
      int64_t gj = j0 + jj, gk = k0 + kk;
      sB[kk][jj] = (gj < N && gk < kend) ? (TC)B[gk * sbk + gj * sbj] : (TC)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      TC a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = sA[kk][ty + 16 * u];
        b[u] = sB[kk][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int64_t gi = i0 + ty + 16 * u;
    if (gi >= M) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int64_t gj = j0 + tx + 16 * v;
      if (gj >= N) continue;
      TC* c = C + gi + gj * ldc;
      *c = (beta == (TC)0) ? alpha * acc[u][v] : fma(alpha, acc[u][v], beta * *c);
    }
  }
}

// Double-float form of k_gemm for FP64 A, B, C: each FP64 operand is split into an FP32
// head and tail as it is staged, and the products run in compensated FP32-pair
// arithmetic (head-head product exact by FMA, the cross terms added to its error,
// TwoSum accumulation), about 2^-44 relative to sum |a_ik b_kj|, on the FP32 pipe that
// GB300 runs 64 times faster than its FP64 pipe. Same tiles, strides and split-K as
// k_gemm.
__device__ __forceinline__ void gemm_dd_mac(float& s, float& c, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float t = __fadd_rn(s, p);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

__global__ void __launch_bounds__(GTH) k_gemm_dd(int64_t M, int64_t N, int64_t K, double alpha,
                                                const double* __restrict__ A, int64_t sai, int64_t sak,
                                                const double* __restrict__ B, int64_t sbk, int64_t sbj, double beta,
                                                double* __restrict__ C, int64_t ldc, int64_t kchunk, int64_t zstride) {
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = kbeg + kchunk < K ? kbeg + kchunk : K;
  C += (int64_t)blockIdx.z * zstride;
  __shared__ float sAh[GBK][GBM + 4], sAl[GBK][GBM + 4];
  __shared__ float sBh[GBK][GBN + 4], sBl[GBK][GBN + 4];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t i0 = (int64_t)blockIdx.x * GBM, j0 = (int64_t)blockIdx.y * GBN;
  float s[4][4], c[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) s[a][b] = c[a][b] = 0.f;
  const bool a_rows_fast = (sai == 1);
  const bool b_rows_fast = (sbk == 1);
  for (int64_t k0 = kbeg; k0 < kend; k0 += GBK) {
#pragma unroll
    for (int e = 0; e < (GBM * GBK) / GTH; ++e) {
      const int idx = tid + e * GTH;
      int ii, kk;
      if (a_rows_fast) {
        ii = idx % GBM;
        kk = idx / GBM;
      } else {
        kk = idx % GBK;
        ii = idx / GBK;
      }
      const int64_t gi = i0 + ii, gk = k0 + kk;
      const double v = (gi < M && gk < kend) ? A[gi * sai + gk * sak] : 0.0;
      const float h = (float)v;
      sAh[kk][ii] = h;
      sAl[kk][ii] = (float)(v - (double)h);
    }
#pragma unroll
    for (int e = 0; e < (GBN * GBK) / GTH; ++e) {
      const int idx = tid + e * GTH;
      int jj, kk;
      if (b_rows_fast) {
        kk = idx % GBK;
        jj = idx / GBK;
      } else {
        jj = idx % GBN;
        kk = idx / GBN;
      }
      const int64_t gj = j0 + jj, gk = k0 + kk;
      const double v = (gj < N && gk < kend) ? B[gk * sbk + gj * sbj] : 0.0;
      const float h = (float)v;
      sBh[kk][jj] = h;
      sBl[kk][jj] = (float)(v - (double)h);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      float ah[4], al[4], bh[4], bl[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        ah[u] = sAh[kk][ty + 16 * u];
        al[u] = sAl[kk][ty + 16 * u];
        bh[u] = sBh[kk][tx + 16 * u];
        bl[u] = sBl[kk][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) gemm_dd_mac(s[u][v], c[u][v], ah[u], al[u], bh[v], bl[v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t gi = i0 + ty + 16 * u;
    if (gi >= M) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t gj = j0 + tx + 16 * v;
      if (gj >= N) continue;
      double* cp = C + gi + gj * ldc;
      const double val = (double)s[u][v] + (double)c[u][v];
      *cp = (beta == 0.0) ? alpha * val : fma(alpha, val, beta * *cp);
    }
  }
}

}  // namespace

namespace {

cudaError_t gemm_grid(int is_f64, int64_t M, int64_t N, int64_t K, double alpha, const void* A, int a_f64, int64_t sai,
                      int64_t sak, const void* B, int64_t sbk, int64_t sbj, double beta, void* C, int64_t ldc,
                      int64_t kchunk, int64_t zstride, int nz, cudaStream_t st) {
  dim3 grid((unsigned)((M + GBM - 1) / GBM), (unsigned)((N + GBN - 1) / GBN), (unsigned)nz);
  if (grid.y > 65535 || nz > 65535) return cudaErrorInvalidValue;
  if (is_f64) {
    if (a_f64 == 1)
      k_gemm<double, double, double><<<grid, GTH, 0, st>>>(M, N, K, alpha, (const double*)A, sai, sak,
                                                           (const double*)B, sbk, sbj, beta, (double*)C, ldc, kchunk,
                                                           zstride);
    else if (a_f64 == 0)
      k_gemm<float, double, double><<<grid, GTH, 0, st>>>(M, N, K, alpha, (const float*)A, sai, sak,
                                                          (const double*)B, sbk, sbj, beta, (double*)C, ldc, kchunk,
                                                          zstride);
    else  // a_f64 == 2: FP32 A and B, FP64 accumulation and output (exact products)
      k_gemm<float, float, double><<<grid, GTH, 0, st>>>(M, N, K, alpha, (const float*)A, sai, sak,
                                                         (const float*)B, sbk, sbj, beta, (double*)C, ldc, kchunk,
                                                         zstride);
  } else {
    if (a_f64) return cudaErrorInvalidValue;
    k_gemm<float, float, float><<<grid, GTH, 0, st>>>(M, N, K, (float)alpha, (const float*)A, sai, sak,
                                                      (const float*)B, sbk, sbj, (float)beta, (float*)C, ldc, kchunk,
                                                      zstride);
  }
  return cudaGetLastError();
}

// C (M x N, ldc) = sum_z Wz + beta C, Wz = W + z M N (M x N column-major, ld M); the
// partials are added in z order in FP64.
template <typename T>
__global__ void k_gemm_reduce(int64_t M, int64_t N, int nz, const T* __restrict__ W, double beta, T* C, int64_t ldc) {
  const int64_t total = M * N;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < nz; ++z) s += (double)W[(size_t)z * total + idx];
    T* c = C + (idx % M) + (idx / M) * ldc;
    *c = (T)(beta == 0.0 ? s : fma(beta, (double)*c, s));
  }
}

}  // namespace

cudaError_t launch_gemm(int is_f64, int64_t M, int64_t N, int64_t K, double alpha, const void* A, int a_f64,
                        int64_t sai, int64_t sak, const void* B, int64_t sbk, int64_t sbj, double beta, void* C,
                        int64_t ldc, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  return gemm_grid(is_f64, M, N, K, alpha, A, a_f64, sai, sak, B, sbk, sbj, beta, C, ldc, K, 0, 1, st);
}

int gemm_split_count(int64_t M, int64_t N, int64_t K, int sms) {
  const int64_t tiles = ((M + GBM - 1) / GBM) * ((N + GBN - 1) / GBN);
  if (tiles >= sms || K < 8 * GBK * 4) return 1;
  int64_t nz = (2LL * sms + tiles - 1) / tiles;
  nz = std::min<int64_t>(nz, K / (8 * GBK));  // at least 8 slices of K per split
  return (int)std::max<int64_t>(1, std::min<int64_t>(nz, 256));
}

cudaError_t launch_gemm_split(int is_f64, int64_t M, int64_t N, int64_t K, double alpha, const void* A, int a_f64,
                              int64_t sai, int64_t sak, const void* B, int64_t sbk, int64_t sbj, double beta, void* C,
                              int64_t ldc, void* work, size_t work_bytes, int sms, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const int nz = gemm_split_count(M, N, K, sms);
  const size_t es = is_f64 ? 8 : 4;
  if (nz <= 1 || !work || (size_t)nz * M * N * es > work_bytes)
    return gemm_grid(is_f64, M, N, K, alpha, A, a_f64, sai, sak, B, sbk, sbj, beta, C, ldc, K, 0, 1, st);
  int64_t kchunk = (K + nz - 1) / nz;
  kchunk = (kchunk + GBK - 1) / GBK * GBK;
  const int nzz = (int)((K + kchunk - 1) / kchunk);
  cudaError_t e = gemm_grid(is_f64, M, N, K, alpha, A, a_f64, sai, sak, B, sbk, sbj, 0.0, work, M, kchunk, M * N,
                            nzz, st);
  if (e != cudaSuccess) return e;
  const int rb = (int)std::min<int64_t>((M * N + 255) / 256, 4LL * sms);
  if (is_f64)
    k_gemm_reduce<double><<<rb, 256, 0, st>>>(M, N, nzz, (const double*)work, beta, (double*)C, ldc);
  else
    k_gemm_reduce<float><<<rb, 256, 0, st>>>(M, N, nzz, (const float*)work, beta, (float*)C, ldc);
  return cudaGetLastError();
}

cudaError_t launch_gemm_dd(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t sai, int64_t sak,
                           const double* B, int64_t sbk, int64_t sbj, double beta, double* C, int64_t ldc, void* work,
                           size_t work_bytes, int sms, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  int nz = gemm_split_count(M, N, K, sms);
  if (nz > 1 && (!work || (size_t)nz * M * N * 8 > work_bytes)) nz = 1;
  dim3 grid((unsigned)((M + GBM - 1) / GBM), (unsigned)((N + GBN - 1) / GBN), 1);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  if (nz <= 1) {
    k_gemm_dd<<<grid, GTH, 0, st>>>(M, N, K, alpha, A, sai, sak, B, sbk, sbj, beta, C, ldc, K, 0);
    return cudaGetLastError();
  }
  int64_t kchunk = (K + nz - 1) / nz;
  kchunk = (kchunk + GBK - 1) / GBK * GBK;
  const int nzz = (int)((K + kchunk - 1) / kchunk);
  grid.z = (unsigned)nzz;
  k_gemm_dd<<<grid, GTH, 0, st>>>(M, N, K, alpha, A, sai, sak, B, sbk, sbj, 0.0, (double*)work, M, kchunk, M * N);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int rb = (int)std::min<int64_t>((M * N + 255) / 256, 4LL * sms);
  k_gemm_reduce<double><<<rb, 256, 0, st>>>(M, N, nzz, (const double*)work, beta, C, ldc);
  return cudaGetLastError();
}

size_t gemm_split_work_bytes(int is_f64, int64_t M, int64_t N, int64_t K, int sms) {
  const int nz = gemm_split_count(M, N, K, sms);
  return nz <= 1 ? 0 : (size_t)nz * M * N * (is_f64 ? 8 : 4);
}

}  // namespace bk
