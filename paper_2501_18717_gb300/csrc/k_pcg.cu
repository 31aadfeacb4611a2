// Kernels of the Nystrom-preconditioned CG comparator (Def. PCG with the preconditioner
// of Eq. precond_def; the comparison of Thm. main), all FP64:
//   k_csr_cols   Y = A X for CSR A and a column-major block X (the block products that
//                build the Nystrom approximation, and the single-vector products of PCG)
//   k_dot_parts  per-CTA partials of a^T b
//   k_pcg_scalar reduction of the partials into the CG scalars, kept on the device so the
//                iteration needs no host round trip
//   k_pcg_xr     x += alpha p, r -= alpha (q + mu p), partials of ||r||^2
//   k_pcg_p      p = z + beta p
//   k_scale_vec  c_i *= f_i (the preconditioner's diagonal on U^T r)
//   k_gemv_t     per-CTA partials of U^T v (U d x r column-major), reduced in CTA order
//   k_gemv_n     z += U c
#include <algorithm>

#include "bk_common.cuh"

namespace bk {
namespace {

constexpr int kPcgThreads = 256;

template <typename TV>
__global__ void k_csr_cols(int64_t d, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                           const TV* __restrict__ vals, int nc, const double* __restrict__ X, int64_t ldx,
                           double* __restrict__ Y, int64_t ldy) {
  const int64_t total = d * nc;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % d;
    const int j = (int)(idx / d);
    const double* x = X + (int64_t)j * ldx;
    double s = 0.0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) s = fma((double)vals[k], x[colidx[k]], s);
    Y[i + (int64_t)j * ldy] = s;
  }
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
  __syncthreads();
  return s;  // valid in thread 0
}

__global__ void k_dot_parts(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* parts) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) parts[blockIdx.x] = s;
}

// sc: [0] rz, [1] alpha, [2] beta, [3] rr, [4] pq.
//   kind 0: pq = sum, alpha = rz / pq      kind 1: beta = sum / rz, rz = sum
//   kind 2: rz = sum                        kind 3: rr = sum
// A non-positive or non-finite pq or rz (breakdown) sets alpha = beta = 0 and sc[5] = 1.
__global__ void k_pcg_scalar(int kind, const double* __restrict__ parts, int nparts, double* sc) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) s += parts[k];
  s = block_sum(s, sh);
  if (threadIdx.x != 0) return;
  if (kind == 0) {
    sc[4] = s;
    const bool ok = s > 0.0 && isfinite(s) && isfinite(sc[0]);
    sc[1] = ok ? sc[0] / s : 0.0;
    if (!ok) sc[5] = 1.0;
  } else if (kind == 1) {
    const bool ok = sc[0] > 0.0 && isfinite(s);
    sc[2] = ok ? s / sc[0] : 0.0;
    if (!ok) sc[5] = 1.0;
    sc[0] = s;
  } else if (kind == 2) {
    sc[0] = s;
  } else {
    sc[3] = s;
  }
}

__global__ void k_pcg_xr(int64_t d, const double* __restrict__ sc, double mu, const double* __restrict__ p,
                         const double* __restrict__ q, double* x, double* r, double* parts) {
  __shared__ double sh[32];
  const double alpha = sc[1];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
    const double pi = p[i];
    x[i] = fma(alpha, pi, x[i]);
    const double ri = fma(-alpha, fma(mu, pi, q[i]), r[i]);
    r[i] = ri;
    s = fma(ri, ri, s);
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) parts[blockIdx.x] = s;
}

__global__ void k_pcg_p(int64_t d, const double* __restrict__ sc, const double* __restrict__ z, double* p) {
  const double beta = sc[2];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

__global__ void k_scale_vec(int n, const double* __restrict__ f, double* c) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) c[i] *= f[i];
}

// U^T v partials: columns in chunks of 8; each thread accumulates its rows for the 8
// columns of a chunk in registers (8 independent loads per row in flight), then the
// warp reduces them once and writes its sums to shared memory; the CTA adds its warps
// in a fixed order and writes parts[cta][j].
constexpr int kGemvCh = 8;
__global__ void k_gemv_t(int64_t d, int r, const double* __restrict__ U, int64_t ldu, const double* __restrict__ v,
                         double* parts) {
  extern __shared__ double wacc[];  // [warps][r]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int j0 = 0; j0 < r; j0 += kGemvCh) {
    double acc[kGemvCh];
#pragma unroll
    for (int u = 0; u < kGemvCh; ++u) acc[u] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += stride) {
      const double vi = v[i];
#pragma unroll
      for (int u = 0; u < kGemvCh; ++u)
        if (j0 + u < r) acc[u] = fma(U[i + (int64_t)(j0 + u) * ldu], vi, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < kGemvCh; ++u) {
      double s = acc[u];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0 && j0 + u < r) wacc[w * r + j0 + u] = s;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < nw; ++k) s += wacc[k * r + j];
    parts[(size_t)blockIdx.x * r + j] = s;
  }
}

// c[j] = sum over CTAs of parts[cta][j]: one warp per column, lanes stride over the
// CTAs, then a fixed shuffle tree (deterministic).
__global__ void k_gemv_t_reduce(int r, int nparts, const double* __restrict__ parts, double* c) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= r) return;
  double s = 0.0;
  for (int k = lane; k < nparts; k += 32) s += parts[(size_t)k * r + warp];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) c[warp] = s;
}

// z += U c: thread per row, 8 columns of loads in flight per step.
__global__ void k_gemv_n(int64_t d, int r, const double* __restrict__ U, int64_t ldu, const double* __restrict__ c,
                         double* z) {
  extern __shared__ double sc_[];
  for (int j = threadIdx.x; j < r; j += blockDim.x) sc_[j] = c[j];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
    double s = z[i];
    for (int j0 = 0; j0 < r; j0 += kGemvCh) {
      double uv[kGemvCh];
#pragma unroll
      for (int u = 0; u < kGemvCh; ++u) uv[u] = j0 + u < r ? U[i + (int64_t)(j0 + u) * ldu] : 0.0;
#pragma unroll
      for (int u = 0; u < kGemvCh; ++u)
        if (j0 + u < r) s = fma(uv[u], sc_[j0 + u], s);
    }
    z[i] = s;
  }
}

}  // namespace

int pcg_parts() { return 256; }
int gemv_parts() { return 1216; }  // 8 CTAs of 256 threads per SM on 152 SMs

cudaError_t launch_csr_cols(int vals_f64, int64_t d, const int* rowptr, const int* colidx, const void* vals, int nc,
                            const double* X, int64_t ldx, double* Y, int64_t ldy, cudaStream_t st) {
  if (d <= 0 || nc <= 0) return cudaSuccess;
  const int64_t total = d * nc;
  const int grid = (int)std::min<int64_t>((total + kPcgThreads - 1) / kPcgThreads, 1 << 16);
  if (vals_f64)
    k_csr_cols<double><<<grid, kPcgThreads, 0, st>>>(d, rowptr, colidx, (const double*)vals, nc, X, ldx, Y, ldy);
  else
    k_csr_cols<float><<<grid, kPcgThreads, 0, st>>>(d, rowptr, colidx, (const float*)vals, nc, X, ldx, Y, ldy);
  return cudaGetLastError();
}

cudaError_t launch_dot_scalar(int kind, int64_t n, const double* a, const double* b, double* parts, double* sc,
                              cudaStream_t st) {
  k_dot_parts<<<pcg_parts(), kPcgThreads, 0, st>>>(n, a, b, parts);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_pcg_scalar<<<1, kPcgThreads, 0, st>>>(kind, parts, pcg_parts(), sc);
  return cudaGetLastError();
}

cudaError_t launch_pcg_xr(int64_t d, const double* sc, double mu, const double* p, const double* q, double* x,
                          double* r, double* parts, cudaStream_t st) {
  k_pcg_xr<<<pcg_parts(), kPcgThreads, 0, st>>>(d, sc, mu, p, q, x, r, parts);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_pcg_scalar<<<1, kPcgThreads, 0, st>>>(3, parts, pcg_parts(), const_cast<double*>(sc));
  return cudaGetLastError();
}

cudaError_t launch_pcg_p(int64_t d, const double* sc, const double* z, double* p, cudaStream_t st) {
  k_pcg_p<<<pcg_parts(), kPcgThreads, 0, st>>>(d, sc, z, p);
  return cudaGetLastError();
}

cudaError_t launch_scale_vec(int n, const double* f, double* c, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_scale_vec<<<(n + 255) / 256, 256, 0, st>>>(n, f, c);
  return cudaGetLastError();
}

}  // namespace bk

namespace bk {

cudaError_t launch_gemv_t(int64_t d, int r, const double* U, int64_t ldu, const double* v, double* parts, double* c,
                          cudaStream_t st) {
  if (r <= 0) return cudaSuccess;
  const size_t smem = (size_t)(kPcgThreads / 32) * r * 8;
  if (smem > 48 * 1024) return cudaErrorInvalidValue;
  k_gemv_t<<<gemv_parts(), kPcgThreads, smem, st>>>(d, r, U, ldu, v, parts);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_gemv_t_reduce<<<(r * 32 + 255) / 256, 256, 0, st>>>(r, gemv_parts(), parts, c);
  return cudaGetLastError();
}

cudaError_t launch_gemv_n(int64_t d, int r, const double* U, int64_t ldu, const double* c, double* z,
                          cudaStream_t st) {
  if (r <= 0) return cudaSuccess;
  if ((size_t)r * 8 > 48 * 1024) return cudaErrorInvalidValue;
  const int grid = (int)std::min<int64_t>((d + kPcgThreads - 1) / kPcgThreads, 4096);
  k_gemv_n<<<grid, kPcgThreads, (size_t)r * 8, st>>>(d, r, U, ldu, c, z);
  return cudaGetLastError();
}

}  // namespace bk
