// Kernels of the one-column solvers: the Nystrom-preconditioned CG comparator (Def. PCG
// with the preconditioner of Eq. precond_def; the comparison of Thm. main) and the
// one-column phase of the shrunk block-CG. Vectors and scalars are FP64; products with
// a stored basis (U of the preconditioner, the locked basis) use its FP32 head/tail copy.
//   k_csr_cols   Y = A X for CSR A and a column-major block X (the block products that
//                build the Nystrom approximation, and the single-vector products of PCG)
//   k_dot_parts  per-CTA partials of a^T b
//   k_pcg_scalar reduction of the partials into the CG scalars, kept on the device so the
//                iteration needs no host round trip
//   k_pcg_xr     x += alpha p, r -= alpha (q + mu p), partials of ||r||^2
//   k_pcg_p      p = z + beta p
//   k_scale_vec  c_i *= f_i (the preconditioner's diagonal on U^T r)
//   k_defl_coef  the deflation coefficients of the shrunk block-CG (one-column Def-CG on
//                the locked basis): out = -(g_V + K g_Q)
//   k_defl_t     per-CTA partials of V^T r for a basis V held as FP32 head/tail arrays
//                (U or the locked basis), in compensated FP32-pair arithmetic
//   k_defl_reduce  their sum over CTAs
//   k_defl_n     z = r + V c, the same arithmetic
//   k_defl_np    p = r + V c + beta p (the shrunk solver's direction update)
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

// partials of a^T (b + mu a) (mu = 0: a^T b)
__global__ void k_dot_parts(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double mu,
                            double* parts) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ai = a[i];
    s = fma(ai, fma(mu, ai, b[i]), s);
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) parts[blockIdx.x] = s;
}

// sc: [0] rz, [1] alpha, [2] beta, [3] rr, [4] pq.
//   kind 0: pq = sum, alpha = rz / pq      kind 1: beta = sum / rz, rz = sum
//   kind 2: rz = sum                        kind 3: rr = sum
//   kind 4: as kind 1 with sum = rr (no partials: unpreconditioned CG, z = r)
// A non-positive or non-finite pq or rz (breakdown) sets alpha = beta = 0 and sc[5] = 1.
__global__ void k_pcg_scalar(int kind, const double* __restrict__ parts, int nparts, double* sc) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) s += parts[k];
  s = block_sum(s, sh);
  if (threadIdx.x != 0) return;
  if (kind == 4) {
    s = sc[3];
    kind = 1;
  }
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

// out[i] = -(g[i] + sum_q K[i + q n] g[n + q]), i < n: minus the coefficients mu_j of
// V in the deflated direction, from g = [V Q_s]^T r and K = (T_s + mu I)^{-1} E_s B_s^T
// (n x m column-major). One thread per coefficient, in a fixed order.
__global__ void k_defl_coef(int n, int m, const double* __restrict__ K, const double* __restrict__ g,
                            double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = g[i];
  for (int q = 0; q < m; ++q) s = fma(K[i + (size_t)q * n], g[n + q], s);
  out[i] = -s;
}

// ---- products with the locked basis of the shrunk block-CG. GB300 issues FP64 FMAs at
// 1/64 of the FP32 rate, so FP64 GEMVs against a d x (s + 1) m basis are FP64-pipe bound
// (d (2s + 1) m FMAs per step). With the basis split once into FP32 head and tail arrays
// (a = ah + al, |al| <= 2^-24 |a|), every multiply-add takes 12 FP32 operations: the
// exact product of the heads by fma (Dekker), the two cross terms, and a TwoSum (Knuth)
// into an (s, c) accumulator. The sum carries about 2^-44 of sum |a_i b_i|; the basis
// reads then bound the kernels by HBM.
__device__ __forceinline__ void pair_mac(float ah, float al, float bh, float bl, float& s, float& c) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float t = __fadd_rn(s, p);
  const float bp = __fadd_rn(t, -s);
  const float err = __fadd_rn(__fadd_rn(s, -__fadd_rn(t, -bp)), __fadd_rn(p, -bp));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

// parts[j * nparts + cta] = sum over the CTA's kDtRows rows of V(i, j) r_i: the CTA
// stages its slice of r (split into head and tail) in shared memory, each warp takes
// columns j = warp, warp + 8, .. and its lanes stride over the rows, so one warp reads
// 4 KB runs of each array.
constexpr int kDtRows = 1024;
__global__ void __launch_bounds__(256) k_defl_t(int64_t d, int nc, const float* __restrict__ Vh,
                                                const float* __restrict__ Vl, int64_t ldv,
                                                const double* __restrict__ r, int nparts, double* __restrict__ parts) {
  __shared__ float rh[kDtRows], rl[kDtRows];
  const int64_t row0 = (int64_t)blockIdx.x * kDtRows;
  const int rows = (int)(d - row0 < kDtRows ? d - row0 : kDtRows);
  for (int k = threadIdx.x; k < kDtRows; k += blockDim.x) {
    const double v = k < rows ? r[row0 + k] : 0.0;
    const float h = __double2float_rn(v);
    rh[k] = h;
    rl[k] = __double2float_rn(v - (double)h);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = w; j < nc; j += nw) {
    const float* ch = Vh + (size_t)j * ldv + row0;
    const float* cl = Vl + (size_t)j * ldv + row0;
    float s = 0.f, c = 0.f;
    if (rows == kDtRows) {
#pragma unroll 4
      for (int k = lane; k < kDtRows; k += 32) pair_mac(ch[k], cl[k], rh[k], rl[k], s, c);
    } else {
      for (int k = lane; k < rows; k += 32) pair_mac(ch[k], cl[k], rh[k], rl[k], s, c);
    }
    double t = (double)s + (double)c;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) parts[(size_t)j * nparts + blockIdx.x] = t;
  }
}

// g[j] = sum over CTAs of parts[j * nparts + cta]: one warp per column, a fixed order.
__global__ void k_defl_reduce(int nc, int nparts, const double* __restrict__ parts, double* __restrict__ g) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nc) return;
  const double* p = parts + (size_t)warp * nparts;
  double s = 0.0;
  for (int k = lane; k < nparts; k += 32) s += p[k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) g[warp] = s;
}

// z = r + V c over nc columns, thread per row; r and z may be the same array.
__global__ void __launch_bounds__(256) k_defl_n(int64_t d, int nc, const float* __restrict__ Vh,
                                                const float* __restrict__ Vl, int64_t ldv,
                                                const double* __restrict__ coef, const double* r, double* z) {
  extern __shared__ float cs[];  // head [nc], tail [nc]
  for (int j = threadIdx.x; j < nc; j += blockDim.x) {
    const double v = coef[j];
    const float h = __double2float_rn(v);
    cs[j] = h;
    cs[nc + j] = __double2float_rn(v - (double)h);
  }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
    const float* ph = Vh + i;
    const float* pl = Vl + i;
    float s = 0.f, c = 0.f;
#pragma unroll 4
    for (int j = 0; j < nc; ++j) pair_mac(ph[(size_t)j * ldv], pl[(size_t)j * ldv], cs[j], cs[nc + j], s, c);
    z[i] = r[i] + ((double)s + (double)c);
  }
}

// p = r + V c + beta p (beta = sc[2]): the deflated direction of the shrunk block-CG in
// one pass, with V c in the arithmetic of k_defl_n.
__global__ void __launch_bounds__(256) k_defl_np(int64_t d, int nc, const float* __restrict__ Vh,
                                                 const float* __restrict__ Vl, int64_t ldv,
                                                 const double* __restrict__ coef, const double* __restrict__ sc,
                                                 const double* __restrict__ r, double* __restrict__ p) {
  extern __shared__ float cs[];  // head [nc], tail [nc]
  for (int j = threadIdx.x; j < nc; j += blockDim.x) {
    const double v = coef[j];
    const float h = __double2float_rn(v);
    cs[j] = h;
    cs[nc + j] = __double2float_rn(v - (double)h);
  }
  __syncthreads();
  const double beta = sc[2];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
    const float* ph = Vh + i;
    const float* pl = Vl + i;
    float s = 0.f, c = 0.f;
#pragma unroll 4
    for (int j = 0; j < nc; ++j) pair_mac(ph[(size_t)j * ldv], pl[(size_t)j * ldv], cs[j], cs[nc + j], s, c);
    p[i] = fma(beta, p[i], r[i] + ((double)s + (double)c));
  }
}

}  // namespace

int pcg_parts() { return 1216; }  // 8 CTAs of 256 threads per SM on 152 SMs

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
  return launch_dot_shift_scalar(kind, n, a, b, 0.0, parts, sc, st);
}

cudaError_t launch_dot_shift_scalar(int kind, int64_t n, const double* a, const double* b, double mu, double* parts,
                                    double* sc, cudaStream_t st) {
  if (kind == 4) {
    k_pcg_scalar<<<1, kPcgThreads, 0, st>>>(4, parts, 0, sc);
    return cudaGetLastError();
  }
  k_dot_parts<<<pcg_parts(), kPcgThreads, 0, st>>>(n, a, b, mu, parts);
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

}  // namespace bk

namespace bk {

cudaError_t launch_defl_coef(int n, int m, const double* K, const double* g, double* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_defl_coef<<<(n + 127) / 128, 128, 0, st>>>(n, m, K, g, out);
  return cudaGetLastError();
}

int defl_parts(int64_t d) { return (int)((d + kDtRows - 1) / kDtRows); }

cudaError_t launch_defl_t(int64_t d, int nc, const float* Vh, const float* Vl, int64_t ldv, const double* r,
                          double* parts, double* g, cudaStream_t st) {
  if (nc <= 0 || d <= 0) return cudaSuccess;
  const int np = defl_parts(d);
  k_defl_t<<<np, 256, 0, st>>>(d, nc, Vh, Vl, ldv, r, np, parts);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_defl_reduce<<<(nc * 32 + 255) / 256, 256, 0, st>>>(nc, np, parts, g);
  return cudaGetLastError();
}

cudaError_t launch_defl_np(int64_t d, int nc, const float* Vh, const float* Vl, int64_t ldv, const double* coef,
                           const double* sc, const double* r, double* p, int sms, cudaStream_t st) {
  if (d <= 0) return cudaSuccess;
  if ((size_t)nc * 8 > 48 * 1024) return cudaErrorInvalidValue;
  const int grid = (int)std::min<int64_t>((d + 255) / 256, (int64_t)sms * 8);
  k_defl_np<<<grid, 256, (size_t)nc * 8, st>>>(d, nc, Vh, Vl, ldv, coef, sc, r, p);
  return cudaGetLastError();
}

cudaError_t launch_defl_n(int64_t d, int nc, const float* Vh, const float* Vl, int64_t ldv, const double* coef,
                          const double* r, double* z, int sms, cudaStream_t st) {
  if (d <= 0) return cudaSuccess;
  if ((size_t)nc * 8 > 48 * 1024) return cudaErrorInvalidValue;
  const int grid = (int)std::min<int64_t>((d + 255) / 256, (int64_t)sms * 8);
  k_defl_n<<<grid, 256, (size_t)nc * 8, st>>>(d, nc, Vh, Vl, ldv, coef, r, z);
  return cudaGetLastError();
}

}  // namespace bk
