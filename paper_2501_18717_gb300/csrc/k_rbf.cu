// Matrix-free RBF kernel operator (the access mode of Sec. 1 where only products with
// A are available): Y = K X with K_ij = exp(-||x_i - x_j||^2 / (2 l^2)) formed on the
// fly, never stored, for the sampling driver (Sec. 5, Def. blansq).
//
// Each K entry exp(t), t = -||x_i - x_j||^2 / (2 l^2) formed in FP64, is evaluated in
// double-float arithmetic (pairs of FP32): Cody-Waite reduction t = k ln2 + r in FP64,
// |r| <= ln2 / 2, then the Taylor polynomial of exp(r) to degree 14 by Horner's rule in
// pair arithmetic (Dekker's product and Knuth's sum, error-free by FMA), scaled by 2^k;
// relative error about 2^-46 (for t >= -70), and the entry comes out as the head and tail the products
// need; for t < -70 the tail falls below the FP32 normal range, so there the error is
// absolute, under 2^-126, and exp(t) for t < -100 is taken as 0. X (FP64) is split into head and tail; the products use compensated FP32-pair
// arithmetic (the head-head product made exact by FMA, the two cross terms added to its
// error, TwoSum accumulation), about 2^-44 relative to sum |K_ik x_k|. The entries are
// therefore accurate to about 1e-14, far below the nugget, unlike an FP32-stored K
// whose rounding is a perturbation of norm ~3e-6 at 40,000 points.
//
// Tile: 128 threads as 4 row groups x 32 column groups, three CTAs per SM; 16 rows x
// 256 columns per CTA (4 rows x 8 columns per thread), so each exp serves all columns
// of a block of up to 256. Smaller CTAs measured faster (one CTA of 384 threads per
// SM: 249 ms per 40,000-point load; two of 192: 216 ms; three of 128: 204 ms), since
// the slice barriers of one CTA no longer stall the whole SM. The K slice (16 rows x
// 16 points) is generated into shared memory per stage; the X slice (16 rows x 256
// columns) comes in as FP32 head and tail.
#include <algorithm>

#include "bk_common.cuh"

namespace bk {
namespace {

constexpr int RB_TH = 128, RB_RG = 4, RB_BM = 4 * RB_RG, RB_BN = 256, RB_BK = 16, RB_NPT = 8;
constexpr int RB_LDK = RB_BM + 4, RB_LDX = RB_BN + 4;
static_assert((RB_BM * RB_BK) % RB_TH == 0, "whole K-slice entries per thread");

__device__ __forceinline__ void dd_mac(float& s, float& c, float ah, float al, float bh, float bl) {
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

// ---- double-float (FP32 pair) arithmetic; the _rn intrinsics keep the compiler from
// contracting the error-free transformations into FMAs
__device__ __forceinline__ void df_fast_two_sum(float a, float b, float& s, float& e) {  // |a| >= |b|
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& ph, float& pl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  df_fast_two_sum(p, e, ph, pl);
}
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& sh, float& sl) {
  const float s = __fadd_rn(ah, bh);
  const float bb = __fsub_rn(s, ah);
  float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
  e = __fadd_rn(e, __fadd_rn(al, bl));
  df_fast_two_sum(s, e, sh, sl);
}

// Taylor coefficients 1 / k!, k = 0..14, as FP32 head and tail
struct ExpCoef {
  float h[15], l[15];
};
constexpr ExpCoef make_exp_coef() {
  ExpCoef c{};
  double f = 1.0;
  for (int k = 0; k < 15; ++k) {
    if (k > 0) f /= (double)k;
    c.h[k] = (float)f;
    c.l[k] = (float)(f - (double)c.h[k]);
  }
  return c;
}
__constant__ ExpCoef kExpCoef = make_exp_coef();

// exp(t) for t <= 0 as a pair (h, l) of FP32 (0 below exp(-100)).
__device__ __forceinline__ void exp_df(double t, float& h, float& l) {
  if (t < -100.0) {
    h = l = 0.f;
    return;
  }
  // ln 2 split into a head of 32 significant bits (k * head is exact for |k| < 2^21)
  // and the rest of its double value; the double's own rounding (1e-16 relative) moves
  // r by at most |k| 1e-16, below the pair arithmetic's 2^-46
  constexpr double kLn2 = 0.69314718055994530942;
  constexpr double kLn2Hi = (double)(long long)(kLn2 * 4294967296.0) / 4294967296.0;
  constexpr double kLn2Lo = kLn2 - kLn2Hi;
  const double kd = rint(t * (1.0 / kLn2));
  double r = fma(-kd, kLn2Hi, t);
  r = fma(-kd, kLn2Lo, r);
  const float rh = (float)r, rl = (float)(r - (double)rh);
  float ph = kExpCoef.h[14], pl = kExpCoef.l[14];
#pragma unroll
  for (int k = 13; k >= 0; --k) {
    float mh, ml;
    df_mul(ph, pl, rh, rl, mh, ml);
    df_add(mh, ml, kExpCoef.h[k], kExpCoef.l[k], ph, pl);
  }
  const int ki = (int)kd;
  h = ldexpf(ph, ki);
  l = ldexpf(pl, ki);
}


// X: the FP32 head and tail (d x N column-major, ldx a multiple of 4, rows d..ldx-1
// zero) of the FP64 block; Y: d x N column-major (ldy) FP64; pts: d points of 3
// coordinates, row stride ldp (FP64). h = 1 / (2 l^2). The slices are double buffered: each thread
// builds its part of slice s + 1 (FP64 exp, FP64 splits) and then runs its products on
// slice s, with one barrier per slice, so the FP64 work of some warps overlaps the FP32
// multiply-adds of others.
__global__ void __launch_bounds__(RB_TH, 3) k_rbf_apply(int64_t d, int N, const double* __restrict__ pts,
                                                        int64_t ldp, double h, const float* __restrict__ Xh,
                                                        const float* __restrict__ Xl, int64_t ldx,
                                                        double* __restrict__ Y, int64_t ldy) {
  extern __shared__ __align__(16) float sm[];
  constexpr int KS = RB_BK * RB_LDK, XS = RB_BK * RB_LDX, STAGE = 2 * KS + 2 * XS;
  double* sP = reinterpret_cast<double*>(sm + 2 * STAGE);  // this CTA's row points
  const int tid = threadIdx.x, rg = tid >> 5, cg = tid & 31;  // rg < RB_RG
  const int64_t i0 = (int64_t)blockIdx.x * RB_BM;
  const int j0 = blockIdx.y * RB_BN;
  for (int q = tid; q < RB_BM * 3; q += RB_TH) {
    const int r = q / 3, c = q % 3;
    sP[q] = (i0 + r < d) ? pts[(i0 + r) * ldp + c] : 0.0;
  }
  float s[4][RB_NPT], cc[4][RB_NPT];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < RB_NPT; ++v) s[u][v] = cc[u][v] = 0.f;
  __syncthreads();

  auto build = [&](int64_t k0, int buf) {
    float* sKh = sm + buf * STAGE;
    float* sKl = sKh + KS;
    float* sXh = sKl + KS;
    float* sXl = sXh + XS;
    // K slice: RB_BM rows x 16 points
#pragma unroll
    for (int e = 0; e < (RB_BM * RB_BK) / RB_TH; ++e) {
      const int q = tid + e * RB_TH;
      const int r = q % RB_BM, kk = q / RB_BM;
      const int64_t gk = k0 + kk;
      float kh = 0.f, kl = 0.f;
      if (i0 + r < d && gk < d) {
        const double dx = sP[r * 3] - pts[gk * ldp];
        const double dy = sP[r * 3 + 1] - pts[gk * ldp + 1];
        const double dz = sP[r * 3 + 2] - pts[gk * ldp + 2];
        exp_df(-h * fma(dx, dx, fma(dy, dy, dz * dz)), kh, kl);
      }
      sKh[kk * RB_LDK + r] = kh;
      sKl[kk * RB_LDK + r] = kl;
    }
    // X slice: 16 rows x 256 columns, 16-byte loads of 4 consecutive rows of a column
    for (int q = tid; q < (RB_BK / 4) * RB_BN; q += RB_TH) {
      const int c4 = q & 3, j = q >> 2;
      const int64_t gk = k0 + 4 * c4;
      float4 h4 = make_float4(0.f, 0.f, 0.f, 0.f), l4 = h4;
      if (gk < ldx && j0 + j < N) {
        h4 = *reinterpret_cast<const float4*>(Xh + (int64_t)(j0 + j) * ldx + gk);
        l4 = *reinterpret_cast<const float4*>(Xl + (int64_t)(j0 + j) * ldx + gk);
      }
      const int kk = 4 * c4;
      sXh[(kk + 0) * RB_LDX + j] = h4.x;
      sXh[(kk + 1) * RB_LDX + j] = h4.y;
      sXh[(kk + 2) * RB_LDX + j] = h4.z;
      sXh[(kk + 3) * RB_LDX + j] = h4.w;
      sXl[(kk + 0) * RB_LDX + j] = l4.x;
      sXl[(kk + 1) * RB_LDX + j] = l4.y;
      sXl[(kk + 2) * RB_LDX + j] = l4.z;
      sXl[(kk + 3) * RB_LDX + j] = l4.w;
    }
  };

  const int64_t nst = (d + RB_BK - 1) / RB_BK;
  build(0, 0);
  __syncthreads();
  for (int64_t st = 0; st < nst; ++st) {
    const int buf = (int)(st & 1);
    if (st + 1 < nst) build((st + 1) * RB_BK, buf ^ 1);
    const float* sKh = sm + buf * STAGE;
    const float* sKl = sKh + KS;
    const float* sXh = sKl + KS;
    const float* sXl = sXh + XS;
#pragma unroll 2
    for (int kk = 0; kk < RB_BK; ++kk) {
      float ah[4], al[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        ah[u] = sKh[kk * RB_LDK + rg + RB_RG * u];
        al[u] = sKl[kk * RB_LDK + rg + RB_RG * u];
      }
#pragma unroll
      for (int v = 0; v < RB_NPT; ++v) {
        const float bh = sXh[kk * RB_LDX + cg + 32 * v];
        const float bl = sXl[kk * RB_LDX + cg + 32 * v];
#pragma unroll
        for (int u = 0; u < 4; ++u) dd_mac(s[u][v], cc[u][v], ah[u], al[u], bh, bl);
      }
    }
    __syncthreads();  // slice st + 1 complete; slice st free for st + 2
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t i = i0 + rg + RB_RG * u;
    if (i >= d) continue;
#pragma unroll
    for (int v = 0; v < RB_NPT; ++v) {
      const int j = j0 + cg + 32 * v;
      if (j < N) Y[(int64_t)j * ldy + i] = (double)s[u][v] + (double)cc[u][v];
    }
  }
}

constexpr size_t rbf_smem() {
  return (size_t)2 * (2 * RB_BK * RB_LDK + 2 * RB_BK * RB_LDX) * 4 + (size_t)RB_BM * 3 * 8;
}

}  // namespace

cudaError_t launch_rbf_apply(int64_t d, int N, const double* pts, int64_t ldp, double lengthscale, const float* Xh,
                             const float* Xl, int64_t ldx, double* Y, int64_t ldy, cudaStream_t st) {
  if (d <= 0 || N <= 0) return cudaSuccess;
  if (!(lengthscale > 0.0) || ldp < 3 || (ldx & 3) || ldx < d || ((uintptr_t)Xh & 15) || ((uintptr_t)Xl & 15))
    return cudaErrorInvalidValue;
  const size_t smem = rbf_smem();
  cudaError_t e = cudaFuncSetAttribute(k_rbf_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t mt = (d + RB_BM - 1) / RB_BM;
  const int nt = (N + RB_BN - 1) / RB_BN;
  if (mt > 0x7fffffff || nt > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)mt, (unsigned)nt);
  k_rbf_apply<<<grid, RB_TH, smem, st>>>(d, N, pts, ldp, 1.0 / (2.0 * lengthscale * lengthscale), Xh, Xl, ldx, Y,
                                         ldy);
  return cudaGetLastError();
}

}  // namespace bk
