// Tall-skinny block products of the block-Lanczos drivers (Sec. 3.2; Thm. cost counts
// one matrix-load per block product). For the ridge path A = Z^T Z is applied
// matrix-free as two passes over the stored Z (Sec. 1, the ridge problem): T = Z P,
// then Y = Z^T T. The same row-tiled product serves a dense operator with a block of
// up to a few hundred columns (the sampling driver, Def. blansq).
//
//   nn:  C (M x N, column-major, ldc) = alpha A B + beta C
//        A (M x K, row-major, lda, FP32), B (K x N, column-major, ldb)
//   tn:  Y (D x N, column-major, ldy) = alpha Z^T T + beta Y
//        Z (R x D, row-major, ldz, FP32), T (R x N, column-major, ldt); the rows are
//        split into chunks whose partial sums are reduced in a fixed order.
//
// Two arithmetic modes share the tiles:
//   FP32  B / T in FP32, FFMA accumulation, FP32 output (the Lanczos basis products).
//   DF    B / T in FP64, split once per product into FP32 head and tail arrays
//         (launch_split_f64) that the kernels stage like FP32 operands; every product of
//         the FP32 matrix
//         entry with the head is made exact with an FMA (its rounding error is
//         representable) and added to a compensated FP32 pair (Knuth's TwoSum), so the
//         sums carry about 44 significant bits. This is the FP64-accurate operator of
//         the refinement residuals (the stored values promoted to FP64) on the FP32
//         pipe, which GB300 runs about 64 times faster than its FP64 pipe.
//
// Tiles: 128 threads as 16 row groups x 8 column groups. FP32 mode: 8 rows x NPT
// columns per thread (128-row tiles); DF mode: 4 rows x NPT columns (64-row tiles).
// Operands are staged in shared memory in 32-deep slices, double buffered with
// cp.async (16-byte copies that zero-fill past the matrix edges).
#include <algorithm>

#include "bk_common.cuh"

namespace bk {
namespace {

constexpr int TS_TH = 128;
constexpr int TS_BK = 32;   // depth of one staged slice
constexpr int TS_LDK = 36;  // padded row length of a slice (floats): conflict-free 16-byte reads

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 16-byte asynchronous copy; bytes beyond src_bytes (0..16) are zero-filled.
__device__ __forceinline__ void cp16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__device__ __forceinline__ int clamp16(int64_t bytes) { return bytes <= 0 ? 0 : (bytes >= 16 ? 16 : (int)bytes); }

// s + c += a * (bh + bl): exact product error by FMA, TwoSum of the running sum with
// the rounded product, and both error terms into c. The _rn intrinsics keep the
// compiler from contracting the additions into FMAs, which would break TwoSum.
__device__ __forceinline__ void df_mac(float& s, float& c, float a, float bh, float bl) {
  const float p = __fmul_rn(a, bh);
  float e = fmaf(a, bh, -p);
  e = fmaf(a, bl, e);
  const float t = __fadd_rn(s, p);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

__device__ __forceinline__ void split_f64(double v, float& h, float& l) {
  h = (float)v;
  l = (float)(v - (double)h);
}

template <bool DF>
struct TsCfg {
  static constexpr int RPT = DF ? 4 : 8;  // rows (nn) or Z columns (tn) per thread
  static constexpr int BM = 16 * RPT;
};

// ---------------------------------------------------------------- nn: C = alpha A B + beta C
// Shared memory per stage: sA[BM][TS_LDK] floats, then sB (FP32: [NT][TS_LDK]; DF: head
// and tail, 2 x [NT][TS_LDK]).
template <int NPT, bool DF>
__global__ void __launch_bounds__(TS_TH, 3) k_tsm_nn(int64_t M, int N, int64_t K, double alpha, const float* __restrict__ A,
                                                  int64_t lda, const float* __restrict__ Bh, const float* __restrict__ Bl,
                                                  int64_t ldb, double beta, void* Cv, int64_t ldc) {
  using Cfg = TsCfg<DF>;
  constexpr int RPT = Cfg::RPT, BM = Cfg::BM, NT = 8 * NPT;
  constexpr int A_FL = BM * TS_LDK, B_FL = (DF ? 2 : 1) * NT * TS_LDK, ST_FL = A_FL + B_FL;
  extern __shared__ __align__(16) float smem[];
  const int tid = threadIdx.x, tr = tid >> 3 & 15, tc = tid & 7;
  // thread layout: lanes 0..7 are the column groups, lanes /8 the row groups; rows of a
  // thread are tr + 16 u, columns tc + 8 v
  const int64_t i0 = (int64_t)blockIdx.y * BM;
  const int j0 = blockIdx.x * NT;
  const int nst = (int)((K + TS_BK - 1) / TS_BK);

  // Staging geometry is fixed per thread: chunk column c4 = tid % 8 (16 bytes of a
  // 32-deep slice) and rows (or columns of B) r0 + 16 e; only the slice offset moves.
  const int c4 = tid & 7, r0 = tid >> 3;
  constexpr int EA = BM / 16, EB = (NT * 8 + TS_TH - 1) / TS_TH;
  const float* a_row = A + (i0 + r0) * lda + c4 * 4;
  const int64_t a_step = 16 * lda;
  unsigned a_ok = 0, b_ok = 0;
#pragma unroll
  for (int e = 0; e < EA; ++e)
    if (i0 + r0 + 16 * e < M) a_ok |= 1u << e;
#pragma unroll
  for (int e = 0; e < EB; ++e)
    if (r0 + 16 * e < NT && j0 + r0 + 16 * e < N) b_ok |= 1u << e;
  auto issue_a = [&](int s, int buf) {
    float* sA = smem + buf * ST_FL + r0 * TS_LDK + c4 * 4;
    const int64_t k = (int64_t)s * TS_BK + c4 * 4;
    const int bytes = clamp16((K - k) * 4);
    const float* src = a_row + (int64_t)s * TS_BK;
#pragma unroll 1
    for (int e = 0; e < EA; ++e, src += a_step) {
      const bool ok = (a_ok >> e & 1u) && bytes;
      cp16(sA + 16 * e * TS_LDK, ok ? src : A, ok ? bytes : 0);
    }
  };
  // B (FP32), or the FP32 head and tail of an FP64 B (DF), into the stage's B area
  auto issue_b32 = [&](int s, int buf) {
    float* sB = smem + buf * ST_FL + A_FL + r0 * TS_LDK + c4 * 4;
    const int64_t k = (int64_t)s * TS_BK + c4 * 4;
    const int bytes = clamp16((K - k) * 4);
#pragma unroll 1
    for (int e = 0; e < EB; ++e) {
      if (r0 + 16 * e >= NT) break;
      const bool ok = (b_ok >> e & 1u) && bytes;
      const int64_t off = (int64_t)(j0 + r0 + 16 * e) * ldb + k;
      cp16(sB + 16 * e * TS_LDK, ok ? Bh + off : Bh, ok ? bytes : 0);
      if constexpr (DF) cp16(sB + NT * TS_LDK + 16 * e * TS_LDK, ok ? Bl + off : Bl, ok ? bytes : 0);
    }
  };

  float acc[RPT][NPT], cmp[DF ? RPT : 1][DF ? NPT : 1];
#pragma unroll
  for (int u = 0; u < RPT; ++u)
#pragma unroll
    for (int v = 0; v < NPT; ++v) {
      acc[u][v] = 0.f;
      if constexpr (DF) cmp[u][v] = 0.f;
    }

  if (nst > 0) {
    issue_a(0, 0);
    issue_b32(0, 0);
    cp_commit();
  }
  for (int s = 0; s < nst; ++s) {
    const int buf = s & 1;
    if (s + 1 < nst) {
      issue_a(s + 1, buf ^ 1);
      issue_b32(s + 1, buf ^ 1);
      cp_commit();
      cp_wait_one();
    } else {
      cp_wait_all();
    }
    __syncthreads();
    const float* sA = smem + buf * ST_FL;
    const float* sB = sA + A_FL;
#pragma unroll 2
    for (int k4 = 0; k4 < TS_BK; k4 += 4) {
      float4 a[RPT];
#pragma unroll
      for (int u = 0; u < RPT; ++u) a[u] = *(const float4*)(sA + (tr + 16 * u) * TS_LDK + k4);
      if constexpr (!DF) {
#pragma unroll
        for (int v = 0; v < NPT; ++v) {
          const float4 b = *(const float4*)(sB + (tc + 8 * v) * TS_LDK + k4);
#pragma unroll
          for (int u = 0; u < RPT; ++u) {
            acc[u][v] = fmaf(a[u].x, b.x, acc[u][v]);
            acc[u][v] = fmaf(a[u].y, b.y, acc[u][v]);
            acc[u][v] = fmaf(a[u].z, b.z, acc[u][v]);
            acc[u][v] = fmaf(a[u].w, b.w, acc[u][v]);
          }
        }
      } else {
        const float* sBl = sB + NT * TS_LDK;
#pragma unroll
        for (int v = 0; v < NPT; ++v) {
          const float4 bh = *(const float4*)(sB + (tc + 8 * v) * TS_LDK + k4);
          const float4 bl = *(const float4*)(sBl + (tc + 8 * v) * TS_LDK + k4);
#pragma unroll
          for (int u = 0; u < RPT; ++u) {
            df_mac(acc[u][v], cmp[u][v], a[u].x, bh.x, bl.x);
            df_mac(acc[u][v], cmp[u][v], a[u].y, bh.y, bl.y);
            df_mac(acc[u][v], cmp[u][v], a[u].z, bh.z, bl.z);
            df_mac(acc[u][v], cmp[u][v], a[u].w, bh.w, bl.w);
          }
        }
      }
    }
    __syncthreads();
  }

  // epilogue through shared memory: consecutive threads write consecutive rows
  if constexpr (!DF) {
    float* sC = smem;  // [NT][BM + 4]
#pragma unroll
    for (int u = 0; u < RPT; ++u)
#pragma unroll
      for (int v = 0; v < NPT; ++v) sC[(tc + 8 * v) * (BM + 4) + tr + 16 * u] = acc[u][v];
    __syncthreads();
    float* C = (float*)Cv;
    for (int q = tid; q < NT * BM; q += TS_TH) {
      const int j = q / BM, row = q % BM;
      const int64_t gi = i0 + row;
      if (gi >= M || j0 + j >= N) continue;
      float* c = C + gi + (int64_t)(j0 + j) * ldc;
      const float val = (float)alpha * sC[j * (BM + 4) + row];
      *c = beta == 0.0 ? val : fmaf((float)beta, *c, val);
    }
  } else {
    double* sC = (double*)smem;  // [NT][BM + 2]
#pragma unroll
    for (int u = 0; u < RPT; ++u)
#pragma unroll
      for (int v = 0; v < NPT; ++v)
        sC[(tc + 8 * v) * (BM + 2) + tr + 16 * u] = (double)acc[u][v] + (double)cmp[u][v];
    __syncthreads();
    double* C = (double*)Cv;
    for (int q = tid; q < NT * BM; q += TS_TH) {
      const int j = q / BM, row = q % BM;
      const int64_t gi = i0 + row;
      if (gi >= M || j0 + j >= N) continue;
      double* c = C + gi + (int64_t)(j0 + j) * ldc;
      const double val = alpha * sC[j * (BM + 2) + row];
      *c = beta == 0.0 ? val : fma(beta, *c, val);
    }
  }
}

// ---------------------------------------------------------------- tn: partials of Z^T T
// CTA (x: Z-column tile of BD = 16 RPT, y: row chunk, z: column tile of T) writes
// W[y][j][k] (FP32 mode: float; DF: double), j < NT of its tile, k < BD of its tile,
// row stride ldw. Thread: Z columns tk RPT .. tk RPT + RPT - 1 (contiguous), T columns
// tc + 8 v. Shared memory per stage: sZ[TS_BK][BD + 4], sT (FP32: [NT][TS_LDK]; DF:
// head and tail).
template <int NPT, bool DF>
__global__ void __launch_bounds__(TS_TH, 3) k_tsm_tn(int64_t R, int64_t D, int N, int64_t rows_per_chunk,
                                                  const float* __restrict__ Z, int64_t ldz, const float* __restrict__ Th,
                                                  const float* __restrict__ Tl, int64_t ldt, void* Wv, int64_t ldw) {
  using Cfg = TsCfg<DF>;
  constexpr int RPT = Cfg::RPT, BD = Cfg::BM, NT = 8 * NPT, LDZ = BD + 4;
  constexpr int Z_FL = TS_BK * LDZ, T_FL = (DF ? 2 : 1) * NT * TS_LDK, ST_FL = Z_FL + T_FL;
  extern __shared__ __align__(16) float smem[];
  const int tid = threadIdx.x, tk = tid >> 3 & 15, tc = tid & 7;
  const int64_t d0 = (int64_t)blockIdx.x * BD;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r1 = r0 + rows_per_chunk < R ? r0 + rows_per_chunk : R;
  const int j0 = blockIdx.z * NT;
  const int nst = r1 > r0 ? (int)((r1 - r0 + TS_BK - 1) / TS_BK) : 0;

  // fixed staging geometry: Z chunks (column c4z = tid % (BD/4), rows rz + (128 / (BD/4)) e),
  // T chunks (column c4 = tid % 8 of the slice, T columns rt + 16 e)
  constexpr int ZC = BD / 4, ZR = TS_TH / ZC, EZ = TS_BK / ZR, ET = (NT * 8 + TS_TH - 1) / TS_TH;
  const int c4z = tid % ZC, rz = tid / ZC, c4 = tid & 7, rt = tid >> 3;
  const int64_t gkz = d0 + c4z * 4;
  const int zbytes = clamp16((D - gkz) * 4);
  const float* z_col = Z + gkz;
  auto issue_z = [&](int s, int buf) {
    float* sZ = smem + buf * ST_FL + rz * LDZ + c4z * 4;
    const int64_t i0 = r0 + (int64_t)s * TS_BK + rz;
#pragma unroll
    for (int e = 0; e < EZ; ++e) {
      const int64_t gi = i0 + ZR * e;
      const bool ok = gi < r1 && zbytes;
      cp16(sZ + ZR * e * LDZ, ok ? z_col + gi * ldz : Z, ok ? zbytes : 0);
    }
  };
  // T (FP32), or the FP32 head and tail of an FP64 T (DF), into the stage's T area
  auto issue_t32 = [&](int s, int buf) {
    float* sT = smem + buf * ST_FL + Z_FL + rt * TS_LDK + c4 * 4;
    const int64_t gi = r0 + (int64_t)s * TS_BK + c4 * 4;
    const int bytes = clamp16((r1 - gi) * 4);
#pragma unroll
    for (int e = 0; e < ET; ++e) {
      const int j = rt + 16 * e;
      if (j >= NT) break;
      const bool ok = (j0 + j) < N && bytes;
      const int64_t off = (int64_t)(j0 + j) * ldt + gi;
      cp16(sT + 16 * e * TS_LDK, ok ? Th + off : Th, ok ? bytes : 0);
      if constexpr (DF) cp16(sT + NT * TS_LDK + 16 * e * TS_LDK, ok ? Tl + off : Tl, ok ? bytes : 0);
    }
  };

  float acc[RPT][NPT], cmp[DF ? RPT : 1][DF ? NPT : 1];
#pragma unroll
  for (int u = 0; u < RPT; ++u)
#pragma unroll
    for (int v = 0; v < NPT; ++v) {
      acc[u][v] = 0.f;
      if constexpr (DF) cmp[u][v] = 0.f;
    }

  if (nst > 0) {
    issue_z(0, 0);
    issue_t32(0, 0);
    cp_commit();
  }
  for (int s = 0; s < nst; ++s) {
    const int buf = s & 1;
    if (s + 1 < nst) {
      issue_z(s + 1, buf ^ 1);
      issue_t32(s + 1, buf ^ 1);
      cp_commit();
      cp_wait_one();
    } else {
      cp_wait_all();
    }
    __syncthreads();
    const float* sZ = smem + buf * ST_FL;
    const float* sT = sZ + Z_FL;
#pragma unroll 2
    for (int i4 = 0; i4 < TS_BK; i4 += 4) {
      if constexpr (!DF) {
        float4 t[NPT];
#pragma unroll
        for (int v = 0; v < NPT; ++v) t[v] = *(const float4*)(sT + (tc + 8 * v) * TS_LDK + i4);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float4 z0 = *(const float4*)(sZ + (i4 + r) * LDZ + tk * RPT);
          const float4 z1 = *(const float4*)(sZ + (i4 + r) * LDZ + tk * RPT + 4);
          const float zz[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
#pragma unroll
          for (int v = 0; v < NPT; ++v) {
            const float tv = r == 0 ? t[v].x : r == 1 ? t[v].y : r == 2 ? t[v].z : t[v].w;
#pragma unroll
            for (int u = 0; u < RPT; ++u) acc[u][v] = fmaf(zz[u], tv, acc[u][v]);
          }
        }
      } else {
        const float* sTl = sT + NT * TS_LDK;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float4 z0 = *(const float4*)(sZ + (i4 + r) * LDZ + tk * RPT);
          const float zz[4] = {z0.x, z0.y, z0.z, z0.w};
#pragma unroll
          for (int v = 0; v < NPT; ++v) {
            const float th = sT[(tc + 8 * v) * TS_LDK + i4 + r];
            const float tl = sTl[(tc + 8 * v) * TS_LDK + i4 + r];
#pragma unroll
            for (int u = 0; u < RPT; ++u) df_mac(acc[u][v], cmp[u][v], zz[u], th, tl);
          }
        }
      }
    }
    __syncthreads();
  }

  // partial sums of this row chunk
  const int64_t kb = d0 + tk * RPT;
  if constexpr (!DF) {
    float* W = (float*)Wv + (size_t)blockIdx.y * N * ldw;
#pragma unroll
    for (int v = 0; v < NPT; ++v) {
      const int j = j0 + tc + 8 * v;
      if (j >= N) continue;
      float* w = W + (int64_t)j * ldw + kb;
      *(float4*)w = make_float4(acc[0][v], acc[1][v], acc[2][v], acc[3][v]);
      *(float4*)(w + 4) = make_float4(acc[4][v], acc[5][v], acc[6][v], acc[7][v]);
    }
  } else {
    double* W = (double*)Wv + (size_t)blockIdx.y * N * ldw;
#pragma unroll
    for (int v = 0; v < NPT; ++v) {
      const int j = j0 + tc + 8 * v;
      if (j >= N) continue;
      double* w = W + (int64_t)j * ldw + kb;
#pragma unroll
      for (int u = 0; u < RPT; ++u) w[u] = (double)acc[u][v] + (double)cmp[u][v];
    }
  }
}

// Y (D x N, column-major, ldy) = alpha sum_c W[c] + beta Y, sums in FP64 in chunk order.
template <typename TW, typename TY>
__global__ void k_tsm_reduce(int64_t D, int N, int chunks, const TW* __restrict__ W, int64_t ldw, double alpha,
                             double beta, TY* Y, int64_t ldy) {
  const int64_t total = D * N;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = idx % D;
    const int j = (int)(idx / D);
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += (double)W[((size_t)c * N + j) * ldw + k];
    TY* y = Y + k + (int64_t)j * ldy;
    const double val = alpha * s;
    *y = (TY)(beta == 0.0 ? val : fma(beta, (double)*y, val));
  }
}

template <bool DF>
constexpr int nn_smem(int NPT) {
  return 2 * (TsCfg<DF>::BM * TS_LDK + (DF ? 2 : 1) * 8 * NPT * TS_LDK) * 4;
}
template <bool DF>
constexpr int tn_smem(int NPT) {
  return 2 * (TS_BK * (TsCfg<DF>::BM + 4) + (DF ? 2 : 1) * 8 * NPT * TS_LDK) * 4;
}

template <int NPT, bool DF>
cudaError_t nn_launch(int64_t M, int N, int64_t K, double alpha, const float* A, int64_t lda, const float* B,
                      const float* Blo,
                      int64_t ldb, double beta, void* C, int64_t ldc, cudaStream_t st) {
  constexpr int smem = nn_smem<DF>(NPT);
  static_assert(8 * NPT * (TsCfg<DF>::BM + 4) * (DF ? 8 : 4) <= smem, "epilogue tile exceeds the stage buffers");
  cudaError_t e = cudaFuncSetAttribute(k_tsm_nn<NPT, DF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int nt = (N + 8 * NPT - 1) / (8 * NPT);
  const int64_t mt = (M + TsCfg<DF>::BM - 1) / TsCfg<DF>::BM;
  // column tiles vary fastest so that the tiles of one row block run together and
  // read that block of A from HBM once
  dim3 grid((unsigned)nt, (unsigned)mt);
  if (mt > 65535) return cudaErrorInvalidValue;
  k_tsm_nn<NPT, DF><<<grid, TS_TH, smem, st>>>(M, N, K, alpha, A, lda, B, Blo, ldb, beta, C, ldc);
  return cudaGetLastError();
}

template <int NPT, bool DF>
cudaError_t tn_launch(int64_t R, int64_t D, int N, const float* Z, int64_t ldz, const float* T, const float* Tlo,
                      int64_t ldt,
                      double alpha, double beta, void* Y, int64_t ldy, void* work, size_t work_bytes, int sms,
                      cudaStream_t st) {
  constexpr int smem = tn_smem<DF>(NPT);
  cudaError_t e = cudaFuncSetAttribute(k_tsm_tn<NPT, DF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  constexpr int BD = TsCfg<DF>::BM, NT = 8 * NPT;
  const int nt = (N + NT - 1) / NT;
  const int64_t dt = (D + BD - 1) / BD;
  const int64_t ldw = dt * BD;
  // row chunks: about six CTAs per SM in total, chunks a multiple of the slice depth
  int64_t chunks = std::max<int64_t>(1, (6LL * sms + dt * nt - 1) / (dt * nt));
  const int64_t max_chunks = std::max<int64_t>(1, (R + 4 * TS_BK - 1) / (4 * TS_BK));
  chunks = std::min<int64_t>(std::min<int64_t>(chunks, max_chunks), 65535);
  int64_t rpc = (R + chunks - 1) / chunks;
  rpc = (rpc + TS_BK - 1) / TS_BK * TS_BK;
  chunks = (R + rpc - 1) / rpc;
  const size_t need = (size_t)chunks * N * ldw * (DF ? 8 : 4);
  if (need > work_bytes || !work) return cudaErrorInvalidValue;
  if (dt > 0x7fffffff) return cudaErrorInvalidValue;
  dim3 grid((unsigned)dt, (unsigned)chunks, (unsigned)nt);
  k_tsm_tn<NPT, DF><<<grid, TS_TH, smem, st>>>(R, D, N, rpc, Z, ldz, T, Tlo, ldt, work, ldw);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t total = D * N;
  const int rb = (int)std::min<int64_t>((total + 255) / 256, 8LL * sms);
  if (DF)
    k_tsm_reduce<double, double><<<rb, 256, 0, st>>>(D, N, (int)chunks, (const double*)work, ldw, alpha, beta,
                                                     (double*)Y, ldy);
  else
    k_tsm_reduce<float, float><<<rb, 256, 0, st>>>(D, N, (int)chunks, (const float*)work, ldw, alpha, beta,
                                                   (float*)Y, ldy);
  return cudaGetLastError();
}

// columns per thread for an N-column product: one tile of 8 NPT >= N when N <= 72,
// else tiles of 64
int pick_npt(int N) { return N <= 72 ? (N + 7) / 8 : 8; }

}  // namespace

bool tsm_supported(const void* A, int64_t lda) {
  return !((uintptr_t)A & 15) && !(lda & 3);
}

namespace {
// hi/lo (rows x cols, column-major, ldd >= rows) = FP32 head and tail of src (rows x
// cols, lds); rows rows..ldd-1 of hi and lo are zeroed
__global__ void k_split_f64(int64_t rows, int cols, const double* __restrict__ src, int64_t lds, float* hi, float* lo,
                            int64_t ldd) {
  const int64_t total = ldd * cols;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % ldd;
    const int j = (int)(idx / ldd);
    float h = 0.f, l = 0.f;
    if (i < rows) split_f64(src[i + (int64_t)j * lds], h, l);
    hi[idx] = h;
    lo[idx] = l;
  }
}
}  // namespace

cudaError_t launch_split_f64(int64_t rows, int cols, const double* src, int64_t lds, float* hi, float* lo, int64_t ldd,
                             cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  if (ldd < rows) return cudaErrorInvalidValue;
  const int64_t total = ldd * cols;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, 8192);
  k_split_f64<<<grid, 256, 0, st>>>(rows, cols, src, lds, hi, lo, ldd);
  return cudaGetLastError();
}

size_t tsm_tn_work_bytes(int64_t R, int64_t D, int N, int df, int sms) {
  const int npt = pick_npt(N);
  const int BD = df ? TsCfg<true>::BM : TsCfg<false>::BM, NT = 8 * npt;
  const int64_t dt = (D + BD - 1) / BD, nt = (N + NT - 1) / NT;
  int64_t chunks = std::max<int64_t>(1, (6LL * sms + dt * nt - 1) / (dt * nt));
  const int64_t max_chunks = std::max<int64_t>(1, (R + 4 * TS_BK - 1) / (4 * TS_BK));
  chunks = std::min<int64_t>(std::min<int64_t>(chunks, max_chunks), 65535);
  return (size_t)chunks * N * dt * BD * (df ? 8 : 4);
}

#define BK_NPT_DISPATCH(NPTV, CALL) \
  switch (NPTV) {                   \
    case 1: return CALL(1);         \
    case 2: return CALL(2);         \
    case 3: return CALL(3);         \
    case 4: return CALL(4);         \
    case 5: return CALL(5);         \
    case 6: return CALL(6);         \
    case 7: return CALL(7);         \
    case 8: return CALL(8);         \
    case 9: return CALL(9);         \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t launch_tsm_nn(int df, int64_t M, int N, int64_t K, double alpha, const float* A, int64_t lda,
                          const float* B, const float* Blo, int64_t ldb, double beta, void* C, int64_t ldc,
                          cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (!tsm_supported(A, lda) || !tsm_supported(B, ldb) || (df && !tsm_supported(Blo, ldb)))
    return cudaErrorInvalidValue;
  const int npt = pick_npt(N);
#define NN_F32(P) nn_launch<P, false>(M, N, K, alpha, A, lda, B, Blo, ldb, beta, C, ldc, st)
#define NN_DF(P) nn_launch<P, true>(M, N, K, alpha, A, lda, B, Blo, ldb, beta, C, ldc, st)
  if (df) {
    BK_NPT_DISPATCH(npt, NN_DF)
  } else {
    BK_NPT_DISPATCH(npt, NN_F32)
  }
#undef NN_F32
#undef NN_DF
}

cudaError_t launch_tsm_tn(int df, int64_t R, int64_t D, int N, const float* Z, int64_t ldz, const float* T,
                          const float* Tlo, int64_t ldt, double alpha, double beta, void* Y, int64_t ldy, void* work,
                          size_t work_bytes, int sms, cudaStream_t st) {
  if (D <= 0 || N <= 0) return cudaSuccess;
  if (!tsm_supported(Z, ldz) || !tsm_supported(T, ldt) || (df && !tsm_supported(Tlo, ldt)))
    return cudaErrorInvalidValue;
  const int npt = pick_npt(N);
#define TN_F32(P) tn_launch<P, false>(R, D, N, Z, ldz, T, Tlo, ldt, alpha, beta, Y, ldy, work, work_bytes, sms, st)
#define TN_DF(P) tn_launch<P, true>(R, D, N, Z, ldz, T, Tlo, ldt, alpha, beta, Y, ldy, work, work_bytes, sms, st)
  if (df) {
    BK_NPT_DISPATCH(npt, TN_DF)
  } else {
    BK_NPT_DISPATCH(npt, TN_F32)
  }
#undef TN_F32
#undef TN_DF
}

}  // namespace bk
