// Tensor-core dense block product Y = A P + mu P with the fused Gram G = P^T Y, for
// FP32 matrices (Sec. 1.2: the loads of A are the cost of the method). 5th-generation
// tensor cores (tcgen05) with TF32 inputs and an FP32 accumulator in tensor memory;
// FP32 accuracy is kept by splitting both operands into a TF32 head and an FP32 tail
// and accumulating three products (A_hi P_hi + A_hi P_lo + A_lo P_hi; the dropped
// A_lo P_lo is ~2^-26 relative).
//
// One CTA computes one 128-row tile of Y over all columns:
//   warp 0      TMA producer: A tile (128 rows x 32 K, 128-byte swizzle) and the two
//               32 x N slices of P^T (head and tail) per stage, 4 stages;
//   warp 1      allocates tensor memory and issues the MMAs (M = 128, N = 16/32/48,
//               K = 8 per instruction, 12 per stage) into one of two accumulators,
//               then commits to the stage's "empty" and the accumulator's "full"
//               barrier;
//   warps 2-5   split each A tile in place into head and tail (the split is
//               elementwise, so the swizzled layout is kept), and drain the
//               accumulator of the previous stage into FP32 registers (one row per
//               thread). The tensor core's FP32 accumulation does not round to
//               nearest, and its error grows with the number of accumulation steps;
//               summing 32-wide K slices in registers keeps the product at FFMA
//               accuracy. The epilogue adds mu P, writes Y in the panel layout and
//               stages P and Y rows for the Gram.
// All threads then form the per-CTA Gram partial (bk_tile.cuh).
//
// P^T is prepared once per product by k_pt_split: rows [0, N) hold the TF32 heads of
// the columns of P, rows [N, 2N) the tails, leading dimension ldk = round_up(d, 32).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <mutex>

#include "bk_batch.cuh"
#include "bk_common.cuh"
#include "bk_sm100.cuh"
#include "bk_tile.cuh"

namespace bk {
namespace {

using namespace sm100;

constexpr int kTcThreads = 192;

template <int MP>
struct TcShape {
  static constexpr int N = MP <= 16 ? 16 : (MP <= 32 ? 32 : 48);  // MMA width (multiple of 16)
  static constexpr int S = 4;                                     // pipeline stages
  static constexpr int kA = 128 * 32 * 4;                         // one A tile (head or tail)
  static constexpr int kB = N * 32 * 4;                           // one P^T slice (head or tail)
  static constexpr int kStage = 2 * kA + 2 * kB;
  static constexpr int kBar = S * kStage;  // barrier area after the stages
  static constexpr int kSmem = kBar + 256 + 1024;  // + barriers, + alignment slack
  static constexpr uint32_t kTmemCols = 128;  // two accumulators of 64 columns
  static_assert(kB % 1024 == 0, "operand tiles must stay on 1024-byte boundaries");
};

__device__ __forceinline__ float tf32_head(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// P (panels) -> P^T head and tail rows, zero beyond d and beyond m.
template <int MP>
__global__ void k_pt_split(int64_t d, const float* __restrict__ P, int64_t ld, int m, float* __restrict__ PT,
                           int64_t ldk) {
  constexpr int N = TcShape<MP>::N;
  const int nq = (m + 3) >> 2;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ldk; k += (int64_t)gridDim.x * blockDim.x) {
    float v[MP];
#pragma unroll
    for (int q = 0; q < MP / 4; ++q) {
      if (k < d && q < nq)
        ldg4(panel_row(P, ld, q, k), v + 4 * q);
      else {
#pragma unroll
        for (int u = 0; u < 4; ++u) v[4 * q + u] = 0.f;
      }
    }
#pragma unroll
    for (int c = 0; c < N; ++c) {
      const float x = (c < MP) ? v[c < MP ? c : 0] : 0.f;
      const float h = tf32_head(x);
      PT[(int64_t)c * ldk + k] = h;
      PT[(int64_t)(N + c) * ldk + k] = x - h;
    }
  }
}

// One 128-row tile of one system: rows [128 tile, 128 tile + 128) of Y and the Gram
// partial number `tile` of `nparts`. amap/bmap point to the system's tensor maps
// (kernel parameters or global memory).
template <int MP>
__device__ __forceinline__ void dense_tc_tile(const CUtensorMap* amap_p, const CUtensorMap* bmap_p, int64_t d,
                                              int tile, const float* __restrict__ P, float* __restrict__ Y,
                                              int64_t ld, int m, float mu, double* parts, int nparts, int* err) {
  using SH = TcShape<MP>;
  constexpr int N = SH::N, S = SH::S;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(base + SH::kBar);
  uint64_t* split = full + S;
  uint64_t* empty = split + S;
  uint64_t* acc_full = empty + S;   // [2]
  uint64_t* acc_empty = acc_full + 2;  // [2]
  uint64_t* cleanup = acc_empty + 2;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(cleanup + 1);
  volatile int* s_abort = reinterpret_cast<volatile int*>(tmem_holder + 1);
  volatile int* s_consumed = s_abort + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = (int)((d + 31) / 32);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full + s, 1);
      mbar_init(split + s, 128);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full + b, 1);
      mbar_init(acc_empty + b, 128);
    }
    mbar_init(cleanup, 1);
    *s_abort = 0;
    *s_consumed = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tmem_holder, SH::kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  int issued = 0;  // k-blocks whose loads warp 0 issued
  float sum[N];    // warps 2-5: this thread's row of the product
  if (warp == 0) {
    if (lane == 0) {
      tma_prefetch_desc(amap_p);
      tma_prefetch_desc(bmap_p);
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % S;
        const uint32_t r = (uint32_t)(kb / S);
        if (*s_abort) break;
        if (r > 0 && !mbar_wait(empty + s, (r - 1) & 1)) {
          *s_abort = 1;
          break;
        }
        uint8_t* st = base + s * SH::kStage;
        mbar_arrive_expect_tx(full + s, SH::kA + 2 * SH::kB);
        tma_load_2d(st, amap_p, full + s, kb * 32, tile * 128);
        tma_load_2d(st + 2 * SH::kA, bmap_p, full + s, kb * 32, 0);
        tma_load_2d(st + 2 * SH::kA + SH::kB, bmap_p, full + s, kb * 32, N);
        issued = kb + 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(128, N);
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % S;
        const uint32_t r = (uint32_t)(kb / S);
        const int b = kb & 1;
        if (*s_abort) break;
        if (kb >= 2 && !mbar_wait(acc_empty + b, (uint32_t)((kb >> 1) - 1) & 1)) {
          *s_abort = 1;
          break;
        }
        if (!mbar_wait(split + s, r & 1)) {
          *s_abort = 1;
          break;
        }
        tc_fence_after();
        uint8_t* st = base + s * SH::kStage;
        const uint32_t ahi = smem_u32(st), alo = smem_u32(st + SH::kA);
        const uint32_t bhi = smem_u32(st + 2 * SH::kA), blo = smem_u32(st + 2 * SH::kA + SH::kB);
        const uint32_t acc = tmem + 64u * b;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t off = 32u * k;  // 8 TF32 elements of K
          mma_tf32(acc, desc_kmajor_sw128(ahi + off), desc_kmajor_sw128(bhi + off), idesc, k != 0);
          mma_tf32(acc, desc_kmajor_sw128(ahi + off), desc_kmajor_sw128(blo + off), idesc, 1u);
          mma_tf32(acc, desc_kmajor_sw128(alo + off), desc_kmajor_sw128(bhi + off), idesc, 1u);
        }
        mma_commit(empty + s);
        mma_commit(acc_full + b);
      }
    }
  } else {
    const int ct = threadIdx.x - 64;  // 0..127
    const int qd = warp & 3;          // tensor-memory lane quarter of this warp
#pragma unroll
    for (int c = 0; c < N; ++c) sum[c] = 0.f;
    for (int kb = 0; kb <= nk; ++kb) {
      // every exit decision below is warp-uniform: the warp runs collective
      // tensor-memory loads
      if (__any_sync(0xffffffffu, *s_abort != 0)) break;
      if (kb < nk) {
        const int s = kb % S;
        const uint32_t r = (uint32_t)(kb / S);
        if (!__all_sync(0xffffffffu, mbar_wait(full + s, r & 1))) {
          *s_abort = 1;
          break;
        }
        uint8_t* st = base + s * SH::kStage;
        float4* h = reinterpret_cast<float4*>(st);
        float4* l = reinterpret_cast<float4*>(st + SH::kA);
#pragma unroll
        for (int j = 0; j < SH::kA / 16 / 128; ++j) {
          const int idx = ct + 128 * j;
          const float4 v = h[idx];
          const float4 hv = make_float4(tf32_head(v.x), tf32_head(v.y), tf32_head(v.z), tf32_head(v.w));
          h[idx] = hv;
          l[idx] = make_float4(v.x - hv.x, v.y - hv.y, v.z - hv.z, v.w - hv.w);
        }
        fence_proxy_async_smem();
        mbar_arrive(split + s);
        if (ct == 0) *s_consumed = kb + 1;
      }
      if (kb >= 1) {  // drain the accumulator of k-block kb - 1
        const int kp = kb - 1, b = kp & 1;
        if (!__all_sync(0xffffffffu, mbar_wait(acc_full + b, (uint32_t)(kp >> 1) & 1))) {
          *s_abort = 1;
          break;
        }
        tc_fence_after();
        uint32_t rr[N / 16][16];
#pragma unroll
        for (int c = 0; c < N / 16; ++c) tmem_ld16(tmem + ((uint32_t)(32 * qd) << 16) + 64u * b + 16u * c, rr[c]);
        tmem_ld_wait();
#pragma unroll
        for (int c = 0; c < N; ++c) sum[c] += __uint_as_float(rr[c / 16][c % 16]);
        tc_fence_before();
        mbar_arrive(acc_empty + b);
      }
    }
  }

  // ---- drain: every role has left its loop
  __syncthreads();
  const bool aborted = *s_abort != 0;
  if (aborted) {
    // let issued loads land and issued MMAs finish before the memory is reused or freed
    if (warp == 0 && lane == 0)
      for (int kb = *s_consumed; kb < issued; ++kb) mbar_wait(full + kb % S, (uint32_t)(kb / S) & 1);
    if (warp == 1 && lane == 0) {
      mma_commit(cleanup);
      mbar_wait(cleanup, 0);
    }
    if (threadIdx.x == 0 && err) atomicExch(err, 1);
  }
  __syncthreads();

  // ---- epilogue: rows of the accumulator -> Y, and the Gram tiles
  float* sX = reinterpret_cast<float*>(base);
  float* sY = sX + 128 * MP;
  if (warp >= 2) {
    const int row = 32 * (warp & 3) + lane;
    const int64_t gi = (int64_t)tile * 128 + row;
    float acc[N];
#pragma unroll
    for (int c = 0; c < N; ++c) acc[c] = aborted ? 0.f : sum[c];
    const int nq = (m + 3) >> 2;
    float pv[MP], yv[MP];
#pragma unroll
    for (int q = 0; q < MP / 4; ++q) {
      const bool live = gi < d && q < nq;
      if (live)
        ldg4(panel_row(P, ld, q, gi), pv + 4 * q);
      else {
#pragma unroll
        for (int u = 0; u < 4; ++u) pv[4 * q + u] = 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) yv[4 * q + u] = live ? fmaf(mu, pv[4 * q + u], acc[4 * q + u]) : 0.f;
      if (live) st4(panel_row(Y, ld, q, gi), yv + 4 * q);
    }
    store_row<MP>(sX, row, pv);
    store_row<MP>(sY, row, yv);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, SH::kTmemCols);
  GramAcc<float, MP> g;
  g.init();
  g.tile(sX, sY, 128);
  __syncthreads();
  gram_finish<float, MP>(g, reinterpret_cast<double*>(base), parts, nparts, tile);
}

template <int MP>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_dense_tc(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap, int64_t d,
               const float* __restrict__ P, float* __restrict__ Y, int64_t ld, int m, float mu, double* parts,
               int nparts, const DevState* state, int* err) {
  if (state && (state->done_a | state->done_b)) return;
  dense_tc_tile<MP>(&amap, &bmap, d, blockIdx.x, P, Y, ld, m, mu, parts, nparts, err);
}

// Batched: CTA i computes row tile tile_row[i] of system tile_sys[i].
template <int MP>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_bdense_tc(const BSys* __restrict__ sys, const int* __restrict__ tile_sys, const int* __restrict__ tile_row,
                const CUtensorMap* __restrict__ maps) {
  const int k = tile_sys[blockIdx.x];
  const BSys& S = sys[k];
  if (S.st->done_a | S.st->done_b) return;
  dense_tc_tile<MP>(maps + 2 * k, maps + 2 * k + 1, S.d, tile_row[blockIdx.x], static_cast<const float*>(S.P),
                    static_cast<float*>(S.Y), S.ld, S.m, (float)S.mu, S.Gp, S.npG, &S.st->timeout);
}

// Batched P^T split over the group's thread-block ranges.
template <int MP>
__global__ void k_bpt_split(const BSys* __restrict__ sys, const int* __restrict__ cta_sys) {
  constexpr int N = TcShape<MP>::N;
  const BSys& S = sys[cta_sys[blockIdx.x]];
  if (S.st->done_a | S.st->done_b) return;
  const int j = blockIdx.x - S.cta0;
  const int64_t d = S.d, ldk = (d + 31) & ~int64_t(31);
  const int nq = (S.m + 3) >> 2;
  const float* P = static_cast<const float*>(S.P);
  for (int64_t k = (int64_t)j * blockDim.x + threadIdx.x; k < ldk; k += (int64_t)S.ncta * blockDim.x) {
    float v[MP];
#pragma unroll
    for (int q = 0; q < MP / 4; ++q) {
      if (k < d && q < nq)
        ldg4(panel_row(P, S.ld, q, k), v + 4 * q);
      else {
#pragma unroll
        for (int u = 0; u < 4; ++u) v[4 * q + u] = 0.f;
      }
    }
#pragma unroll
    for (int c = 0; c < N; ++c) {
      const float x = (c < MP) ? v[c < MP ? c : 0] : 0.f;
      const float h = tf32_head(x);
      S.pt[(int64_t)c * ldk + k] = h;
      S.pt[(int64_t)(N + c) * ldk + k] = x - h;
    }
  }
}

template <int MP>
cudaError_t batch_tc_impl(BSys* sys, const int* cta_sys, int ncta, const BatchTc& tc, cudaStream_t st) {
  using SH = TcShape<MP>;
  k_bpt_split<MP><<<ncta, 128, 0, st>>>(sys, cta_sys);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  auto k = k_bdense_tc<MP>;
  if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SH::kSmem)) != cudaSuccess) return e;
  k<<<tc.ntiles, kTcThreads, SH::kSmem, st>>>(sys, tc.tile_sys, tc.tile_row,
                                               static_cast<const CUtensorMap*>(tc.maps));
  return cudaGetLastError();
}

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2D FP32 tensor (inner extent x, outer extent y, row pitch in elements) read in boxes
// of 32 x box_y with 128-byte swizzle; out-of-range elements read as zero.
cudaError_t make_map(CUtensorMap* map, const float* ptr, int64_t x, int64_t y, int64_t pitch, int box_y) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)x, (cuuint64_t)y};
  cuuint64_t strides[1] = {(cuuint64_t)pitch * 4};
  cuuint32_t box[2] = {32u, (cuuint32_t)box_y};
  cuuint32_t estr[2] = {1u, 1u};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int MP>
cudaError_t dense_tc_impl(int64_t d, const float* A, int64_t lda, double mu, const float* P, float* Y, int64_t ld,
                          int m, double* parts, int nparts, const DevState* state, float* pt, int* err,
                          cudaStream_t st) {
  using SH = TcShape<MP>;
  const int64_t ldk = (d + 31) & ~int64_t(31);
  CUtensorMap amap, bmap;
  cudaError_t e;
  if ((e = make_map(&amap, A, d, d, lda, 128)) != cudaSuccess) return e;
  if ((e = make_map(&bmap, pt, d, 2 * SH::N, ldk, SH::N)) != cudaSuccess) return e;
  int g = (int)((ldk + 255) / 256);
  if (g > 152 * 8) g = 152 * 8;
  k_pt_split<MP><<<g, 256, 0, st>>>(d, P, ld, m, pt, ldk);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  auto k = k_dense_tc<MP>;
  if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SH::kSmem)) != cudaSuccess) return e;
  k<<<nparts, kTcThreads, SH::kSmem, st>>>(amap, bmap, d, P, Y, ld, m, (float)mu, parts, nparts, state, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_batch_dense_tc(int mp, BSys* sys, const int* cta_sys, int ncta, const BatchTc& tc,
                                  cudaStream_t st) {
  if (tc.ntiles < 1) return cudaSuccess;
  switch (mp) {
    case 4: return batch_tc_impl<4>(sys, cta_sys, ncta, tc, st);
    case 8: return batch_tc_impl<8>(sys, cta_sys, ncta, tc, st);
    case 16: return batch_tc_impl<16>(sys, cta_sys, ncta, tc, st);
    case 24: return batch_tc_impl<24>(sys, cta_sys, ncta, tc, st);
    case 36: return batch_tc_impl<36>(sys, cta_sys, ncta, tc, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t tc_make_maps(int mp, int64_t d, const float* A, int64_t lda, const float* pt, void* out) {
  const int n = mp <= 16 ? 16 : (mp <= 32 ? 32 : 48);
  CUtensorMap* maps = static_cast<CUtensorMap*>(out);
  cudaError_t e = make_map(maps, A, d, d, lda, 128);
  if (e != cudaSuccess) return e;
  return make_map(maps + 1, pt, d, 2 * n, (d + 31) & ~int64_t(31), n);
}

bool dense_tc_usable(int64_t d, const void* A, int64_t lda, int mp) {
  if (std::getenv("BK_NO_TC")) return false;
  if (mp > 36 || d < 1 || d > (int64_t)1 << 31) return false;
  if ((reinterpret_cast<uintptr_t>(A) & 15) != 0 || (lda & 3) != 0) return false;  // TMA: 16-byte rows
  return encode_fn() != nullptr;
}
int dense_tc_tiles(int64_t d) { return (int)((d + 127) / 128); }
size_t dense_tc_pt_bytes(int64_t d, int mp) {
  const int n = mp <= 16 ? 16 : (mp <= 32 ? 32 : 48);
  return (size_t)2 * n * (size_t)((d + 31) & ~int64_t(31)) * 4;
}

cudaError_t launch_dense_gram_tc(int mp, int64_t d, const float* A, int64_t lda, double mu, const float* P, float* Y,
                                 int64_t ld, int m, double* parts, int nparts, const DevState* state, float* pt,
                                 int* err, cudaStream_t st) {
  if (nparts != dense_tc_tiles(d)) return cudaErrorInvalidValue;
  switch (mp) {
    case 4: return dense_tc_impl<4>(d, A, lda, mu, P, Y, ld, m, parts, nparts, state, pt, err, st);
    case 8: return dense_tc_impl<8>(d, A, lda, mu, P, Y, ld, m, parts, nparts, state, pt, err, st);
    case 16: return dense_tc_impl<16>(d, A, lda, mu, P, Y, ld, m, parts, nparts, state, pt, err, st);
    case 24: return dense_tc_impl<24>(d, A, lda, mu, P, Y, ld, m, parts, nparts, state, pt, err, st);
    case 36: return dense_tc_impl<36>(d, A, lda, mu, P, Y, ld, m, parts, nparts, state, pt, err, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bk
