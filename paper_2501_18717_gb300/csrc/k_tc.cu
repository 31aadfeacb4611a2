// Tensor-core dense block product Y = A P + mu P with the fused Gram G = P^T Y, for
// FP32 matrices (Sec. 1.2: the loads of A are the cost of the method). 5th-generation
// tensor cores (tcgen05) with TF32 inputs and an FP32 accumulator in tensor memory;
// FP32 accuracy is kept by splitting both operands into a TF32 head and a TF32 tail
// (both rounded to nearest, tf32_split) and accumulating three products (A_hi P_hi +
// A_hi P_lo + A_lo P_hi; the dropped A_lo P_lo is ~2^-24 relative).
//
// One CTA computes one 128-row tile of Y over all columns, in pipeline steps of 64
// columns of K (two 128-byte swizzle boxes). A tiles land in a ring of 4 stages that
// is refilled as soon as the split warps have read a tile; the P^T slices have their
// own ring of 3 stages that the MMAs release; the split head/tail of A lives in tensor
// memory (two stages), which the MMAs read as their A operand.
//   warp 0      TMA producer for A (128 rows x 32 K per box, 128-byte swizzle);
//   warp 2      TMA producer for the P^T head and tail slices (adjacent rows, from L2);
//   warp 1      allocates tensor memory and issues the MMAs into one of two
//               accumulators: per 8-wide K step A_hi [P_hi; P_lo] (2N columns) and
//               A_lo P_hi added to the first N columns; then commits to the A stage's
//               "empty", the P^T stage's "empty" and the accumulator's "full" barrier;
//   warps 3-10  read their rows of the swizzled A tile, split them into head and tail
//               and store both into tensor memory; then drain the accumulator of the
//               previous step into FP32 registers (each lane quarter is read by two
//               warps, one per half of the columns). The tensor core's FP32
//               accumulation does not round to nearest and its error grows with the
//               number of accumulation steps; summing 64-wide K slices in registers
//               keeps the product at FFMA accuracy.
// The epilogue joins the column halves in shared memory, adds mu P, writes Y in the
// panel layout and stages P and Y rows; all threads then form the per-CTA Gram
// partial (bk_tile.cuh).
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

constexpr int kTcThreads = 352;  // warp 0 A loads, warp 1 MMA, warp 2 P^T loads, warps 3-10 split / drain

template <int MP>
struct TcShape {
  static constexpr int N = MP <= 16 ? 16 : (MP <= 32 ? 32 : 48);  // columns of P (multiple of 16)
  static constexpr int KS = 64;                                   // K per pipeline step (two 32-wide boxes)
  static constexpr int R = 4;                                     // A landing stages
  static constexpr int RB = 3;                                    // P^T slice stages
  static constexpr int W = 2;                                     // A head/tail stages in tensor memory
  static constexpr int kBox = 128 * 32 * 4;                       // one A box: 128 rows x 32 K
  static constexpr int kA = 2 * kBox;                             // one A stage as loaded
  static constexpr int kBBox = 2 * N * 32 * 4;                    // one P^T box: head N rows, tail N rows
  static constexpr int kB = 2 * kBBox;                            // one P^T stage
  static constexpr int kOffB = R * kA;                            // P^T ring
  static constexpr int kBar = kOffB + RB * kB;                    // barrier area after the buffers
  static constexpr int kSmem = kBar + 512 + 1024;                 // + barriers, + alignment slack
  static constexpr uint32_t kAccCols = 128;                       // one accumulator: 2N <= 96 columns
  static constexpr uint32_t kACols = 128;                         // one A stage: head 64 + tail 64 columns
  static constexpr uint32_t kAOff = 2 * kAccCols;                 // A stages after the two accumulators
  static constexpr uint32_t kTmemCols = 512;
  static_assert(kAOff + W * kACols <= kTmemCols, "tensor memory budget");
  static_assert(kBBox % 1024 == 0, "operand tiles must stay on 1024-byte boundaries");
  static_assert((N / 2) % 8 == 0, "each drain warp reads whole 8-column groups");
  static_assert((128 * (N + 1) * 4) % 16 == 0, "Gram staging stays 16-byte aligned");
  static_assert(kSmem <= 232448, "shared memory per CTA");
  static_assert(128 * (N + 1 + 2 * MP) * 4 <= kOffB, "epilogue staging fits in the A ring");
};

// TF32 value nearest to x (round to nearest, ties away from zero).
__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// x = h + l + e with h, l exact TF32 values and |e| <= 2^-24 |x| (about FP32 rounding):
// h is x rounded to TF32 (|x - h| <= 2^-12 |x|) and l is that difference rounded to
// TF32. A truncated head leaves a 13-bit tail that the MMA would truncate again (error
// up to 2^-22 |x|), which showed as more block-CG iterations.
__device__ __forceinline__ void tf32_split(float x, float& h, float& l) {
  h = tf32_rn(x);
  l = tf32_rn(x - h);
}

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
      float h, l;
      tf32_split(x, h, l);
      PT[(int64_t)c * ldk + k] = h;
      PT[(int64_t)(N + c) * ldk + k] = l;
    }
  }
}

// One 128-row tile of one system: rows [128 tile, 128 tile + 128) of Y and the Gram
// partial number `tile` of `nparts`. amap/bmap point to the system's tensor maps
// (kernel parameters or global memory).
template <int MP>
__device__ __forceinline__ void dense_tc_tile(const CUtensorMap* amap_p, const CUtensorMap* bmap_p, int64_t d,
                                              int tile, const float* __restrict__ P, float* __restrict__ Y,
                                              int64_t ld, int m, float mu, double* parts, int nparts, int* err,
                                              long long wait) {
  using SH = TcShape<MP>;
  constexpr int N = SH::N, R = SH::R, RB = SH::RB, W = SH::W, NH = N / 2;
  constexpr int kConv = kTcThreads - 96;  // split / drain threads (warps 3..10)
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* raw = base;                 // R x kA: A tiles as loaded (128-byte swizzle)
  uint8_t* bring = base + SH::kOffB;   // RB x 2 kB: P^T head + tail slices
  uint64_t* raw_full = reinterpret_cast<uint64_t*>(base + SH::kBar);
  uint64_t* raw_empty = raw_full + R;
  uint64_t* b_full = raw_empty + R;    // [RB]
  uint64_t* b_empty = b_full + RB;     // [RB]
  uint64_t* w_split = b_empty + RB;    // [W]
  uint64_t* w_empty = w_split + W;     // [W]
  uint64_t* acc_full = w_empty + W;    // [2]
  uint64_t* acc_empty = acc_full + 2;  // [2]
  uint64_t* cleanup = acc_empty + 2;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(cleanup + 1);
  volatile int* s_abort = reinterpret_cast<volatile int*>(tmem_holder + 1);
  volatile int* s_a_consumed = s_abort + 1;  // A tiles read by the split warps
  volatile int* s_b_consumed = s_abort + 2;  // P^T slices taken by the MMA thread
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = (int)((d + SH::KS - 1) / SH::KS);  // pipeline steps of KS columns

  if (threadIdx.x == 0) {
    for (int s = 0; s < R; ++s) {
      mbar_init(raw_full + s, 1);
      mbar_init(raw_empty + s, kConv);
    }
    for (int t = 0; t < RB; ++t) {
      mbar_init(b_full + t, 1);
      mbar_init(b_empty + t, 1);
    }
    for (int w = 0; w < W; ++w) {
      mbar_init(w_split + w, kConv);
      mbar_init(w_empty + w, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full + b, 1);
      mbar_init(acc_empty + b, kConv);
    }
    mbar_init(cleanup, 1);
    *s_abort = 0;
    *s_a_consumed = 0;
    *s_b_consumed = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tmem_holder, SH::kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  int issued = 0;  // loads issued by this producer thread (warp 0: A tiles, warp 2: P^T slices)
  float sum[NH];   // warps 3..10: half a row of the product (this warp's columns)
  if (warp == 0) {
    if (lane == 0) {  // A tiles, up to R ahead of the split warps
      tma_prefetch_desc(amap_p);
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % R;
        if (*s_abort) break;
        if (kb >= R && !mbar_wait(raw_empty + s, (uint32_t)((kb / R) - 1) & 1, wait)) {
          *s_abort = 1;
          break;
        }
        mbar_arrive_expect_tx(raw_full + s, SH::kA);
        tma_load_2d(raw + s * SH::kA, amap_p, raw_full + s, kb * SH::KS, tile * 128);
        tma_load_2d(raw + s * SH::kA + SH::kBox, amap_p, raw_full + s, kb * SH::KS + 32, tile * 128);
        issued = kb + 1;
      }
    }
  } else if (warp == 2) {
    if (lane == 0) {  // P^T head and tail slices (L2-resident), up to RB ahead of the MMAs
      tma_prefetch_desc(bmap_p);
      for (int kb = 0; kb < nk; ++kb) {
        const int t = kb % RB;
        if (*s_abort) break;
        if (kb >= RB && !mbar_wait(b_empty + t, (uint32_t)((kb / RB) - 1) & 1, wait)) {
          *s_abort = 1;
          break;
        }
        uint8_t* bs = bring + t * SH::kB;
        mbar_arrive_expect_tx(b_full + t, SH::kB);
#pragma unroll
        for (int j = 0; j < 2; ++j) {  // box j: head rows, then tail rows
          tma_load_2d(bs + j * SH::kBBox, bmap_p, b_full + t, kb * SH::KS + 32 * j, 0);
          tma_load_2d(bs + j * SH::kBBox + SH::kBBox / 2, bmap_p, b_full + t, kb * SH::KS + 32 * j, N);
        }
        issued = kb + 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // per 8-wide K step: A_hi [P_hi; P_lo] (2N columns: head products in [0, N),
      // tail products in [N, 2N)), then A_lo P_hi accumulated into [0, N)
      constexpr uint32_t idesc2 = idesc_tf32(128, 2 * N);
      constexpr uint32_t idesc1 = idesc_tf32(128, N);
      for (int kb = 0; kb < nk; ++kb) {
        const int w = kb % W, t = kb % RB, b = kb & 1;
        if (*s_abort) break;
        if (kb >= 2 && !mbar_wait(acc_empty + b, (uint32_t)((kb >> 1) - 1) & 1, wait)) {
          *s_abort = 1;
          break;
        }
        if (!mbar_wait(b_full + t, (uint32_t)(kb / RB) & 1, wait)) {
          *s_abort = 1;
          break;
        }
        *s_b_consumed = kb + 1;
        if (!mbar_wait(w_split + w, (uint32_t)(kb / W) & 1, wait)) {
          *s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t ahi = tmem + SH::kAOff + SH::kACols * w, alo = ahi + 64;  // tensor-memory A
        const uint32_t bst = smem_u32(bring + t * SH::kB);
        const uint32_t acc = tmem + SH::kAccCols * b;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          // 8 TF32 elements of K: 8 columns of A; 32 bytes into box k / 4 of P^T (its
          // P_hi rows followed by its P_lo rows)
          const uint64_t bd = desc_kmajor_sw128(bst + SH::kBBox * (k >> 2) + 32u * (k & 3));
          mma_tf32_ts(acc, ahi + 8u * k, bd, idesc2, k != 0);
          mma_tf32_ts(acc, alo + 8u * k, bd, idesc1, 1u);
        }
        mma_commit(w_empty + w);
        mma_commit(b_empty + t);
        mma_commit(acc_full + b);
      }
    }
  } else {
    const int ct = threadIdx.x - 96;       // 0 .. kConv - 1
    const int qd = warp & 3;               // tensor-memory lane quarter of this warp
    const int half = (warp - 3) >> 2;      // which half of the columns this warp drains
#pragma unroll
    for (int c = 0; c < NH; ++c) sum[c] = 0.f;
    for (int kb = 0; kb <= nk; ++kb) {
      // every exit decision below is warp-uniform: the warp runs collective
      // tensor-memory loads
      if (__any_sync(0xffffffffu, *s_abort != 0)) break;
      if (kb < nk) {
        const int s = kb % R, w = kb % W;
        if (!__all_sync(0xffffffffu, mbar_wait(raw_full + s, (uint32_t)(kb / R) & 1, wait))) {
          *s_abort = 1;
          break;
        }
        if (kb >= W && !__all_sync(0xffffffffu, mbar_wait(w_empty + w, (uint32_t)((kb / W) - 1) & 1, wait))) {
          *s_abort = 1;
          break;
        }
        // this thread's row of the tile and its half of the 64 K columns (box `half`):
        // 8 chunks of 16 bytes, chunk c of row r stored at chunk position c ^ (r % 8)
        const int row = 32 * qd + lane;
        const uint8_t* rrow = raw + s * SH::kA + half * SH::kBox + row * 128;
        float4 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = *reinterpret_cast<const float4*>(rrow + ((j ^ (row & 7)) << 4));
        mbar_arrive(raw_empty + s);  // the A tile is in registers: its buffer can refill
        if (ct == 0) *s_a_consumed = kb + 1;
        const uint32_t arow = tmem + ((uint32_t)(32 * qd) << 16) + SH::kAOff + SH::kACols * w + 32u * half;
#pragma unroll
        for (int g = 0; g < 2; ++g) {  // 16 columns at a time
          uint32_t hv[16], lv[16];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float4 q = v[4 * g + j];
            const float x[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              float h, l;
              tf32_split(x[u], h, l);
              hv[4 * j + u] = __float_as_uint(h);
              lv[4 * j + u] = __float_as_uint(l);
            }
          }
          tmem_st16(arow + 16u * g, hv);       // head
          tmem_st16(arow + 64 + 16u * g, lv);  // tail
        }
        tmem_st_wait();
        tc_fence_before();
        mbar_arrive(w_split + w);
      }
      if (kb >= 1) {  // drain the accumulator of k-block kb - 1
        const int kp = kb - 1, b = kp & 1;
        if (!__all_sync(0xffffffffu, mbar_wait(acc_full + b, (uint32_t)(kp >> 1) & 1, wait))) {
          *s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t row_addr = tmem + ((uint32_t)(32 * qd) << 16) + SH::kAccCols * b + NH * half;
        uint32_t rh[NH / 8][8], rt[NH / 8][8];
#pragma unroll
        for (int c = 0; c < NH / 8; ++c) {
          tmem_ld8(row_addr + 8u * c, rh[c]);      // A_hi P_hi + A_lo P_hi
          tmem_ld8(row_addr + N + 8u * c, rt[c]);  // A_hi P_lo
        }
        tmem_ld_wait();
#pragma unroll
        for (int c = 0; c < NH; ++c)
          sum[c] += __uint_as_float(rh[c / 8][c % 8]) + __uint_as_float(rt[c / 8][c % 8]);
        tc_fence_before();
        mbar_arrive(acc_empty + b);
      }
    }
  }

  // ---- drain: every role has left its loop
  __syncthreads();
  const bool aborted = *s_abort != 0;
  if (aborted) {
    // let issued loads land and issued MMAs finish before the memory is reused or freed;
    // these waits keep the default limit whatever the caller's: they wait for copies
    // and MMAs already issued, which complete by themselves
    if (warp == 0 && lane == 0)
      for (int kb = *s_a_consumed; kb < issued; ++kb) mbar_wait(raw_full + kb % R, (uint32_t)(kb / R) & 1);
    if (warp == 2 && lane == 0)
      for (int kb = *s_b_consumed; kb < issued; ++kb) mbar_wait(b_full + kb % RB, (uint32_t)(kb / RB) & 1);
    if (warp == 1 && lane == 0) {
      mma_commit(cleanup);
      mbar_wait(cleanup, 0);
    }
    if (threadIdx.x == 0 && err) atomicExch(err, 1);
  }
  __syncthreads();

  // ---- epilogue: the two column halves of each row meet in shared memory
  constexpr int SA = N + 1;                      // odd row stride: conflict-free column access
  float* sAcc = reinterpret_cast<float*>(base);  // 128 x SA
  float* sX = sAcc + 128 * SA;                   // 128 x MP
  float* sY = sX + 128 * MP;
  if (warp >= 3) {
    const int row = 32 * (warp & 3) + lane, half = (warp - 3) >> 2;
#pragma unroll
    for (int c = 0; c < NH; ++c) sAcc[row * SA + NH * half + c] = aborted ? 0.f : sum[c];
  }
  __syncthreads();
  if (warp >= 3 && warp < 7) {
    const int row = 32 * (warp & 3) + lane;
    const int64_t gi = (int64_t)tile * 128 + row;
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
      for (int u = 0; u < 4; ++u) {
        const int c = 4 * q + u;
        yv[c] = live ? fmaf(mu, pv[c], sAcc[row * SA + c]) : 0.f;
      }
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
  gram_tile<128, kTcThreads>(g, sX, sY);
  __syncthreads();
  gram_finish<float, MP>(g, reinterpret_cast<double*>(base), parts, nparts, tile);
}

template <int MP>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_dense_tc(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap, int64_t d,
               const float* __restrict__ P, float* __restrict__ Y, int64_t ld, int m, float mu, double* parts,
               int nparts, const DevState* state, int* err, long long wait) {
  if (state && (state->done_a | state->done_b)) return;
  dense_tc_tile<MP>(&amap, &bmap, d, blockIdx.x, P, Y, ld, m, mu, parts, nparts, err, wait);
}

// Batched: CTA i computes row tile tile_row[i] of system tile_sys[i].
template <int MP>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_bdense_tc(const BSys* __restrict__ sys, const int* __restrict__ tile_sys, const int* __restrict__ tile_row,
                const CUtensorMap* __restrict__ maps, long long wait) {
  const int k = tile_sys[blockIdx.x];
  const BSys& S = sys[k];
  if (S.st->done_a | S.st->done_b) return;
  dense_tc_tile<MP>(maps + 2 * k, maps + 2 * k + 1, S.d, tile_row[blockIdx.x], static_cast<const float*>(S.P),
                    static_cast<float*>(S.Y), S.ld, S.m, (float)S.mu, S.Gp, S.npG, &S.st->timeout, wait);
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
      float h, l;
      tf32_split(x, h, l);
      S.pt[(int64_t)c * ldk + k] = h;
      S.pt[(int64_t)(N + c) * ldk + k] = l;
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
                                               static_cast<const CUtensorMap*>(tc.maps),
                                               tc.wait_cycles > 0 ? tc.wait_cycles : sm100::kWaitCycles);
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
                          long long wait, cudaStream_t st) {
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
  k<<<nparts, kTcThreads, SH::kSmem, st>>>(amap, bmap, d, P, Y, ld, m, (float)mu, parts, nparts, state, err,
                                           wait > 0 ? wait : sm100::kWaitCycles);
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
  if (mp > kTcMaxPadded || d < 1 || d > (int64_t)1 << 31) return false;
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
                                 int* err, long long wait_cycles, cudaStream_t st) {
  if (nparts != dense_tc_tiles(d)) return cudaErrorInvalidValue;
  switch (mp) {
    case 4: return dense_tc_impl<4>(d, A, lda, mu, P, Y, ld, m, parts, nparts, state, pt, err, wait_cycles, st);
    case 8: return dense_tc_impl<8>(d, A, lda, mu, P, Y, ld, m, parts, nparts, state, pt, err, wait_cycles, st);
    case 16: return dense_tc_impl<16>(d, A, lda, mu, P, Y, ld, m, parts, nparts, state, pt, err, wait_cycles, st);
    case 24: return dense_tc_impl<24>(d, A, lda, mu, P, Y, ld, m, parts, nparts, state, pt, err, wait_cycles, st);
    case 36: return dense_tc_impl<36>(d, A, lda, mu, P, Y, ld, m, parts, nparts, state, pt, err, wait_cycles, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bk
