// FP64-accurate dense products Y = A X of FP32-stored values A (d x d, row-major) and
// an FP64 block X (d x N, column-major) on the BF16 tensor cores, by an error-free
// splitting in the manner of Ozaki, Ogita and Oishi (2012). This is the stored-K
// matrix-load of the sampling driver (Sec. 5), which needs its products accurate far
// beyond FP32 because an FP32 basis cannot resolve the spectrum near the nugget.
//
// Splitting. Each row of A and each column of X is cut into K blocks of KB = 512
// elements. A block with largest magnitude below 2^e is written as
//     v = 2^e sum_i a_i 2^-(6 + 7 i),  i = 0 .. ND - 1,
// with ND = 7 signed integer digits |a_i| <= 64 (each exact in BF16): a_0 rounds
// v 2^(6 - e) to the nearest integer and every later digit rounds what is left, so
// every value is kept to 2^-49 of its block's bound 2^e (FP32 values of A within
// 2^-25 of the bound exactly). Per K block, the product of the A digits of
// row r and the X digits of column c is
//     2^(e_A + e_X - 12) sum_s 2^-7s g_s,   g_s = sum_{i + j = s} sum_k a_i x_j,
// over s = i + j <= ND - 1 (28 digit pairs; the dropped pairs are below 2^-49 of
// the block's largest product). A digit product is an integer of magnitude at most
// 2^12, so g_s, a sum of at most 7 x 512 of them, is an integer below 2^24: the
// tensor core's FP32 accumulation forms it exactly, whatever its rounding. Each g_s
// has its own accumulator in tensor memory for the K block; at the end of a block the
// drain warps scale the seven integers by exact powers of two and add them into a
// running unevaluated FP32 pair (about 48 bits), which becomes FP64 at the end.
//
// k_ozgemm: persistent CTAs walk items (128-row tile of A, 64-column tile of X).
//   warp 0      TMA producer: per 64-wide K stage, the 7 X digit tiles (64 x 64) into
//               one of two X slots, then the 7 A digit tiles (128 x 64) into a ring
//               of A slots, digit by digit;
//   warp 1      tensor-memory allocation; lane 0 issues, per stage and A digit i, the
//               products with the X digits j <= ND - 1 - i into accumulator s = i + j
//               (M = 128, K = 16; the X digit tiles lie back to back and accumulator s
//               sits at column 64 s, so one MMA of N = 64 nn covers nn <= 4 consecutive
//               digits j: 10 MMAs per 16 of K instead of 28); at the end of a K block it
//               commits the seven accumulators to the drain;
//   warps 2-9   drain: tensor-memory lane quarter warp % 4 holds rows 32 (warp % 4) +
//               lane, and each warp takes 32 of the 64 columns; they add each K block
//               into the running pairs (released as soon as the accumulators are read)
//               and write Y.
// Every mbarrier wait is bounded (bk_sm100.cuh); a wait that gives up makes the kernel
// drain its own issued copies and MMAs, free tensor memory, set *err and return.
#include <cuda.h>
#include <cuda_bf16.h>

#include <climits>

#include "bk_common.cuh"
#include "bk_sm100.cuh"

namespace bk {
namespace {

using namespace sm100;

constexpr int kOzDigits = 7;             // digits per value (ND)
constexpr int kOzKB = 512;               // K block: one scale per row (column) and block
constexpr int kOzStagesPerBlock = kOzKB / 64;
constexpr int kOzNP = 64;                // columns of X per item
constexpr int kOzDrainWarps = 8;
constexpr int kOzThreads = 64 + 32 * kOzDrainWarps;
constexpr int kOzASlots = 6;             // ring of A digit tiles
constexpr int kOzBoxA = 128 * 128;       // bytes of a 128 x 64 BF16 box
constexpr int kOzBoxX = kOzNP * 128;     // bytes of a 64 x 64 BF16 box
constexpr int kOzXSlot = kOzDigits * kOzBoxX;
constexpr int kOzBar = 2 * kOzXSlot + kOzASlots * kOzBoxA;
constexpr int kOzSmem = kOzBar + 256 + 1024;
constexpr uint32_t kOzTmemCols = 512;    // 7 accumulators x 64 columns = 448 used
constexpr int kOzNoBlock = INT_MIN / 4;  // exponent of an all-zero block
static_assert(kOzSmem <= 232448, "shared memory per CTA");
static_assert(kOzDigits * kOzNP <= (int)kOzTmemCols, "accumulators in tensor memory");

// ---------------------------------------------------------------- digit split
// One warp per (row, K block): the block's largest magnitude gives e (|v| < 2^e), then
// the ND digits of every element. Row r, element k of the source is src[r ld + k]
// (r < R, k < Kd); the digits go to dig[(i Rpad + r) ldk + k] (rows R .. Rpad - 1 are
// written as zeros), the exponent to eblk[r nkb + kb] (kOzNoBlock for an all-zero
// block).
// The digits of one (row, K block) from the warp's values v[u] = element k0 + lane + 32 u.
template <typename T>
__device__ __forceinline__ void oz_digits(const T (&v)[kOzKB / 32], int lane, int64_t r, int64_t R, int64_t Rpad,
                                          int64_t Kd, int64_t kb, __nv_bfloat16* __restrict__ dig, int64_t ldk,
                                          int* __restrict__ eblk, int64_t nkb) {
  const int64_t k0 = kb * kOzKB;
  T amax = 0;
#pragma unroll
  for (int u = 0; u < kOzKB / 32; ++u) amax = fmax(amax, fabs(v[u]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  int e = 0;
  if (amax > 0) frexp(amax, &e);  // amax = f 2^e, f in [0.5, 1): |v| < 2^e
#pragma unroll
  for (int u = 0; u < kOzKB / 32; ++u) {
    const int64_t k = k0 + lane + 32 * u;
    if (k >= Kd) continue;
    T rem = amax > 0 ? ldexp(v[u], -e) : (T)0;  // in (-1, 1), exact
#pragma unroll
    for (int i = 0; i < kOzDigits; ++i) {
      const int sh = 6 + 7 * i;
      const T dgt = rint(ldexp(rem, sh));  // |dgt| <= 64
      rem = rem - ldexp(dgt, -sh);         // exact: what the digit leaves
      dig[((int64_t)i * Rpad + r) * ldk + k] = __float2bfloat16_rn((float)dgt);
    }
  }
  if (lane == 0 && r < R) eblk[r * nkb + kb] = amax > 0 ? e : kOzNoBlock;
}

// FP64 values by integer arithmetic (FP64 instructions run at 1/58 of the FP32 rate
// here): the block bound from the bit patterns (|v| orders like its pattern), then
// N = round(v 2^(48 - e)) from the mantissa by a rounding shift (|N| <= 2^48, so
// |v 2^-e - N 2^-48| <= 2^-49, the bound of the FP32 path), and balanced base-128
// digits of N from the bottom: a_i = ((N + 64) mod 128) - 64, N <- (N - a_i) / 128, with
// N = sum_i a_i 2^(42 - 7 i), i.e. v 2^-e ~= sum_i a_i 2^-(6 + 7 i), |a_i| <= 64.
template <>
__device__ __forceinline__ void oz_digits<double>(const double (&v)[kOzKB / 32], int lane, int64_t r, int64_t R,
                                                  int64_t Rpad, int64_t Kd, int64_t kb,
                                                  __nv_bfloat16* __restrict__ dig, int64_t ldk,
                                                  int* __restrict__ eblk, int64_t nkb) {
  const int64_t k0 = kb * kOzKB;
  unsigned long long amax = 0;
#pragma unroll
  for (int u = 0; u < kOzKB / 32; ++u) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v[u]) & 0x7fffffffffffffffull;
    amax = b > amax ? b : amax;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long x = __shfl_xor_sync(0xffffffffu, amax, o);
    amax = x > amax ? x : amax;
  }
  int e = 0;
  if (amax) frexp(__longlong_as_double((long long)amax), &e);  // |v| < 2^e
#pragma unroll
  for (int u = 0; u < kOzKB / 32; ++u) {
    const int64_t k = k0 + lane + 32 * u;
    if (k >= Kd) continue;
    const unsigned long long b = (unsigned long long)__double_as_longlong(v[u]);
    const int ev = (int)((b >> 52) & 0x7ff);
    unsigned long long mant = b & 0xfffffffffffffull;
    int E = -1074;  // value = mant 2^E
    if (ev) {
      mant |= 1ull << 52;
      E = ev - 1075;
    }
    const int sh = E + 48 - e;
    long long N;
    if (!amax || !mant)
      N = 0;
    else if (sh >= 0)
      N = (long long)(mant << sh);  // only for subnormal blocks; |N| < 2^48
    else if (-sh > 63)
      N = 0;
    else
      N = (long long)((mant + (1ull << (-sh - 1))) >> (-sh));
    if (b >> 63) N = -N;
    int a[kOzDigits];
#pragma unroll
    for (int i = kOzDigits - 1; i > 0; --i) {
      a[i] = (int)((N + 64) & 127) - 64;
      N = (N - a[i]) >> 7;
    }
    a[0] = (int)N;
#pragma unroll
    for (int i = 0; i < kOzDigits; ++i) dig[((int64_t)i * Rpad + r) * ldk + k] = __float2bfloat16_rn((float)a[i]);
  }
  if (lane == 0 && r < R) eblk[r * nkb + kb] = amax ? e : kOzNoBlock;
}

template <typename T>
__global__ void k_oz_split(int64_t R, int64_t Rpad, int64_t Kd, const T* __restrict__ src, int64_t ld,
                           __nv_bfloat16* __restrict__ dig, int64_t ldk, int* __restrict__ eblk, int64_t nkb) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < Rpad * nkb; w += nw) {
    const int64_t r = w / nkb, kb = w - r * nkb;
    const int64_t k0 = kb * kOzKB;
    T v[kOzKB / 32];
#pragma unroll
    for (int u = 0; u < kOzKB / 32; ++u) {
      const int64_t k = k0 + lane + 32 * u;
      v[u] = (r < R && k < Kd) ? src[r * ld + k] : (T)0;
    }
    oz_digits<T>(v, lane, r, R, Rpad, Kd, kb, dig, ldk, eblk, nkb);
  }
}

// The same split of the transposed source: element k of row r is src[k ld + r] (the
// columns of a row-major matrix). A block of 32 warps stages 32 rows x one K block
// through shared memory (coalesced reads along r), then warp w splits row r0 + w.
constexpr int kOzTRows = 32;
template <typename T>
__global__ void __launch_bounds__(1024) k_oz_split_t(int64_t R, int64_t Rpad, int64_t Kd, const T* __restrict__ src,
                                                     int64_t ld, __nv_bfloat16* __restrict__ dig, int64_t ldk,
                                                     int* __restrict__ eblk, int64_t nkb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);  // [kOzKB][kOzTRows + 1]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t rtiles = Rpad / kOzTRows;
  for (int64_t b = blockIdx.x; b < rtiles * nkb; b += gridDim.x) {
    const int64_t r0 = (b / nkb) * kOzTRows, kb = b % nkb, k0 = kb * kOzKB;
#pragma unroll
    for (int u = 0; u < kOzKB / 32; ++u) {
      const int kk = w + 32 * u;
      const int64_t r = r0 + lane, k = k0 + kk;
      tile[kk * (kOzTRows + 1) + lane] = (r < R && k < Kd) ? src[k * ld + r] : (T)0;
    }
    __syncthreads();
    T v[kOzKB / 32];
#pragma unroll
    for (int u = 0; u < kOzKB / 32; ++u) v[u] = tile[(lane + 32 * u) * (kOzTRows + 1) + w];
    oz_digits<T>(v, lane, r0 + w, R, Rpad, Kd, kb, dig, ldk, eblk, nkb);
    __syncthreads();
  }
}

// One warp per row: emax = the largest block exponent of the row (0 for an all-zero
// row) and erel = e - emax per block, written at erel[r rs + kb ks] (kOzNoBlock kept).
// Rows R .. Rpad - 1 (padding) are written as all-zero rows.
__global__ void k_oz_rel(int64_t R, int64_t Rpad, int64_t nkb, const int* __restrict__ eblk, int* __restrict__ erel,
                         int64_t rs, int64_t ks, int* __restrict__ emax) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < Rpad; r += nw) {
    int m = kOzNoBlock;
    if (r < R)
      for (int64_t kb = lane; kb < nkb; kb += 32) m = max(m, eblk[r * nkb + kb]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (m == kOzNoBlock) m = 0;
    for (int64_t kb = lane; kb < nkb; kb += 32) {
      const int e = r < R ? eblk[r * nkb + kb] : kOzNoBlock;
      erel[r * rs + kb * ks] = e == kOzNoBlock ? kOzNoBlock : e - m;
    }
    if (lane == 0) emax[r] = m;
  }
}

// ---------------------------------------------------------------- products
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum_f(float a, float b, float& s, float& e) {  // |a| >= |b|
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
// (ah, al) += (bh, bl), unevaluated FP32 pairs (about 2^-47 of the result)
__device__ __forceinline__ void pair_add(float& ah, float& al, float bh, float bl) {
  float s, e, t, f;
  two_sum_f(ah, bh, s, e);
  two_sum_f(al, bl, t, f);
  e = __fadd_rn(e, t);
  fast_two_sum_f(s, e, s, e);
  e = __fadd_rn(e, f);
  fast_two_sum_f(s, e, ah, al);
}
// 2^k as FP32 for -126 <= k <= 127
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

struct OzArgs {
  int64_t M, K;        // rows of A, K extent (columns of A = rows of X)
  int N;               // live columns of X and Y
  int64_t Rpad, Cpad;  // digit rows per plane (A, X)
  int64_t nkb;         // K blocks
  const int* ea_rel;   // [r nkb + kb]
  const int* ex_rel;   // [kb Cpad + c]
  const int* ea_max;   // [r]
  const int* ex_max;   // [c]
  double* Y;           // column-major, ldy; with nkc > 1 the partial of chunk kc starts at column kc N
  int64_t ldy;
  int64_t nkc, kbc;    // K chunks (split-K) and K blocks per chunk
  long long wait;
  int* err;
};

__global__ void __launch_bounds__(kOzThreads, 1)
    k_ozgemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapX, const OzArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* xbase = base;                    // 2 X slots
  uint8_t* abase = base + 2 * kOzXSlot;     // ring of A digit tiles
  uint64_t* xfull = reinterpret_cast<uint64_t*>(base + kOzBar);
  uint64_t* xempty = xfull + 2;
  uint64_t* afull = xempty + 2;
  uint64_t* aempty = afull + kOzASlots;
  uint64_t* accf = aempty + kOzASlots;
  uint64_t* acce = accf + 1;
  uint64_t* cleanup = acce + 1;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(cleanup + 1);
  volatile int* s_abort = reinterpret_cast<volatile int*>(tmem_holder + 1);
  volatile long long* s_cons_x = reinterpret_cast<volatile long long*>(base + kOzBar + 224);  // X stages seen by the MMA thread
  volatile long long* s_cons_a = s_cons_x + 1;                                                // A tiles seen
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t mtiles = a.Rpad / 128, ntiles = a.Cpad / kOzNP;
  const int64_t nks = (a.K + 63) / 64;
  const int64_t tiles = mtiles * ntiles;
  const int64_t items = tiles * a.nkc;
  // item it: K chunk it / tiles (its K blocks [kb0, kb1), stages [ks0, ks1)), then row
  // tile and column tile
  auto krange = [&](int64_t it, int64_t& kb0, int64_t& kb1, int64_t& ks0, int64_t& ks1) {
    kb0 = (it / tiles) * a.kbc;
    kb1 = kb0 + a.kbc < a.nkb ? kb0 + a.kbc : a.nkb;
    ks0 = kb0 * kOzStagesPerBlock;
    ks1 = kb1 * kOzStagesPerBlock < nks ? kb1 * kOzStagesPerBlock : nks;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(xfull + s, 1);
      mbar_init(xempty + s, 1);
    }
    for (int s = 0; s < kOzASlots; ++s) {
      mbar_init(afull + s, 1);
      mbar_init(aempty + s, 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, 32 * kOzDrainWarps);
    mbar_init(cleanup, 1);
    *s_abort = 0;
    *s_cons_x = 0;
    *s_cons_a = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tmem_holder, kOzTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  long long issued_x = 0, issued_a = 0;  // producer: copies issued
  if (warp == 0) {
    if (lane == 0) {
      tma_prefetch_desc(&mapA);
      tma_prefetch_desc(&mapX);
      long long gx = 0, ga = 0;
      for (int64_t it = blockIdx.x; it < items && !*s_abort; it += gridDim.x) {
        const int64_t mt = (it % tiles) / ntiles, nt = it % ntiles;
        int64_t kb0, kb1, ks0, ks1;
        krange(it, kb0, kb1, ks0, ks1);
        for (int64_t ks = ks0; ks < ks1 && !*s_abort; ++ks, ++gx) {
          const int xs = (int)(gx & 1);
          if (gx >= 2 && !mbar_wait(xempty + xs, (uint32_t)((gx >> 1) - 1) & 1, a.wait)) {
            *s_abort = 1;
            break;
          }
          mbar_arrive_expect_tx(xfull + xs, kOzXSlot);
          for (int j = 0; j < kOzDigits; ++j)
            tma_load_2d(xbase + xs * kOzXSlot + j * kOzBoxX, &mapX, xfull + xs, (int)(ks * 64),
                        (int)(j * a.Cpad + nt * kOzNP));
          issued_x = gx + 1;
          for (int i = 0; i < kOzDigits; ++i, ++ga) {
            const int as = (int)(ga % kOzASlots);
            if (ga >= kOzASlots && !mbar_wait(aempty + as, (uint32_t)((ga / kOzASlots) - 1) & 1, a.wait)) {
              *s_abort = 1;
              break;
            }
            mbar_arrive_expect_tx(afull + as, kOzBoxA);
            tma_load_2d(abase + as * kOzBoxA, &mapA, afull + as, (int)(ks * 64), (int)(i * a.Rpad + mt * 128));
            issued_a = ga + 1;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc1 = idesc_bf16(128, kOzNP), idesc2 = idesc_bf16(128, 2 * kOzNP);
      constexpr uint32_t idesc3 = idesc_bf16(128, 3 * kOzNP), idesc4 = idesc_bf16(128, 4 * kOzNP);
      long long gx = 0, ga = 0, per = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; it < items && ok && !*s_abort; it += gridDim.x) {
        int64_t kb0, kb1, ks0, ks1;
        krange(it, kb0, kb1, ks0, ks1);
        for (int64_t p0 = ks0; p0 < ks1 && ok && !*s_abort; p0 += kOzStagesPerBlock, ++per) {
          if (per >= 1 && !mbar_wait(acce, (uint32_t)(per - 1) & 1, a.wait)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int64_t p1 = p0 + kOzStagesPerBlock < ks1 ? p0 + kOzStagesPerBlock : ks1;
          for (int64_t ks = p0; ks < p1 && ok; ++ks, ++gx) {
            const int xs = (int)(gx & 1);
            if (!mbar_wait(xfull + xs, (uint32_t)(gx >> 1) & 1, a.wait)) {
              ok = false;
              break;
            }
            *s_cons_x = gx + 1;
            tc_fence_after();
            const uint32_t xa = smem_u32(xbase + xs * kOzXSlot);
            for (int i = 0; i < kOzDigits; ++i, ++ga) {
              const int as = (int)(ga % kOzASlots);
              if (!mbar_wait(afull + as, (uint32_t)(ga / kOzASlots) & 1, a.wait)) {
                ok = false;
                break;
              }
              *s_cons_a = ga + 1;
              tc_fence_after();
              const uint32_t aa = smem_u32(abase + as * kOzBoxA);
              // the X digit tiles lie back to back, so X digits j0 .. j0 + nn - 1 form one
              // B operand of 64 nn rows whose products land in accumulators i + j0 ..
              // i + j0 + nn - 1 (accumulator s at column 64 s): up to N = 256 per MMA
              for (int j0 = 0; i + j0 < kOzDigits; j0 += 4) {
                const int nn = kOzDigits - i - j0 < 4 ? kOzDigits - i - j0 : 4;
                const uint32_t acc = tmem + (uint32_t)((i + j0) * kOzNP);
                const uint32_t id = nn == 4 ? idesc4 : (nn == 3 ? idesc3 : (nn == 2 ? idesc2 : idesc1));
#pragma unroll
                for (int k = 0; k < 4; ++k)  // 16 BF16 of K = 32 bytes into the 128-byte rows
                  mma_bf16(acc, desc_kmajor_sw128(aa + 32u * k), desc_kmajor_sw128(xa + j0 * kOzBoxX + 32u * k), id,
                           (ks == p0 && i == 0 && k == 0) ? 0u : 1u);
              }
              mma_commit(aempty + as);
            }
            if (ok) mma_commit(xempty + xs);
          }
          if (ok) mma_commit(accf);
        }
      }
      if (!ok) *s_abort = 1;
    }
  } else {
    // warps 2-9: lane quarter warp % 4 (rows 32 (warp % 4) + lane), column half hf
    const int q = warp & 3, hf = (warp - 2) >> 2;
    const int row = 32 * q + lane;
    long long per = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
      if (__any_sync(0xffffffffu, *s_abort != 0)) break;
      const int64_t mt = (it % tiles) / ntiles, nt = it % ntiles;
      int64_t kb0, kb1, ks0, ks1;
      krange(it, kb0, kb1, ks0, ks1);
      const int64_t r = mt * 128 + row;
      const int64_t cbase = nt * kOzNP + hf * 32;
      float H[32], L[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) H[c] = L[c] = 0.f;
      for (int64_t kb = kb0; kb < kb1; ++kb, ++per) {
        if (!__all_sync(0xffffffffu, mbar_wait(accf, (uint32_t)per & 1, a.wait))) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int ea = r < a.M ? a.ea_rel[r * a.nkb + kb] : kOzNoBlock;
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(hf * 32);
#pragma unroll
        for (int c0 = 0; c0 < 32; c0 += 8) {
          uint32_t g[kOzDigits][8];
#pragma unroll
          for (int s = 0; s < kOzDigits; ++s) tmem_ld8(taddr + (uint32_t)(s * kOzNP + c0), g[s]);
          tmem_ld_wait();
          if (c0 == 24) {  // every accumulator read: the MMAs of the next block may start
            tc_fence_before();
            mbar_arrive(acce);
          }
#pragma unroll
          for (int cc = 0; cc < 8; ++cc) {
            const int ex = a.ex_rel[kb * a.Cpad + cbase + c0 + cc];
            const int sc = ea + ex;  // <= 0 unless a block is empty
            if (ea == kOzNoBlock || ex == kOzNoBlock || sc < -100) continue;
            // block value relative to 2^(sc): sum_s g_s 2^-7s (integers |g_s| < 2^24)
            float h = __uint_as_float(g[0][cc]), l = 0.f;
#pragma unroll
            for (int s = 1; s < kOzDigits; ++s) {
              float e;
              two_sum_f(h, __uint_as_float(g[s][cc]) * pow2f(-7 * s), h, e);
              l = __fadd_rn(l, e);
            }
            fast_two_sum_f(h, l, h, l);
            const float p2 = pow2f(sc);
            pair_add(H[c0 + cc], L[c0 + cc], h * p2, l * p2);
          }
        }
      }
      if (!ok) break;
      if (r < a.M) {
        const int eam = a.ea_max[r];
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int64_t col = cbase + c;
          if (col < a.N)
            a.Y[((it / tiles) * (a.nkc > 1 ? a.N : 0) + col) * a.ldy + r] =
                ldexp((double)H[c] + (double)L[c], eam + a.ex_max[col] - 12);
        }
      }
    }
    if (!ok) *s_abort = 1;
  }

  // ---- drain: every role has left its loop
  __syncthreads();
  if (*s_abort) {
    // issued copies land and issued MMAs complete before the memory is reused or freed;
    // these waits keep the default limit: they wait for work already issued
    if (warp == 0 && lane == 0) {
      for (long long g = *s_cons_x; g < issued_x; ++g) mbar_wait(xfull + (int)(g & 1), (uint32_t)(g >> 1) & 1);
      for (long long g = *s_cons_a; g < issued_a; ++g)
        mbar_wait(afull + (int)(g % kOzASlots), (uint32_t)(g / kOzASlots) & 1);
    }
    if (warp == 1 && lane == 0) {
      mma_commit(cleanup);
      mbar_wait(cleanup, 0);
    }
    if (threadIdx.x == 0 && a.err) atomicExch(a.err, 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, kOzTmemCols);
}

}  // namespace

// Y[c ldy + r] = sum over chunks of part[(kc N + c) M + r], chunks in order
__global__ void k_oz_sum(int64_t M, int N, int64_t nkc, const double* __restrict__ part, double* __restrict__ Y,
                         int64_t ldy) {
  const int64_t total = M * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = idx / M, r = idx - c * M;
    double s = 0.0;
    for (int64_t k = 0; k < nkc; ++k) s += part[(k * N + c) * M + r];
    Y[c * ldy + r] = s;
  }
}

// C = alpha Y + beta C (Y: M x N column-major, ld M; C: ldc); C is not read when beta = 0
__global__ void k_oz_axpby(int64_t M, int N, double alpha, const double* __restrict__ Y, double beta, double* C,
                           int64_t ldc) {
  const int64_t total = M * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = idx / M, r = idx - c * M;
    double* o = C + c * ldc + r;
    *o = beta == 0.0 ? alpha * Y[idx] : fma(alpha, Y[idx], beta * *o);
  }
}

// ---------------------------------------------------------------- host side
namespace {

int64_t oz_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }
size_t oz_al(size_t b) { return (b + 255) & ~size_t(255); }

// digits, block exponents, relative exponents and row maxima of an R x K operand
// (rows padded to Rpad) inside one buffer
struct OzOperand {
  int64_t R, Rpad, K, ldk, nkb;
  __nv_bfloat16* dig;
  int* eblk;
  int* erel;
  int* emax;
};
size_t oz_operand_bytes(int64_t Rpad, int64_t K) {
  const int64_t ldk = oz_up(K, 64), nkb = (K + kOzKB - 1) / kOzKB;
  return oz_al((size_t)kOzDigits * Rpad * ldk * 2) + 2 * oz_al((size_t)Rpad * nkb * 4) + oz_al((size_t)Rpad * 4);
}
OzOperand oz_operand(int64_t R, int64_t Rpad, int64_t K, void* buf) {
  OzOperand o;
  o.R = R;
  o.Rpad = Rpad;
  o.K = K;
  o.ldk = oz_up(K, 64);
  o.nkb = (K + kOzKB - 1) / kOzKB;
  char* p = static_cast<char*>(buf);
  o.dig = reinterpret_cast<__nv_bfloat16*>(p);
  p += oz_al((size_t)kOzDigits * Rpad * o.ldk * 2);
  o.eblk = reinterpret_cast<int*>(p);
  p += oz_al((size_t)Rpad * o.nkb * 4);
  o.erel = reinterpret_cast<int*>(p);
  p += oz_al((size_t)Rpad * o.nkb * 4);
  o.emax = reinterpret_cast<int*>(p);
  return o;
}
// the operand of the left factor (rows padded to 128) and of the right factor (to 64)
OzOperand oz_left(int64_t R, int64_t K, void* buf) { return oz_operand(R, oz_up(R, 128), K, buf); }
OzOperand oz_right(int64_t R, int64_t K, void* buf) { return oz_operand(R, oz_up(R, kOzNP), K, buf); }
size_t oz_left_bytes(int64_t R, int64_t K) { return oz_operand_bytes(oz_up(R, 128), K); }
size_t oz_right_bytes(int64_t R, int64_t K) { return oz_operand_bytes(oz_up(R, kOzNP), K); }

// Digits of a source whose row r, element k is src[r ld + k] (transposed: src[k ld + r]);
// relative exponents by row then block (left factor) or by block then row (right).
template <typename T>
cudaError_t oz_split(const OzOperand& o, const T* src, int64_t ld, bool transposed, bool right, int sms,
                     cudaStream_t st) {
  cudaError_t e;
  if (!transposed) {
    const int64_t warps = o.Rpad * o.nkb;
    int64_t grid = (warps + 7) / 8;
    if (grid > (int64_t)sms * 16) grid = (int64_t)sms * 16;
    k_oz_split<T><<<(int)grid, 256, 0, st>>>(o.R, o.Rpad, o.K, src, ld, o.dig, o.ldk, o.eblk, o.nkb);
  } else {
    const size_t smem = (size_t)kOzKB * (kOzTRows + 1) * sizeof(T);
    if ((e = cudaFuncSetAttribute(k_oz_split_t<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
      return e;
    int64_t grid = (o.Rpad / kOzTRows) * o.nkb;
    if (grid > (int64_t)sms * 4) grid = (int64_t)sms * 4;
    k_oz_split_t<T><<<(int)grid, 1024, smem, st>>>(o.R, o.Rpad, o.K, src, ld, o.dig, o.ldk, o.eblk, o.nkb);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int64_t g2 = (o.Rpad + 7) / 8;
  if (g2 > (int64_t)sms * 16) g2 = (int64_t)sms * 16;
  k_oz_rel<<<(int)g2, 256, 0, st>>>(o.R, o.Rpad, o.nkb, o.eblk, o.erel, right ? 1 : o.nkb, right ? o.Rpad : 1,
                                    o.emax);
  return cudaGetLastError();
}

// Split-K plan: with fewer output tiles than two per SM, items also cut K into chunks
// of whole K blocks (at least two per SM in all); the partials are summed in chunk order.
void oz_plan(int64_t M, int64_t N, int64_t K, int sms, int64_t* nkc, int64_t* kbc) {
  const int64_t tiles = (oz_up(M, 128) / 128) * (oz_up(N, kOzNP) / kOzNP);
  const int64_t nkb = (K + kOzKB - 1) / kOzKB;
  int64_t want = tiles >= 2 * (int64_t)sms ? 1 : (2 * (int64_t)sms + tiles - 1) / tiles;
  if (want > nkb) want = nkb;
  if (want < 1) want = 1;
  *kbc = (nkb + want - 1) / want;
  *nkc = (nkb + *kbc - 1) / *kbc;
}
size_t oz_part_bytes(int64_t M, int64_t N, int64_t K, int sms) {
  int64_t nkc, kbc;
  oz_plan(M, N, K, sms, &nkc, &kbc);
  return nkc > 1 ? oz_al((size_t)nkc * N * M * 8) : 0;
}

// Y (A.R x X.R, column-major ldy) = A X^T over the common K; part holds
// oz_part_bytes(A.R, X.R, K, sms) for the split-K partials
cudaError_t oz_gemm(const OzOperand& A, const OzOperand& X, double* Y, int64_t ldy, double* part,
                    long long wait_cycles, int* err, int sms, cudaStream_t st) {
  if (A.K != X.K) return cudaErrorInvalidValue;
  CUtensorMap ma, mx;
  cudaError_t e;
  if ((e = make_map_bf16(&ma, A.dig, A.K, (int64_t)kOzDigits * A.Rpad, A.ldk, 128)) != cudaSuccess) return e;
  if ((e = make_map_bf16(&mx, X.dig, X.K, (int64_t)kOzDigits * X.Rpad, X.ldk, kOzNP)) != cudaSuccess) return e;
  OzArgs args;
  args.M = A.R;
  args.K = A.K;
  args.N = (int)X.R;
  args.Rpad = A.Rpad;
  args.Cpad = X.Rpad;
  args.nkb = A.nkb;
  args.ea_rel = A.erel;
  args.ex_rel = X.erel;
  args.ea_max = A.emax;
  args.ex_max = X.emax;
  oz_plan(A.R, X.R, A.K, sms, &args.nkc, &args.kbc);
  if (args.nkc > 1 && !part) return cudaErrorInvalidValue;
  args.Y = args.nkc > 1 ? part : Y;
  args.ldy = args.nkc > 1 ? A.R : ldy;
  args.wait = wait_cycles > 0 ? wait_cycles : kWaitCycles;
  args.err = err;
  if ((e = cudaFuncSetAttribute(k_ozgemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem)) != cudaSuccess)
    return e;
  const int64_t items = (A.Rpad / 128) * (X.Rpad / kOzNP) * args.nkc;
  const int grid = (int)(items < sms ? items : sms);
  k_ozgemm<<<grid, kOzThreads, kOzSmem, st>>>(ma, mx, args);
  if ((e = cudaGetLastError()) != cudaSuccess || args.nkc == 1) return e;
  const int64_t total = A.R * X.R;
  int64_t g = (total + 255) / 256;
  if (g > (int64_t)sms * 8) g = (int64_t)sms * 8;
  k_oz_sum<<<(int)g, 256, 0, st>>>(A.R, (int)X.R, args.nkc, part, Y, ldy);
  return cudaGetLastError();
}

}  // namespace

bool ozaki_usable(int64_t d, int N) {
  // TMA coordinates are 32-bit: the digit planes of the left factor stack 7 x Rpad rows
  return d >= 1 && N >= 1 && N <= 4096 && (int64_t)kOzDigits * oz_up(d, 128) < ((int64_t)1 << 31);
}
size_t ozaki_a_bytes(int64_t d) { return oz_left_bytes(d, d); }
size_t ozaki_x_bytes(int64_t d, int N, int sms) { return oz_al(oz_right_bytes(N, d)) + oz_part_bytes(d, N, d, sms); }

cudaError_t launch_ozaki_split_a(int64_t d, const float* A, int64_t lda, void* abuf, int sms, cudaStream_t st) {
  return oz_split<float>(oz_left(d, d, abuf), A, lda, false, false, sms, st);
}

cudaError_t launch_ozaki_apply(int64_t d, int N, const void* abuf, const double* X, int64_t ldx, double* Y,
                               int64_t ldy, void* xbuf, long long wait_cycles, int* err, int sms, cudaStream_t st) {
  if (!ozaki_usable(d, N)) return cudaErrorInvalidValue;
  const OzOperand oa = oz_left(d, d, const_cast<void*>(abuf));
  const OzOperand ox = oz_right(N, d, xbuf);
  double* part = reinterpret_cast<double*>(static_cast<char*>(xbuf) + oz_al(oz_right_bytes(N, d)));
  // column c of X is row c of the right factor (elements X[c ldx + k])
  cudaError_t e = oz_split<double>(ox, X, ldx, false, true, sms, st);
  if (e != cudaSuccess) return e;
  return oz_gemm(oa, ox, Y, ldy, part, wait_cycles, err, sms, st);
}

// Gram form A = Z^T Z (Z: n x d row-major): the digits of Z (rows of Z) and of Z^T
// (columns of Z), made once per operator.
bool ozaki_gram_usable(int64_t n, int64_t d, int N) { return ozaki_usable(n, N) && ozaki_usable(d, N); }
size_t ozaki_gram_bytes(int64_t n, int64_t d) { return oz_al(oz_left_bytes(n, d)) + oz_left_bytes(d, n); }
size_t oz_gram_part_bytes(int64_t n, int64_t d, int N, int sms) {
  const size_t a = oz_part_bytes(n, N, d, sms), b = oz_part_bytes(d, N, n, sms);
  return a > b ? a : b;
}
size_t ozaki_gram_work_bytes(int64_t n, int64_t d, int N, int sms) {
  return oz_al(oz_right_bytes(N, d)) + oz_al(oz_right_bytes(N, n)) + oz_al((size_t)n * N * 8) +
         oz_gram_part_bytes(n, d, N, sms);
}

cudaError_t launch_ozaki_split_gram(int64_t n, int64_t d, int z_f64, const void* Z, int64_t ldz, void* zbuf, int sms,
                                    cudaStream_t st) {
  const OzOperand oz = oz_left(n, d, zbuf);
  const OzOperand ot = oz_left(d, n, static_cast<char*>(zbuf) + oz_al(oz_left_bytes(n, d)));
  cudaError_t e = z_f64 ? oz_split<double>(oz, (const double*)Z, ldz, false, false, sms, st)
                        : oz_split<float>(oz, (const float*)Z, ldz, false, false, sms, st);
  if (e != cudaSuccess) return e;
  return z_f64 ? oz_split<double>(ot, (const double*)Z, ldz, true, false, sms, st)
               : oz_split<float>(ot, (const float*)Z, ldz, true, false, sms, st);
}

cudaError_t launch_ozaki_gram_apply(int64_t n, int64_t d, int N, const void* zbuf, const double* X, int64_t ldx,
                                    double* Y, int64_t ldy, void* work, long long wait_cycles, int* err, int sms,
                                    cudaStream_t st) {
  if (!ozaki_gram_usable(n, d, N)) return cudaErrorInvalidValue;
  char* zb = static_cast<char*>(const_cast<void*>(zbuf));
  const OzOperand oz = oz_left(n, d, zb);
  const OzOperand ot = oz_left(d, n, zb + oz_al(oz_left_bytes(n, d)));
  char* w = static_cast<char*>(work);
  const OzOperand ox = oz_right(N, d, w);
  w += oz_al(oz_right_bytes(N, d));
  const OzOperand ov = oz_right(N, n, w);
  w += oz_al(oz_right_bytes(N, n));
  double* V = reinterpret_cast<double*>(w);  // n x N column-major
  w += oz_al((size_t)n * N * 8);
  double* part = reinterpret_cast<double*>(w);
  cudaError_t e = oz_split<double>(ox, X, ldx, false, true, sms, st);
  if (e == cudaSuccess) e = oz_gemm(oz, ox, V, n, part, wait_cycles, err, sms, st);      // V = Z X
  if (e == cudaSuccess) e = oz_split<double>(ov, V, n, false, true, sms, st);
  if (e == cudaSuccess) e = oz_gemm(ot, ov, Y, ldy, part, wait_cycles, err, sms, st);    // Y = Z^T V
  return e;
}

// General FP64 product C = alpha A B + beta C (A: M x K with element (i, k) at
// A[i sai + k sak], B: K x N with element (k, j) at B[k sbk + j sbj]) through the Ozaki
// split; each operand must be contiguous along K (sak = 1, sbk = 1) or along the other
// index (sai = 1, sbj = 1: the transposed split).
bool ozaki_gemm_usable(int64_t M, int64_t N, int64_t K, int64_t sai, int64_t sak, int64_t sbk, int64_t sbj) {
  return M >= 1 && N >= 1 && N <= 4096 && K >= 1 && (sak == 1 || sai == 1) && (sbk == 1 || sbj == 1) &&
         (int64_t)kOzDigits * oz_up(M, 128) < ((int64_t)1 << 31);
}
size_t ozaki_gemm_work_bytes(int64_t M, int64_t N, int64_t K, int sms) {
  return oz_al(oz_left_bytes(M, K)) + oz_al(oz_right_bytes(N, K)) + oz_part_bytes(M, N, K, sms) +
         oz_al((size_t)M * N * 8);
}
cudaError_t launch_ozaki_gemm(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t sai,
                              int64_t sak, const double* B, int64_t sbk, int64_t sbj, double beta, double* C,
                              int64_t ldc, void* work, long long wait_cycles, int* err, int sms, cudaStream_t st) {
  if (!ozaki_gemm_usable(M, N, K, sai, sak, sbk, sbj)) return cudaErrorInvalidValue;
  char* w = static_cast<char*>(work);
  const OzOperand oa = oz_left(M, K, w);
  w += oz_al(oz_left_bytes(M, K));
  const OzOperand ob = oz_right(N, K, w);
  w += oz_al(oz_right_bytes(N, K));
  double* part = reinterpret_cast<double*>(w);
  w += oz_part_bytes(M, N, K, sms);
  double* Y = reinterpret_cast<double*>(w);  // M x N column-major
  cudaError_t e = sak == 1 ? oz_split<double>(oa, A, sai, false, false, sms, st)
                           : oz_split<double>(oa, A, sak, true, false, sms, st);
  if (e == cudaSuccess)
    e = sbk == 1 ? oz_split<double>(ob, B, sbj, false, true, sms, st)
                 : oz_split<double>(ob, B, sbk, true, true, sms, st);
  if (e == cudaSuccess) e = oz_gemm(oa, ob, Y, M, part, wait_cycles, err, sms, st);
  if (e != cudaSuccess) return e;
  int64_t g = (M * N + 255) / 256;
  if (g > (int64_t)sms * 8) g = (int64_t)sms * 8;
  k_oz_axpby<<<(int)g, 256, 0, st>>>(M, (int)N, alpha, Y, beta, C, ldc);
  return cudaGetLastError();
}

}  // namespace bk
