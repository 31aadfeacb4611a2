// BF16 tensor-core products of the Gram-form operator A = Z^T Z (the ridge problem of
// Sec. 1, applied matrix-free; one matrix-load per product, Sec. 1.2): Y = Z^T (Z X)
// for a block X of up to 128 columns, FP32 in and out, on tcgen05 with FP32
// accumulation in tensor memory.
//
// Z (FP32, n x d row-major) is split once per call into a BF16 head and tail
// (z = zh + zl + e, |e| <= 2^-18 |z|) and stored twice: row-major (n x d) for V = Z X,
// transposed (d x n) for Y = Z^T V. Both products then read only K-major operands:
// rows of 64 BF16 (128 bytes) brought in by TMA boxes with the 128-byte swizzle. The
// block operand is split the same way at each product. A product is the sum of the
// three BF16 products Ah Bh + Ah Bl + Al Bh; the dropped Al Bl is below 2^-17
// relative, so the operator is applied to about 2^-16 of sum |z_ik x_k| (against
// 2^-8 for a single BF16 product), and the FP64 refinement residual of the ridge
// path keeps the result FP64-accurate.
//
// k_bgemm: C (M x NP) = A (M x K) B^T, B given as NP x K. Persistent CTAs walk work
// items: 128-row tiles of M (the second product also cuts K into chunks, split-K).
//   warp 0      TMA producer: stages of A head/tail (128 x 64) and B head/tail
//               (NP x 64) into a ring of kStages;
//   warp 1      tensor-memory allocation; lane 0 issues the MMAs (M = 128, N = NP,
//               K = 16 each, 12 per stage) into one of two accumulators, switching
//               every kDrain stages;
//   warps 2-5   drain each accumulator into FP32 registers (the tensor core's FP32
//               accumulation is not round-to-nearest, so at most kDrain x 64 K
//               elements are summed there), then write the item: the BF16 head and
//               tail of V^T (first product) or an FP32 partial of the K chunk
//               (second product), which k_bsum adds in a fixed chunk order.
// Every mbarrier wait is bounded (bk_sm100.cuh); a wait that gives up makes the
// kernel drain its own issued copies and MMAs, free tensor memory, set *err and
// return, and the caller reports BK_TIMEOUT.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "bk_common.cuh"
#include "bk_sm100.cuh"

namespace bk {
namespace {

using namespace sm100;

constexpr int kBgThreads = 192;
constexpr int kDrain = 16;  // stages (x 64 K elements) summed in one accumulator
constexpr int kBoxA = 128 * 128;  // bytes of a 128 x 64 BF16 box

template <int NP>
struct BgShape {
  static constexpr int kBoxB = NP * 128;                        // NP x 64 BF16
  static constexpr int kStage = 2 * kBoxA + 2 * kBoxB;          // A head, A tail, B head, B tail
  static constexpr int kStages = (220 * 1024) / kStage > 4 ? 4 : (220 * 1024) / kStage;
  static constexpr int kBar = kStages * kStage;
  static constexpr int kSmem = kBar + 256 + 1024;               // + barriers, + alignment slack
  static constexpr uint32_t kTmemCols = 2 * NP <= 32 ? 32 : (2 * NP <= 64 ? 64 : (2 * NP <= 128 ? 128 : 256));
  static_assert(NP % 16 == 0 && NP >= 16 && NP <= 128, "N of a BF16 MMA with M = 128");
  static_assert(kBoxB % 1024 == 0, "operand boxes stay on 1024-byte boundaries");
  static_assert(kStages >= 2 && kSmem <= 232448, "shared memory per CTA");
};

struct BgArgs {
  int64_t M, K;       // rows of A, K extent
  int64_t kchunk;     // K elements per work item (multiple of 64)
  int64_t nkc;        // K chunks: items = ceil(M / 128) * nkc
  int N;              // live columns of the result (<= NP)
  int mode;           // 0: write V^T head/tail (BF16); 1: write FP32 partials
  __nv_bfloat16* vth;  // mode 0: NP x ldv, row c = column c of the result
  __nv_bfloat16* vtl;
  int64_t ldv;
  float* part;        // mode 1: part[(chunk * NP + c) * ldp + row]
  int64_t ldp;
  long long wait;     // limit of each pipeline wait (SM clocks)
  int* err;
};

template <int NP>
__global__ void __launch_bounds__(kBgThreads, 1)
    k_bgemm(const __grid_constant__ CUtensorMap mah, const __grid_constant__ CUtensorMap mal,
            const __grid_constant__ CUtensorMap mbh, const __grid_constant__ CUtensorMap mbl, const BgArgs a) {
  using SH = BgShape<NP>;
  constexpr int S = SH::kStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(base + SH::kBar);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;   // [2]
  uint64_t* acce = accf + 2;    // [2]
  uint64_t* cleanup = acce + 2;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(cleanup + 1);
  volatile int* s_abort = reinterpret_cast<volatile int*>(tmem_holder + 1);
  volatile int* s_consumed = s_abort + 1;  // stages whose data the MMA thread has seen
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t mtiles = (a.M + 127) / 128;
  const int64_t items = mtiles * a.nkc;
  const int64_t ksl_total = (a.K + 63) / 64;  // 64-wide K slices of the whole K range
  const int64_t ksl_chunk = a.kchunk / 64;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf + b, 1);
      mbar_init(acce + b, 128);
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

  // the K slices [ks0, ks1) of item it
  auto slices = [&](int64_t it, int64_t& ks0, int64_t& ks1) {
    const int64_t kc = it % a.nkc;
    ks0 = kc * ksl_chunk;
    ks1 = ks0 + ksl_chunk < ksl_total ? ks0 + ksl_chunk : ksl_total;
  };

  int64_t issued = 0;  // producer: stages issued
  if (warp == 0) {
    if (lane == 0) {
      tma_prefetch_desc(&mah);
      tma_prefetch_desc(&mal);
      tma_prefetch_desc(&mbh);
      tma_prefetch_desc(&mbl);
      int64_t g = 0;
      for (int64_t it = blockIdx.x; it < items && !*s_abort; it += gridDim.x) {
        const int64_t mt = it / a.nkc;
        int64_t ks0, ks1;
        slices(it, ks0, ks1);
        for (int64_t ks = ks0; ks < ks1; ++ks, ++g) {
          const int s = (int)(g % S);
          if (*s_abort) break;
          if (g >= S && !mbar_wait(empty + s, (uint32_t)((g / S) - 1) & 1, a.wait)) {
            *s_abort = 1;
            break;
          }
          uint8_t* st = base + (size_t)s * SH::kStage;
          mbar_arrive_expect_tx(full + s, SH::kStage);
          const int x = (int)(ks * 64);
          tma_load_2d(st, &mah, full + s, x, (int)(mt * 128));
          tma_load_2d(st + kBoxA, &mal, full + s, x, (int)(mt * 128));
          tma_load_2d(st + 2 * kBoxA, &mbh, full + s, x, 0);
          tma_load_2d(st + 2 * kBoxA + SH::kBoxB, &mbl, full + s, x, 0);
          issued = g + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(128, NP);
      int64_t g = 0, grp = 0;
      for (int64_t it = blockIdx.x; it < items && !*s_abort; it += gridDim.x) {
        int64_t ks0, ks1;
        slices(it, ks0, ks1);
        for (int64_t k0 = ks0; k0 < ks1 && !*s_abort; k0 += kDrain, ++grp) {
          const int b = (int)(grp & 1);
          if (grp >= 2 && !mbar_wait(acce + b, (uint32_t)((grp >> 1) - 1) & 1, a.wait)) {
            *s_abort = 1;
            break;
          }
          tc_fence_after();
          const uint32_t acc = tmem + (uint32_t)(NP * b);
          const int64_t k1 = k0 + kDrain < ks1 ? k0 + kDrain : ks1;
          bool ok = true;
          for (int64_t ks = k0; ks < k1; ++ks, ++g) {
            const int s = (int)(g % S);
            if (!mbar_wait(full + s, (uint32_t)(g / S) & 1, a.wait)) {
              ok = false;
              break;
            }
            *s_consumed = (int)(g + 1);
            tc_fence_after();
            const uint32_t sa = smem_u32(base + (size_t)s * SH::kStage);
            const uint32_t sb = sa + 2 * kBoxA;
#pragma unroll
            for (int k = 0; k < 4; ++k) {  // 16 BF16 of K = 32 bytes into the 128-byte rows
              const uint64_t ah = desc_kmajor_sw128(sa + 32u * k);
              const uint64_t al = desc_kmajor_sw128(sa + kBoxA + 32u * k);
              const uint64_t bh = desc_kmajor_sw128(sb + 32u * k);
              const uint64_t bl = desc_kmajor_sw128(sb + SH::kBoxB + 32u * k);
              mma_bf16(acc, ah, bh, idesc, (ks != k0 || k != 0) ? 1u : 0u);
              mma_bf16(acc, ah, bl, idesc, 1u);
              mma_bf16(acc, al, bh, idesc, 1u);
            }
            mma_commit(empty + s);
          }
          if (!ok) {
            *s_abort = 1;
            break;
          }
          mma_commit(accf + b);
        }
      }
    }
  } else {
    // warps 2-5: tensor-memory lane quarter (warp % 4) holds rows 32 (warp % 4) + lane
    const int q = warp & 3;
    const int row = 32 * q + lane;
    int64_t grp = 0;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
      if (__any_sync(0xffffffffu, *s_abort != 0)) break;
      const int64_t mt = it / a.nkc, kc = it % a.nkc;
      int64_t ks0, ks1;
      slices(it, ks0, ks1);
      float sum[NP];
#pragma unroll
      for (int c = 0; c < NP; ++c) sum[c] = 0.f;
      bool ok = true;
      for (int64_t k0 = ks0; k0 < ks1; k0 += kDrain, ++grp) {
        const int b = (int)(grp & 1);
        if (!__all_sync(0xffffffffu, mbar_wait(accf + b, (uint32_t)(grp >> 1) & 1, a.wait))) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t addr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(NP * b);
#pragma unroll
        for (int c0 = 0; c0 < NP; c0 += 16) {
          uint32_t r[16];
          tmem_ld16(addr + (uint32_t)c0, r);
          tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 16; ++j) sum[c0 + j] += __uint_as_float(r[j]);
        }
        tc_fence_before();
        mbar_arrive(acce + b);
      }
      if (!ok) {
        *s_abort = 1;
        break;
      }
      const int64_t r = mt * 128 + row;
      if (r < a.M) {
        if (a.mode == 0) {
#pragma unroll
          for (int c = 0; c < NP; ++c) {
            const float v = c < a.N ? sum[c] : 0.f;
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
            a.vth[(int64_t)c * a.ldv + r] = h;
            a.vtl[(int64_t)c * a.ldv + r] = l;
          }
        } else {
#pragma unroll
          for (int c = 0; c < NP; ++c)
            if (c < a.N) a.part[((int64_t)kc * NP + c) * a.ldp + r] = sum[c];
        }
      }
    }
  }

  // ---- drain: every role has left its loop
  __syncthreads();
  if (*s_abort) {
    // issued copies land and issued MMAs complete before the memory is reused or freed;
    // these waits keep the default limit: they wait for work already issued
    if (warp == 0 && lane == 0)
      for (int64_t g = *s_consumed; g < issued; ++g) mbar_wait(full + (int)(g % S), (uint32_t)(g / S) & 1);
    if (warp == 1 && lane == 0) {
      mma_commit(cleanup);
      mbar_wait(cleanup, 0);
    }
    if (threadIdx.x == 0 && a.err) atomicExch(a.err, 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, SH::kTmemCols);
}

// Y[r + c ldy] = alpha sum_chunk part[(chunk NP + c) ldp + r] + beta Y (fixed chunk order)
__global__ void k_bsum(int64_t d, int N, int NP, int64_t nkc, const float* __restrict__ part, int64_t ldp,
                       double alpha, double beta, float* Y, int64_t ldy) {
  const int64_t total = d * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = idx / d, r = idx - c * d;
    float s = 0.f;
    for (int64_t k = 0; k < nkc; ++k) s += part[(k * NP + c) * ldp + r];
    float* y = Y + c * ldy + r;
    *y = beta == 0.0 ? (float)(alpha * s) : (float)(alpha * s + beta * (double)*y);
  }
}

// Z (FP32, n x d row-major, ldz) -> head/tail BF16, row-major (n x ldk) and transposed
// (d x ldn), through 32 x 32 shared-memory tiles.
__global__ void k_zsplit(int64_t n, int64_t d, const float* __restrict__ Z, int64_t ldz, __nv_bfloat16* zh,
                         __nv_bfloat16* zl, int64_t ldk, __nv_bfloat16* th, __nv_bfloat16* tl, int64_t ldn) {
  __shared__ __nv_bfloat16 sh[32][33], sl[32][33];
  const int64_t tr = (n + 31) / 32, tc = (d + 31) / 32;
  for (int64_t t = blockIdx.x; t < tr * tc; t += gridDim.x) {
    const int64_t i0 = (t / tc) * 32, k0 = (t % tc) * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
      const int64_t i = i0 + y, k = k0 + threadIdx.x;
      __nv_bfloat16 h = __float2bfloat16_rn(0.f), l = h;
      if (i < n && k < d) {
        const float z = Z[i * ldz + k];
        h = __float2bfloat16_rn(z);
        l = __float2bfloat16_rn(z - __bfloat162float(h));
        zh[i * ldk + k] = h;
        zl[i * ldk + k] = l;
      }
      sh[y][threadIdx.x] = h;
      sl[y][threadIdx.x] = l;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
      const int64_t k = k0 + y, i = i0 + threadIdx.x;
      if (k < d && i < n) {
        th[k * ldn + i] = sh[threadIdx.x][y];
        tl[k * ldn + i] = sl[threadIdx.x][y];
      }
    }
    __syncthreads();
  }
}

// X (FP32, d x N column-major, ldx) -> X^T head/tail BF16 (NP x ldk), rows N..NP-1 zero.
__global__ void k_xsplit(int64_t d, int N, int NP, const float* __restrict__ X, int64_t ldx, __nv_bfloat16* xh,
                         __nv_bfloat16* xl, int64_t ldk) {
  const int64_t total = (int64_t)NP * d;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = idx / d, k = idx - c * d;
    const float v = c < N ? X[c * ldx + k] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    xh[c * ldk + k] = h;
    xl[c * ldk + k] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

}  // namespace

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 encode_bf16_fn() {
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

// 2D BF16 tensor (inner extent x, outer extent y, row pitch in elements) read in boxes
// of 64 x box_y with the 128-byte swizzle; elements outside the tensor read as zero.
cudaError_t make_map_bf16(CUtensorMap* map, const void* ptr, int64_t x, int64_t y, int64_t pitch, int box_y) {
  auto fn = encode_bf16_fn();
  if (!fn) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)x, (cuuint64_t)y};
  cuuint64_t strides[1] = {(cuuint64_t)pitch * 2};
  cuuint32_t box[2] = {64u, (cuuint32_t)box_y};
  cuuint32_t estr[2] = {1u, 1u};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

namespace {

int64_t up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// the BF16 copies inside the caller's buffer
struct ZCopies {
  __nv_bfloat16 *zh, *zl, *th, *tl;
  int64_t ldk, ldn;
};
ZCopies zcopies(int64_t n, int64_t d, const void* buf) {
  ZCopies z;
  z.ldk = up(d, 64);
  z.ldn = up(n, 64);
  __nv_bfloat16* p = static_cast<__nv_bfloat16*>(const_cast<void*>(buf));
  z.zh = p;
  z.zl = z.zh + (size_t)n * z.ldk;
  z.th = z.zl + (size_t)n * z.ldk;
  z.tl = z.th + (size_t)d * z.ldn;
  return z;
}

int np_of(int N) { return (int)up(N, 16); }

template <int NP>
cudaError_t bgemm_impl(const CUtensorMap& ah, const CUtensorMap& al, const CUtensorMap& bh, const CUtensorMap& bl,
                       const BgArgs& args, int grid, cudaStream_t st) {
  using SH = BgShape<NP>;
  auto k = k_bgemm<NP>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SH::kSmem);
  if (e != cudaSuccess) return e;
  k<<<grid, kBgThreads, SH::kSmem, st>>>(ah, al, bh, bl, args);
  return cudaGetLastError();
}

cudaError_t bgemm(int NP, const CUtensorMap& ah, const CUtensorMap& al, const CUtensorMap& bh, const CUtensorMap& bl,
                  const BgArgs& args, int grid, cudaStream_t st) {
  switch (NP) {
    case 16: return bgemm_impl<16>(ah, al, bh, bl, args, grid, st);
    case 32: return bgemm_impl<32>(ah, al, bh, bl, args, grid, st);
    case 48: return bgemm_impl<48>(ah, al, bh, bl, args, grid, st);
    case 64: return bgemm_impl<64>(ah, al, bh, bl, args, grid, st);
    case 80: return bgemm_impl<80>(ah, al, bh, bl, args, grid, st);
    case 96: return bgemm_impl<96>(ah, al, bh, bl, args, grid, st);
    case 112: return bgemm_impl<112>(ah, al, bh, bl, args, grid, st);
    case 128: return bgemm_impl<128>(ah, al, bh, bl, args, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

// K chunks of the second product: enough items for two per SM, chunks of whole slices
void plan_chunks(int64_t n, int64_t d, int sms, int64_t* kchunk, int64_t* nkc) {
  const int64_t mtiles = (d + 127) / 128, slices = (n + 63) / 64;
  int64_t want = (2 * (int64_t)sms + mtiles - 1) / mtiles;
  if (want < 1) want = 1;
  if (want > slices) want = slices;
  const int64_t per = (slices + want - 1) / want;
  *kchunk = per * 64;
  *nkc = (slices + per - 1) / per;
}

}  // namespace

bool bf16_gram_usable(int64_t n, int64_t d, int N) {
  return n >= 1 && d >= 1 && N >= 1 && N <= 128 && n < ((int64_t)1 << 31) && d < ((int64_t)1 << 31) &&
         encode_bf16_fn() != nullptr;
}

size_t bf16_gram_copy_bytes(int64_t n, int64_t d) {
  return (size_t)2 * 2 * ((size_t)n * up(d, 64) + (size_t)d * up(n, 64)) + 256;
}

size_t bf16_gram_work_bytes(int64_t n, int64_t d, int N, int sms) {
  const int NP = np_of(N);
  int64_t kchunk, nkc;
  plan_chunks(n, d, sms, &kchunk, &nkc);
  return (size_t)2 * 2 * NP * (up(d, 64) + up(n, 64))  // X^T and V^T head/tail
         + (size_t)4 * nkc * NP * up(d, 4)              // FP32 partials
         + 1024;
}

cudaError_t launch_bf16_gram_split(int64_t n, int64_t d, const float* Z, int64_t ldz, void* buf, cudaStream_t st) {
  ZCopies z = zcopies(n, d, buf);
  const int64_t tiles = ((n + 31) / 32) * ((d + 31) / 32);
  const int grid = (int)(tiles < 152 * 16 ? tiles : 152 * 16);
  k_zsplit<<<grid, dim3(32, 8), 0, st>>>(n, d, Z, ldz, z.zh, z.zl, z.ldk, z.th, z.tl, z.ldn);
  return cudaGetLastError();
}

cudaError_t launch_bf16_gram_apply(int64_t n, int64_t d, int N, const void* buf, const float* X, int64_t ldx, float* Y,
                                   int64_t ldy, double alpha, double beta, void* work, size_t work_bytes,
                                   long long wait_cycles, int* err, int sms, cudaStream_t st) {
  if (!bf16_gram_usable(n, d, N) || work_bytes < bf16_gram_work_bytes(n, d, N, sms)) return cudaErrorInvalidValue;
  const int NP = np_of(N);
  ZCopies z = zcopies(n, d, buf);
  int64_t kchunk, nkc;
  plan_chunks(n, d, sms, &kchunk, &nkc);
  __nv_bfloat16* xh = static_cast<__nv_bfloat16*>(work);
  __nv_bfloat16* xl = xh + (size_t)NP * z.ldk;
  __nv_bfloat16* vh = xl + (size_t)NP * z.ldk;
  __nv_bfloat16* vl = vh + (size_t)NP * z.ldn;
  float* part = reinterpret_cast<float*>(
      (reinterpret_cast<uintptr_t>(vl + (size_t)NP * z.ldn) + 255) & ~uintptr_t(255));
  const int64_t ldp = up(d, 4);
  const long long wait = wait_cycles > 0 ? wait_cycles : sm100::kWaitCycles;
  cudaError_t e;
  {
    const int64_t total = (int64_t)NP * d;
    const int g = (int)((total + 255) / 256 < 152 * 8 ? (total + 255) / 256 : 152 * 8);
    k_xsplit<<<g, 256, 0, st>>>(d, N, NP, X, ldx, xh, xl, z.ldk);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // V^T = (Z X)^T: A = Z (n x d), B = X^T (NP x d), all of K = d in one item
  CUtensorMap ah, al, bh, bl;
  if ((e = make_map_bf16(&ah, z.zh, d, n, z.ldk, 128)) != cudaSuccess) return e;
  if ((e = make_map_bf16(&al, z.zl, d, n, z.ldk, 128)) != cudaSuccess) return e;
  if ((e = make_map_bf16(&bh, xh, d, NP, z.ldk, NP)) != cudaSuccess) return e;
  if ((e = make_map_bf16(&bl, xl, d, NP, z.ldk, NP)) != cudaSuccess) return e;
  BgArgs a1{};
  a1.M = n;
  a1.K = d;
  a1.kchunk = up(d, 64);
  a1.nkc = 1;
  a1.N = N;
  a1.mode = 0;
  a1.vth = vh;
  a1.vtl = vl;
  a1.ldv = z.ldn;
  a1.wait = wait;
  a1.err = err;
  const int64_t items1 = (n + 127) / 128;
  if ((e = bgemm(NP, ah, al, bh, bl, a1, (int)(items1 < sms ? items1 : sms), st)) != cudaSuccess) return e;
  // Y = Z^T V: A = Z^T (d x n), B = V^T (NP x n), K = n cut into nkc chunks
  if ((e = make_map_bf16(&ah, z.th, n, d, z.ldn, 128)) != cudaSuccess) return e;
  if ((e = make_map_bf16(&al, z.tl, n, d, z.ldn, 128)) != cudaSuccess) return e;
  if ((e = make_map_bf16(&bh, vh, n, NP, z.ldn, NP)) != cudaSuccess) return e;
  if ((e = make_map_bf16(&bl, vl, n, NP, z.ldn, NP)) != cudaSuccess) return e;
  BgArgs a2{};
  a2.M = d;
  a2.K = n;
  a2.kchunk = kchunk;
  a2.nkc = nkc;
  a2.N = N;
  a2.mode = 1;
  a2.part = part;
  a2.ldp = ldp;
  a2.wait = wait;
  a2.err = err;
  const int64_t items2 = ((d + 127) / 128) * nkc;
  if ((e = bgemm(NP, ah, al, bh, bl, a2, (int)(items2 < sms ? items2 : sms), st)) != cudaSuccess) return e;
  const int64_t total = d * N;
  const int g = (int)((total + 255) / 256 < 152 * 8 ? (total + 255) / 256 : 152 * 8);
  k_bsum<<<g, 256, 0, st>>>(d, N, NP, nkc, part, ldp, alpha, beta, Y, ldy);
  return cudaGetLastError();
}

}  // namespace bk
