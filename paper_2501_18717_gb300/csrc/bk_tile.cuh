// Fused tall-skinny Gram accumulation G += X_tile^T Y_tile for a tile of rows staged in
// shared memory (row-major, stride MP). Used by every kernel that produces a block and
// needs its Gram matrix in the same pass (P^T Y after a block product, R^T R after the
// residual update), so the blocks are never re-read for the Grams.
//
// Work split: the MP x MP result is cut into 4x4 register blocks; only the blocks on or
// above the diagonal are formed (NT of them). Thread s owns block s mod NT and the tile
// rows congruent to s / NT modulo NPH = blockDim / NT. When there are more blocks than
// threads (width 68 in 128-thread blocks: 153 blocks), thread s owns blocks s, s +
// blockDim, ... (BPT = ceil(NT / blockDim) of them) and every row of the tile.
//
// Precision: FP64 tiles accumulate in FP64. FP32 tiles multiply and add in FP32 within
// one tile (at most TM / NPH rows per thread) and carry the running sum across tiles as
// an unevaluated FP32 pair (hi, lo) with Knuth's TwoSum, so the sum over the whole block
// is formed with about twice FP32 precision; the per-CTA result is converted to FP64 and
// the CTA partials are added in FP64 in a fixed order (deterministic).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bk {

template <int MP>
struct GramShape {
  static constexpr int NB = MP / 4;
  static constexpr int NT = NB * (NB + 1) / 2;
  static constexpr int NE = NT * 16;
};

// Phases of the Gram accumulation in a block of `threads` (1 when blocks outnumber threads).
template <int MP>
__host__ __device__ constexpr int gram_phases(int threads) {
  return threads / GramShape<MP>::NT > 0 ? threads / GramShape<MP>::NT : 1;
}

// Blocks per thread for a kernel launched with NTH threads per block.
template <int MP, int NTH>
__host__ __device__ constexpr int gram_bpt() {
  return GramShape<MP>::NT <= NTH ? 1 : (GramShape<MP>::NT + NTH - 1) / NTH;
}

// BPT: blocks per thread; the kernel's blocks must have at least ceil(NT / BPT) threads.
template <typename T, int MP, int BPT = gram_bpt<MP, 128>()>
struct GramAcc;

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (i, j) of the t-th upper-triangular 4x4 block
template <int NB>
__device__ __forceinline__ void gram_block_ij(int t, int& bi, int& bj) {
  int tt = t, r = 0;
  while (tt >= NB - r) {
    tt -= NB - r;
    ++r;
  }
  bi = r;
  bj = r + tt;
}

template <int MP, int BPT>
struct GramAcc<float, MP, BPT> {
  using S = GramShape<MP>;
  int t, ph, nph, bi[BPT], bj[BPT], nb;
  bool active;
  float hi[BPT][16], lo[BPT][16];

  __device__ void init() {
    if (BPT == 1 || S::NT <= (int)blockDim.x) {  // BPT == 1: NT fits the block
      nph = blockDim.x / S::NT;
      t = threadIdx.x % S::NT;
      ph = threadIdx.x / S::NT;
      active = ph < nph;
      nb = 1;
    } else {  // more blocks than threads: blocks t, t + blockDim, ...; all rows
      nph = 1;
      t = threadIdx.x;
      ph = 0;
      active = true;
      nb = 0;
      for (int k = 0; k < BPT; ++k) nb += (t + k * (int)blockDim.x < S::NT) ? 1 : 0;
    }
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
      const int b = t + k * (int)blockDim.x;
      gram_block_ij<S::NB>(b < S::NT ? b : 0, bi[k], bj[k]);
#pragma unroll
      for (int e = 0; e < 16; ++e) hi[k][e] = lo[k][e] = 0.f;
    }
  }

  __device__ void tile(const float* sX, const float* sY, int rows) {
    if (!active) return;
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
      if (BPT > 1 && k >= nb) break;
      float acc[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) acc[e] = 0.f;
      for (int r = ph; r < rows; r += nph) {
        float4 x = *reinterpret_cast<const float4*>(sX + r * MP + 4 * bi[k]);
        float4 y = *reinterpret_cast<const float4*>(sY + r * MP + 4 * bj[k]);
        float xa[4] = {x.x, x.y, x.z, x.w};
        float yb[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a * 4 + b] = fmaf(xa[a], yb[b], acc[a * 4 + b]);
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        float s, err;
        two_sum(hi[k][e], acc[e], s, err);
        hi[k][e] = s;
        lo[k][e] = __fadd_rn(lo[k][e], err);
      }
    }
  }

  // tile() for a block of exactly NPH phases (one Gram block per thread) and a tile of
  // ROWS rows: the same rows in the same order, with a compile-time stride so the row
  // loop unrolls and the next rows' loads issue ahead of the multiply-adds.
  template <int ROWS, int NPH>
  __device__ void tile_fixed(const float* sX, const float* sY) {
    static_assert(BPT == 1, "one Gram block per thread");
    if (!active) return;
    constexpr int IT = ROWS / NPH;
    float acc[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[e] = 0.f;
    auto row = [&](int r) {
      float4 x = *reinterpret_cast<const float4*>(sX + r * MP + 4 * bi[0]);
      float4 y = *reinterpret_cast<const float4*>(sY + r * MP + 4 * bj[0]);
      float xa[4] = {x.x, x.y, x.z, x.w};
      float yb[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a * 4 + b] = fmaf(xa[a], yb[b], acc[a * 4 + b]);
    };
#pragma unroll 8
    for (int it = 0; it < IT; ++it) row(ph + it * NPH);
    if (ph < ROWS - IT * NPH) row(ph + IT * NPH);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      float s, err;
      two_sum(hi[0][e], acc[e], s, err);
      hi[0][e] = s;
      lo[0][e] = __fadd_rn(lo[0][e], err);
    }
  }

  __device__ double value(int k, int e) const { return (double)hi[k][e] + (double)lo[k][e]; }
};

template <int MP, int BPT>
struct GramAcc<double, MP, BPT> {
  using S = GramShape<MP>;
  int t, ph, nph, bi[BPT], bj[BPT], nb;
  bool active;
  double hi[BPT][16];

  __device__ void init() {
    if (BPT == 1 || S::NT <= (int)blockDim.x) {  // BPT == 1: NT fits the block
      nph = blockDim.x / S::NT;
      t = threadIdx.x % S::NT;
      ph = threadIdx.x / S::NT;
      active = ph < nph;
      nb = 1;
    } else {
      nph = 1;
      t = threadIdx.x;
      ph = 0;
      active = true;
      nb = 0;
      for (int k = 0; k < BPT; ++k) nb += (t + k * (int)blockDim.x < S::NT) ? 1 : 0;
    }
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
      const int b = t + k * (int)blockDim.x;
      gram_block_ij<S::NB>(b < S::NT ? b : 0, bi[k], bj[k]);
#pragma unroll
      for (int e = 0; e < 16; ++e) hi[k][e] = 0.0;
    }
  }

  __device__ void tile(const double* sX, const double* sY, int rows) {
    if (!active) return;
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
      if (BPT > 1 && k >= nb) break;
      for (int r = ph; r < rows; r += nph) {
        const double2* px = reinterpret_cast<const double2*>(sX + r * MP + 4 * bi[k]);
        const double2* py = reinterpret_cast<const double2*>(sY + r * MP + 4 * bj[k]);
        double2 x01 = px[0], x23 = px[1], y01 = py[0], y23 = py[1];
        double xa[4] = {x01.x, x01.y, x23.x, x23.y};
        double yb[4] = {y01.x, y01.y, y23.x, y23.y};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) hi[k][a * 4 + b] = fma(xa[a], yb[b], hi[k][a * 4 + b]);
      }
    }
  }

  __device__ double value(int k, int e) const { return hi[k][e]; }
};

// One tile of ROWS rows in a block of NTH threads: FP32 Grams with one block per thread
// take the fixed-stride loop, the others the general one (same rows, same order).
template <int ROWS, int NTH, typename T, int MP, int BPT>
__device__ __forceinline__ void gram_tile(GramAcc<T, MP, BPT>& g, const T* sX, const T* sY) {
  if constexpr (sizeof(T) == 4 && BPT == 1 && GramShape<MP>::NT <= NTH)
    g.template tile_fixed<ROWS, gram_phases<MP>(NTH)>(sX, sY);
  else
    g.tile(sX, sY, ROWS);
}

// Combine the phases of one CTA (fixed order) and write the CTA partial:
// parts[e * nparts + cta] for e in [0, NE). sred needs nph * NT * 16 doubles and may
// alias the tile buffers (the caller synchronises before calling).
template <typename T, int MP, int BPT>
__device__ void gram_finish(const GramAcc<T, MP, BPT>& g, double* sred, double* parts, int nparts, int cta) {
  using S = GramShape<MP>;
  if (g.active) {
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
      if (BPT > 1 && k >= g.nb) break;
      const int b = g.t + k * (int)blockDim.x;  // block index (one block per thread when nph > 0)
#pragma unroll
      for (int e = 0; e < 16; ++e) sred[(g.ph * S::NT + b) * 16 + e] = g.value(k, e);
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < S::NE; idx += blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < g.nph; ++p) s += sred[p * S::NE + idx];
    parts[(size_t)idx * nparts + cta] = s;
  }
}

// Row `row` of a shared tile (stride MP) from MP register values.
template <int MP>
__device__ __forceinline__ void store_row(float* s, int row, const float (&v)[MP]) {
  float4* p = reinterpret_cast<float4*>(s + row * MP);
#pragma unroll
  for (int q = 0; q < MP / 4; ++q) p[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}
template <int MP>
__device__ __forceinline__ void store_row(double* s, int row, const double (&v)[MP]) {
  double2* p = reinterpret_cast<double2*>(s + row * MP);
#pragma unroll
  for (int q = 0; q < MP / 2; ++q) p[q] = make_double2(v[2 * q], v[2 * q + 1]);
}
// Four consecutive columns (chunk q) of row `row` as one 16-byte store (FP32) or two
// (FP64); conflict-free when consecutive threads store consecutive rows.
template <int MP>
__device__ __forceinline__ void store4(float* s, int row, int q, const float (&v)[4]) {
  *reinterpret_cast<float4*>(s + row * MP + 4 * q) = make_float4(v[0], v[1], v[2], v[3]);
}
template <int MP>
__device__ __forceinline__ void store4(double* s, int row, int q, const double (&v)[4]) {
  double2* p = reinterpret_cast<double2*>(s + row * MP + 4 * q);
  p[0] = make_double2(v[0], v[1]);
  p[1] = make_double2(v[2], v[3]);
}
template <typename T, int MP>
__device__ __forceinline__ void zero_row(T* s, int row) {
#pragma unroll
  for (int c = 0; c < MP; ++c) s[row * MP + c] = (T)0;
}

// ---------------------------------------------------------------- block layout
// A d x m block is stored as panels of four columns: element (i, c) lives at
// ((c / 4) * ld + i) * 4 + c % 4, so one row of a panel is one 16-byte (FP32) or
// 32-byte (FP64) vector and consecutive rows are contiguous. Columns m..4*ceil(m/4)-1
// of the last panel are padding and hold zeros in every block the library writes.
template <typename T>
__device__ __forceinline__ const T* panel_row(const T* base, int64_t ld, int q, int64_t i) {
  return base + ((int64_t)q * ld + i) * 4;
}
template <typename T>
__device__ __forceinline__ T* panel_row(T* base, int64_t ld, int q, int64_t i) {
  return base + ((int64_t)q * ld + i) * 4;
}
__device__ __forceinline__ void ldg4(const float* p, float* v) {
  float4 t = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ldg4(const double* p, double* v) {
  double2 a = __ldg(reinterpret_cast<const double2*>(p));
  double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
// plain (coherent) load for blocks the same kernel also writes
__device__ __forceinline__ void ld4(const float* p, float* v) {
  float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double* v) {
  double2 a = reinterpret_cast<const double2*>(p)[0];
  double2 b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double* v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}


// Shared bytes a Gram-fused kernel needs: two tiles of TM rows, or the phase buffer.
template <typename T, int MP>
inline size_t gram_smem_bytes(int tm, int threads) {
  size_t tiles = 2 * (size_t)tm * MP * sizeof(T);
  size_t red = (size_t)gram_phases<MP>(threads) * GramShape<MP>::NE * sizeof(double);
  return tiles > red ? tiles : red;
}

}  // namespace bk
