// Row loop of the direction update shared by the single-system and batched solvers:
// x += P xc; unless the inner solve stopped, Q = W Ti (W held in Q) and P = Q + P T^T.
// Thread per row of the panel blocks, both rows loaded up front. The two triangular
// products run in place over the row registers as sequences of row updates that read
// one contiguous row of Ti or T^T from shared memory (16-byte broadcasts):
//   q = w Ti,      k descending: slot c > k already holds its partial sum;
//   p = q + p T^T, k ascending:  slot c < k already holds its partial sum.
// The inner loops have a constant trip count with a compile-time predicate, so they
// unroll completely and the row arrays stay in registers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bk_tile.cuh"

namespace bk {

// One row after its P and W values are in registers: x += p xc, then (unless the solve
// stopped) w <- w Ti, p <- w + p T^T, and both rows stored.
template <typename T, int MP>
__device__ __forceinline__ void update_pq_row(int64_t i, int m, T* Q, T* P, int64_t ld, const T* sTi, const T* sTT,
                                              const T* sxc, bool do_x, bool upd, double* x, T (&p)[MP],
                                              T (&w)[MP]) {
  if (do_x) {
    T xs = 0;
#pragma unroll
    for (int k = 0; k < MP; ++k) xs = fma(p[k], sxc[k], xs);
    x[i] += (double)xs;
  }
  if (upd) {
#pragma unroll
    for (int k = MP - 1; k >= 0; --k) {
      const T* r = sTi + k * MP;
      const T wk = w[k];
#pragma unroll
      for (int c = 0; c < MP; ++c)
        if (c > k) w[c] = fma(wk, r[c], w[c]);
      w[k] = wk * r[k];
    }
#pragma unroll
    for (int k = 0; k < MP; ++k) {
      const T* r = sTT + k * MP;
      const T pk = p[k];
#pragma unroll
      for (int c = 0; c < MP; ++c)
        if (c < k) p[c] = fma(pk, r[c], p[c]);
      p[k] = fma(pk, r[k], w[k]);
    }
#pragma unroll
    for (int q = 0; q < MP / 4; ++q)
      if (4 * q < m) {
        st4(panel_row(Q, ld, q, i), w + 4 * q);
        st4(panel_row(P, ld, q, i), p + 4 * q);
      }
  }
}

template <typename T, int MP>
__device__ __forceinline__ void update_pq_rows(int64_t i0, int64_t stride, int64_t d, int m, T* Q, T* P, int64_t ld,
                                               const T* sTi, const T* sTT, const T* sxc, bool do_x, bool upd,
                                               double* x) {
  double xi = (do_x && i0 < d) ? x[i0] : 0.0;  // x one row ahead (a register)
  for (int64_t i = i0; i < d; i += stride) {
    asm volatile("" ::: "memory");  // no hoisting of the shared reads across rows
    const double xcur = xi;
    if (do_x && i + stride < d) xi = x[i + stride];
    T p[MP], w[MP];
#pragma unroll
    for (int q = 0; q < MP / 4; ++q) {
      if (4 * q < m) {
        ld4(panel_row(P, ld, q, i), p + 4 * q);
        if (upd)
          ld4(panel_row(Q, ld, q, i), w + 4 * q);
        else {
#pragma unroll
          for (int u = 0; u < 4; ++u) w[4 * q + u] = (T)0;
        }
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) p[4 * q + u] = w[4 * q + u] = (T)0;
      }
    }
    if (do_x) {
      T xs = 0;
#pragma unroll
      for (int k = 0; k < MP; ++k) xs = fma(p[k], sxc[k], xs);
      x[i] = xcur + (double)xs;
    }
    update_pq_row<T, MP>(i, m, Q, P, ld, sTi, sTT, sxc, false, upd, x, p, w);
  }
}

// 16-byte asynchronous copy global -> shared (zero-filled when src_bytes is 0)
__device__ __forceinline__ void upd_cp16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void upd_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void upd_cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void upd_cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// FP32 rows with the next row in flight: each thread copies its own row's live panels
// of P and W into its slots of a two-stage shared-memory ring (cp.async, 16 bytes each,
// zero-filled past d, no registers held) and updates the previous row meanwhile. It
// reads only its own slots, which cp.async.wait_group makes visible to it, so there is
// no barrier. ring holds 2 stages x 2 arrays x MP / 4 panels x blockDim 16-byte slots.
template <int MP>
__device__ __forceinline__ void update_pq_rows_async(int64_t i0, int64_t stride, int64_t d, int m, float* Q, float* P,
                                                     int64_t ld, const float* sTi, const float* sTT,
                                                     const float* sxc, bool do_x, bool upd, double* x,
                                                     float4* ring) {
  constexpr int NQ = MP / 4;
  const int nt = blockDim.x, t = threadIdx.x;
  auto issue = [&](int64_t i, int s) {
    const bool ok = i < d;
    const int bytes = ok ? 16 : 0;
    const int64_t ii = ok ? i : 0;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      if (4 * q < m) {
        upd_cp16(ring + ((s * 2 + 0) * NQ + q) * nt + t, panel_row(P, ld, q, ii), bytes);
        if (upd) upd_cp16(ring + ((s * 2 + 1) * NQ + q) * nt + t, panel_row(Q, ld, q, ii), bytes);
      }
    upd_cp_commit();
  };
  int s = 0;
  issue(i0, 0);
  // x of the row is read one row ahead too (a register), so its read-modify-write
  // does not wait on memory inside the row
  double xi = (do_x && i0 < d) ? x[i0] : 0.0;
  for (int64_t i = i0; i < d; i += stride, s ^= 1) {
    issue(i + stride, s ^ 1);
    const double xcur = xi;
    if (do_x && i + stride < d) xi = x[i + stride];
    upd_cp_wait1();  // this row's copies have landed
    float p[MP], w[MP];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
      if (4 * q < m) {
        a = ring[((s * 2 + 0) * NQ + q) * nt + t];
        if (upd) b = ring[((s * 2 + 1) * NQ + q) * nt + t];
      }
      p[4 * q] = a.x;
      p[4 * q + 1] = a.y;
      p[4 * q + 2] = a.z;
      p[4 * q + 3] = a.w;
      w[4 * q] = b.x;
      w[4 * q + 1] = b.y;
      w[4 * q + 2] = b.z;
      w[4 * q + 3] = b.w;
    }
    if (do_x) {
      float xs = 0.f;
#pragma unroll
      for (int k = 0; k < MP; ++k) xs = fmaf(p[k], sxc[k], xs);
      x[i] = xcur + (double)xs;
    }
    update_pq_row<float, MP>(i, m, Q, P, ld, sTi, sTT, sxc, false, upd, x, p, w);
  }
  upd_cp_wait0();
}

}  // namespace bk
