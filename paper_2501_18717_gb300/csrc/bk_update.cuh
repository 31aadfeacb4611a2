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

template <typename T, int MP>
__device__ __forceinline__ void update_pq_rows(int64_t i0, int64_t stride, int64_t d, int m, T* Q, T* P, int64_t ld,
                                               const T* sTi, const T* sTT, const T* sxc, bool do_x, bool upd,
                                               double* x) {
  for (int64_t i = i0; i < d; i += stride) {
    asm volatile("" ::: "memory");  // no hoisting of the shared reads across rows
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
}

}  // namespace bk
