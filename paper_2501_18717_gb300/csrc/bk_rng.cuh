// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the Box-Muller transform on the
// device: the Gaussian sketch Omega of the start block (layout defined in bk.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bk {

struct U4 {
  uint32_t x0, x1, x2, x3;
};

__device__ __forceinline__ U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                       uint32_t k1) {
  // Ten rounds; round constants and Weyl key increments from the SC'11 definition.
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

// Both normals of Philox block c of `stream`.
__device__ __forceinline__ void normal_pair(uint64_t seed, uint32_t stream, uint64_t c, double& z0,
                                            double& z1) {
  U4 w = philox10((uint32_t)c, (uint32_t)(c >> 32), stream, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double two53 = 1.1102230246251565e-16;  // 2^-53
  double u1 = ((double)(w.x0 >> 5) * 67108864.0 + (double)(w.x1 >> 6) + 0.5) * two53;
  double u2 = ((double)(w.x2 >> 5) * 67108864.0 + (double)(w.x3 >> 6) + 0.5) * two53;
  double r = sqrt(-2.0 * log(u1));
  double ang = 6.283185307179586 * u2;  // 2 pi u2, the same product the host generator forms
  z0 = r * cos(ang);
  z1 = r * sin(ang);
}

// Normal k of a stream (one Philox block per pair; the caller may recompute a pair).
__device__ __forceinline__ double normal_at(uint64_t seed, uint32_t stream, uint64_t k) {
  double z0, z1;
  normal_pair(seed, stream, k >> 1, z0, z1);
  return (k & 1) ? z1 : z0;
}

}  // namespace bk
