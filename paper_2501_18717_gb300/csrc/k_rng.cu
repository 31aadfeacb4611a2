// Gaussian sketch Omega on the device: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11) and the Box-Muller
// transform. The paper draws Omega with independent standard normal entries
// (Sec. 2.2.2, Eq. nystromBKI_def; Thm. main); the stream layout is given in bk.h.
#include "bk_common.cuh"
#include "bk_rng.cuh"

namespace bk {
namespace {

__global__ void k_gaussian(uint64_t seed, uint32_t stream, int64_t n, int64_t offset, double* out) {
  // thread per Philox block covering normals [offset, offset + n)
  int64_t first_blk = offset >> 1;
  int64_t last_blk = (offset + n - 1) >> 1;
  for (int64_t blk = first_blk + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; blk <= last_blk;
       blk += (int64_t)gridDim.x * blockDim.x) {
    double z0, z1;
    normal_pair(seed, stream, (uint64_t)blk, z0, z1);
    int64_t k0 = 2 * blk, k1 = 2 * blk + 1;
    if (k0 >= offset && k0 < offset + n) out[k0 - offset] = z0;
    if (k1 >= offset && k1 < offset + n) out[k1 - offset] = z1;
  }
}

template <typename T>
__global__ void k_omega(int64_t d, int l, int64_t ld, uint64_t seed, double scale, T* out) {
  int64_t n = d * (int64_t)l;
  int64_t nblk = (n + 1) >> 1;
  for (int64_t blk = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; blk < nblk;
       blk += (int64_t)gridDim.x * blockDim.x) {
    double z0, z1;
    normal_pair(seed, 3u, (uint64_t)blk, z0, z1);
    int64_t k0 = 2 * blk, k1 = k0 + 1;
    // entry k is (row k mod d, column k / d) of Omega, stored as column c = j + 1 of a
    // panel block (element (i, c) at ((c / 4) ld + i) 4 + c % 4)
    int64_t j0 = k0 / d, i0 = k0 - j0 * d;
    out[(((j0 + 1) >> 2) * ld + i0) * 4 + ((j0 + 1) & 3)] = (T)(z0 * scale);
    if (k1 < n) {
      int64_t j1 = k1 / d, i1 = k1 - j1 * d;
      out[(((j1 + 1) >> 2) * ld + i1) * 4 + ((j1 + 1) & 3)] = (T)(z1 * scale);
    }
  }
}

inline int grid_for(int64_t work, int threads) {
  int64_t g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 152 * 16) g = 152 * 16;
  return (int)g;
}

}  // namespace

cudaError_t launch_gaussian(uint64_t seed, uint32_t stream, int64_t n, int64_t offset, double* out,
                            cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t nblk = ((offset + n - 1) >> 1) - (offset >> 1) + 1;
  k_gaussian<<<grid_for(nblk, 256), 256, 0, st>>>(seed, stream, n, offset, out);
  return cudaGetLastError();
}

cudaError_t launch_omega(int is_f64, int64_t d, int l, int64_t ld, uint64_t seed, double scale, void* out,
                         cudaStream_t st) {
  if (l <= 0 || d <= 0) return cudaSuccess;
  int64_t nblk = (d * (int64_t)l + 1) >> 1;
  if (is_f64)
    k_omega<double><<<grid_for(nblk, 256), 256, 0, st>>>(d, l, ld, seed, scale, (double*)out);
  else
    k_omega<float><<<grid_for(nblk, 256), 256, 0, st>>>(d, l, ld, seed, scale, (float*)out);
  return cudaGetLastError();
}

}  // namespace bk
