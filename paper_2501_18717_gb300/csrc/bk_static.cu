// bk_block_apply_static: the block product with its Gram matrix, with no device memory
// allocation. The paper has no counterpart; this exists for callers that may not let
// a library allocate device memory (see include/bk.h).
//
// The only scratch of the block product is the per-CTA Gram partials. Here they live in
// a file-scope __device__ array of fixed size, so the call allocates nothing. The array
// exists once per device that loads this library and stays resident until the process
// exits. Every call on a device shares it: calls whose kernels overlap on the GPU race
// on it, and each call overwrites every partial it reads (nothing needs clearing).
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/bk.h"
#include "bk_common.cuh"
#include "bk_ctx.h"

namespace {

// 4 MiB of FP64 partials. The widest block (m <= 36) has 720 partial entries per CTA
// and the block-product grids run at most four CTAs per SM, so the array holds the
// partials of every launch on GPUs with up to 182 SMs (4 x 182 x 720 <= 2^19); larger
// grids are refused with BK_ERR_TOO_LARGE.
constexpr size_t kStaticParts = (size_t)1 << 19;
constexpr int kStaticMaxWidth = 36;
__device__ __align__(256) double g_static_parts[kStaticParts];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_parts_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once per device.
// The host-side name g_static_parts is only a stand-in for the symbol and must never be
// handed to a kernel.
cudaError_t static_parts(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mutex);
  if (!g_parts_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_parts);
    if (e != cudaSuccess) return e;
    g_parts_ptr[device] = static_cast<double*>(p);
  }
  *out = g_parts_ptr[device];
  return cudaSuccess;
}

// True if p is device (or managed) memory that the given device owns. Memory of another
// GPU is refused: the kernels run on the current device and would otherwise read it
// over the peer link or fault.
bool on_device(const void* p, int device) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == device;
}

}  // namespace

extern "C" bk_status bk_block_apply_static(const bk_operator* A, double mu, int32_t dtype, int64_t m,
                                           const void* P, void* Y, int64_t ld, double* G, void* cuda_stream) {
  // the same operator and argument checks as bk_block_apply
  bk_status s = bkx::check_operator(A);
  if (s != BK_OK) return s;
  if (!P || !Y || !G) return BK_ERR_ARG;
  if (m < 1 || ld < A->rows || !std::isfinite(mu)) return BK_ERR_ARG;
  if (dtype != BK_F64 && dtype != BK_F32) return BK_ERR_UNSUPPORTED;
  // no conversion buffer: the values must already be in the block precision
  if (A->dtype != dtype) return BK_ERR_UNSUPPORTED;
  const int mp = bk::padded_width((int)m);
  if (mp < 0 || m > kStaticMaxWidth) return BK_ERR_UNSUPPORTED;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    return BK_ERR_CUDA;
  }
  // no staging buffer either: every array must be memory of the current device
  if (!on_device(A->vals, device) || !on_device(P, device) || !on_device(Y, device) || !on_device(G, device))
    return BK_ERR_ARG;
  if (A->kind == BK_CSR && (!on_device(A->rowptr, device) || !on_device(A->colidx, device))) return BK_ERR_ARG;

  const int is64 = dtype == BK_F64;
  const int64_t d = A->rows;
  const int nparts = (A->kind == BK_CSR) ? bk::csr_spmm_gram_grid(is64, mp, d, device)
                                         : bk::dense_gram_grid(is64, mp, d, device);
  if ((size_t)nparts * bk::gram_entries(mp) > kStaticParts) return BK_ERR_TOO_LARGE;
  double* parts = nullptr;
  if (static_parts(device, &parts) != cudaSuccess) {
    cudaGetLastError();
    return BK_ERR_CUDA;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaError_t e = (A->kind == BK_CSR)
                      ? bk::launch_csr_spmm_gram(is64, mp, d, A->rowptr, A->colidx, A->vals, mu, P, Y, ld, (int)m,
                                                 parts, nparts, nullptr, st)
                      : bk::launch_dense_gram(is64, mp, d, A->vals, A->ld, mu, P, Y, ld, (int)m, parts, nparts,
                                              nullptr, st);
  if (e == cudaSuccess) e = bk::launch_reduce_gram(mp, (int)m, parts, nparts, G, nullptr, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return BK_ERR_CUDA;
  }
  return BK_OK;
}
