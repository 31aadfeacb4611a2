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

#include <mutex>

#include "../../include/bk.h"
#include "bk_common.cuh"

namespace {

// 4 MiB of FP64 partials: the full grid of the block-product kernel (three CTAs per SM
// on up to 240 SMs) times the 720 partial entries of the widest block (m <= 36).
constexpr size_t kStaticParts = (size_t)1 << 19;
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

bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" bk_status bk_block_apply_static(const bk_operator* A, double mu, int32_t dtype, int64_t m,
                                           const void* P, void* Y, int64_t ld, double* G, void* cuda_stream) {
  if (!A || !A->vals || !P || !Y || !G) return BK_ERR_ARG;
  if (A->kind != BK_DENSE && A->kind != BK_CSR) return BK_ERR_UNSUPPORTED;
  if (dtype != BK_F64 && dtype != BK_F32) return BK_ERR_UNSUPPORTED;
  // no conversion buffer: the values must already be in the block precision
  if (A->dtype != dtype) return BK_ERR_UNSUPPORTED;
  if (A->rows <= 0 || A->rows != A->cols || A->rows > (int64_t)INT32_MAX - 1) return BK_ERR_ARG;
  if (m < 1 || ld < A->rows || !(mu == mu)) return BK_ERR_ARG;
  if (A->kind == BK_DENSE && A->ld < A->cols) return BK_ERR_ARG;
  if (A->kind == BK_CSR && (!A->rowptr || !A->colidx || A->nnz < 0)) return BK_ERR_ARG;
  const int mp = bk::padded_width((int)m);
  if (mp < 0 || m > bk::kMaxWidth) return BK_ERR_UNSUPPORTED;
  // no staging buffer either: every array must be device-accessible
  if (!on_device(A->vals) || !on_device(P) || !on_device(Y) || !on_device(G)) return BK_ERR_ARG;
  if (A->kind == BK_CSR && (!on_device(A->rowptr) || !on_device(A->colidx))) return BK_ERR_ARG;

  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return BK_ERR_CUDA;
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
