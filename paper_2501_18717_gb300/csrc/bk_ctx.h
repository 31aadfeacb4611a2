// Context and workspace of the C ABI, shared by the entry-point files (bk_api.cu,
// bk_krylov_api.cu). Internal: nothing here is part of include/bk.h.
#pragma once

#include <cuda_runtime.h>

#include <cstdio>
#include <map>

#include "../../include/bk.h"
#include "bk_common.cuh"

enum Slot {
  WS_P, WS_R, WS_Y, WS_OMEGA, WS_XIN, WS_X64, WS_R64, WS_B64, WS_PARTS_G, WS_PARTS_S, WS_MATS, WS_STATE,
  WS_OP_VALS, WS_OP_ROW, WS_OP_COL, WS_VALS_INNER, WS_NORMP, WS_TMP_IN, WS_TMP_OUT, WS_TMP_G, WS_TMP_S,
  // block-Lanczos drivers
  WS_LQ, WS_LW, WS_LV, WS_LC, WS_LSMALL, WS_LBAND, WS_LBWORK, WS_LZ, WS_LRHS, WS_LX, WS_LAX, WS_LRES, WS_LB0,
  WS_LSHIFT, WS_LB64, WS_LQ2, WS_SPLIT, WS_TSM, WS_NYU, WS_PCG, WS_SPLITB, WS_DEFL,
  // batched solver
  WS_BATCH, WS_BATCH_VALS,
  // tensor-core dense product: P^T head/tail, timeout flag
  WS_PT, WS_TCERR,
  // BF16 Gram-form loads: head/tail copies of Z, product workspace
  WS_BF16, WS_BF16W,
  // single solve: trial iterate and residual of a refinement pass; FP64-block fallback
  // (iterate, residual, correction kept across the nested solve)
  WS_XT, WS_RT, WS_FB_X, WS_FB_R, WS_FB_D,
  // Ozaki-split products: digits and exponents of the operator, of the block
  WS_OZ_A, WS_OZ_X, WS_OZ_G,
  WS_COUNT
};

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct bk_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;  // created when the caller passes the legacy default stream
  char last_error[256] = {0};
  Buf ws[WS_COUNT];
  bk::DevState* hstate = nullptr;  // pinned mirror of the device control block
  double* hparts = nullptr;        // pinned buffer for norm partials and small reads
  int sms = 152;
  std::map<int, int> tune;     // autotuner: floor(log2 d) -> sketch columns
  std::map<int, int> tune_tc;  // autotuner: floor(log2 d) -> 1 tensor-core product, 0 CUDA-core
  int force_tc = -1;           // autotuner timing: -1 none, else the product kernel to use
};

namespace bkx {

constexpr int kHostParts = 1024;

inline bk_ctx*& err_ctx() {
  static thread_local bk_ctx* c = nullptr;
  return c;
}

inline bk_status from_cuda(cudaError_t e, const char* what = nullptr, int line = 0, const char* file = "") {
  if (e == cudaSuccess) return BK_OK;
  cudaGetLastError();  // clear a sticky launch error so the context stays usable
  if (err_ctx())
    std::snprintf(err_ctx()->last_error, sizeof(err_ctx()->last_error), "%s:%d %s: %s", file, line,
                  what ? what : "", cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return BK_ERR_OOM;
  return BK_ERR_CUDA;
}

#define BK_CK(expr)                                                         \
  do {                                                                      \
    cudaError_t e_ = (expr);                                                \
    if (e_ != cudaSuccess) return bkx::from_cuda(e_, #expr, __LINE__, __FILE__); \
  } while (0)

inline cudaError_t ws_get(bk_ctx* c, Slot s, size_t bytes, void** out) {
  Buf& b = c->ws[s];
  if (bytes == 0) bytes = 16;
  if (b.bytes < bytes) {
    if (b.p) {
      cudaError_t e = cudaStreamSynchronize(c->stream);
      if (e != cudaSuccess) return e;
      cudaFree(b.p);
      b.p = nullptr;
      b.bytes = 0;
    }
    size_t want = (bytes + (1u << 20) - 1) & ~((size_t)(1u << 20) - 1);
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
      b.p = nullptr;
      return e;
    }
    b.bytes = want;
  }
  *out = b.p;
  return cudaSuccess;
}

inline bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Argument checks of a dense or CSR operator, shared by every entry point that takes
// one (the same rules for the context calls and the allocation-free block product).
inline bk_status check_operator(const bk_operator* A) {
  if (!A || !A->vals) return BK_ERR_ARG;
  if (A->kind != BK_DENSE && A->kind != BK_CSR) return BK_ERR_UNSUPPORTED;
  if (A->dtype != BK_F64 && A->dtype != BK_F32) return BK_ERR_UNSUPPORTED;
  if (A->rows <= 0 || A->rows != A->cols) return BK_ERR_ARG;
  if (A->rows > (int64_t)INT32_MAX - 1) return BK_ERR_UNSUPPORTED;
  if (A->kind == BK_DENSE && A->ld < A->cols) return BK_ERR_ARG;
  if (A->kind == BK_CSR && (!A->rowptr || !A->colidx || A->nnz < 0 || A->nnz > (int64_t)INT32_MAX))
    return BK_ERR_ARG;
  return BK_OK;
}

// Device view of a borrowed input array: the pointer itself, or a staged copy.
inline cudaError_t stage_in(bk_ctx* c, Slot s, const void* p, size_t bytes, const void** out) {
  if (is_device_ptr(p)) {
    *out = p;
    return cudaSuccess;
  }
  void* d = nullptr;
  cudaError_t e = ws_get(c, s, bytes, &d);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, c->stream);
  *out = d;
  return e;
}

// Host sum of per-CTA partials in fixed order.
inline cudaError_t host_sum(bk_ctx* c, const double* dparts, int n, double* out) {
  cudaError_t e = cudaMemcpyAsync(c->hparts, dparts, (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return e;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += c->hparts[i];
  *out = s;
  return cudaSuccess;
}

}  // namespace bkx
