// bfp_noalloc.cu -- bfp_jacobi_noalloc: damped Jacobi with its qcomp window in
// a static device array instead of caller- or library-allocated memory.
//
// Who needs it: callers that cannot allocate device memory at the point of the
// call -- code running inside a host callback or another context where CUDA
// allocation calls are not allowed, code whose device memory budget is owned
// by another framework's allocator, or code that must never trigger the
// implicit device synchronisation a cudaMalloc / cudaFree can cause.  Such a
// caller still provides the inputs and the output; the only scratch this op
// needs (the w_tmp-bit window of the qcomp first pass) comes from g_window.
//
// g_window is a file-scope __device__ array: every GPU that loads this library
// holds its kWindowMax * 4 bytes (16 MiB) until the process exits.  All calls
// on a device share it and it keeps the contents of the last call; calls that
// overlap on the GPU (different streams without ordering) race on it.  The
// window never needs clearing: the first pass writes every entry the second
// pass reads.
#include "bfp_host.h"

using namespace bfp;

namespace {

constexpr int64_t kWindowMax = int64_t(1) << 22;   // int32 entries (rows * ld of the output)

__device__ __align__(256) int32_t g_window[kWindowMax];

// Device address of g_window on the current device.  The host-side symbol g_window is not a
// device address and must not be passed to a kernel.  The address is looked up on every call,
// so it stays right after a device reset or a new primary context in the same process; a failed
// lookup clears the runtime's last-error state so that it is not reported by a later, unrelated
// launch check.
int32_t window_address(void** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_window) != cudaSuccess || p == nullptr) {
    (void)cudaGetLastError();
    return BFP_ERR_CUDA;
  }
  *out = p;
  return BFP_OK;
}

}  // namespace

extern "C" {

int64_t bfp_noalloc_window_capacity(void) { return kWindowMax; }

int32_t bfp_jacobi_noalloc(const bfp_stencil* A, const bfp_vec* y, const bfp_vec* r, const bfp_vec* y_out,
                           const bfp_q* q, const bfp_stats* st, bfp_stream stream) {
  int32_t rc;
  if (!q || !y_out) return BFP_ERR_ARG;
  if ((rc = check_vec(y_out))) return rc;
  bfp_q qq = *q;
  qq.tmp = nullptr;
  // the window is used by qcomp when w_tmp = w_out + w_add fits in 32 bits (the relaxation row's
  // w_add 2 unless the caller gives one); nnqcomp, and qcomp with a wider w_tmp, need no scratch
  const int w_add = q->w_add < 0 ? capped_wadd(2, wadd_cap()) : q->w_add;
  if (q->mode == BFP_QCOMP && q->w_out + w_add <= 32) {
    if (rows_of(y_out) * y_out->ld > kWindowMax) return BFP_ERR_CAPACITY;
    void* w = nullptr;
    if ((rc = window_address(&w))) return rc;
    qq.tmp = w;
  }
  return bfp_jacobi(A, y, r, y_out, &qq, st, stream);
}

}  // extern "C"
