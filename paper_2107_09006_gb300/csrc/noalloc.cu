// Allocation-free normal-equations product w = A^T (A p).
//
// Some callers cannot call cudaMalloc: code whose device memory must all come from a
// framework's own pool or a fixed budget set aside at start-up, and real-time loops
// that must not enter the CUDA memory allocator (cudaMalloc and cudaFree can
// synchronise the device and take an unbounded time).  This entry point lets them
// apply the operator C = A^T A without the library allocating anything: the caller
// passes A in CSR and CSC form, p and w; the intermediate q = A p lives in a
// file-scope device array of fixed size, the same array for every call.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/ls_schwarz.h"
#include "kernels.h"

namespace {

constexpr int64_t kMaxRows = int64_t(1) << 23;  // 8,388,608 rows: 64 MB of FP64 per device
constexpr int kMaxDevices = 64;

// Scratch for q = A p.  Every call overwrites q[0 .. m) before reading it, so nothing
// needs clearing between calls.
static __device__ __align__(256) double g_q[kMaxRows];

// Device address of g_q, looked up once per device and context: the address belongs to
// the module loaded into one CUDA context, so a new context on the same device (after
// cudaDeviceReset, or a context the caller made current through the driver API) gets a
// fresh lookup instead of a stale pointer.
struct ScratchAddr {
  double* ptr;
  unsigned long long ctx;  // driver context id the address was taken in (0: unknown)
};

std::mutex g_mu;
ScratchAddr g_addr[kMaxDevices] = {};

thread_local std::string g_msg;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Id of the context current on this thread, 0 if none is current or the driver does
// not report one.  The two driver functions are fetched through the runtime, so the
// library does not link the driver library itself.
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
    cudaGetLastError();  // a symbol the driver lacks is not an error of the caller's work
  });
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

int pow2_lanes(double avg) {
  int v = 1;
  while (v < 32 && v < avg) v <<= 1;
  return v;
}

}  // namespace

extern "C" const char* ls_noalloc_last_error(void) { return g_msg.c_str(); }

extern "C" ls_status ls_normal_product_noalloc(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col,
                                               const double* val, const int64_t* col_ptr, const int32_t* row,
                                               const double* cval, int64_t nnz, const double* p, double* w,
                                               void* stream) {
  g_msg.clear();
  if (m < 1 || n < 1 || nnz < 0 || !row_ptr || !col_ptr || !p || !w || (nnz > 0 && (!col || !val || !row || !cval))) {
    g_msg = "invalid argument";
    return LS_ERR_INVALID;
  }
  if (m > kMaxRows) {
    g_msg = "m = " + std::to_string(m) + " exceeds the fixed scratch of " + std::to_string(kMaxRows) + " rows";
    return LS_ERR_INVALID;
  }
  // An error left by the caller's earlier work is reported and left in place (peek, not
  // get): it is not this call's to clear, and after it nothing here can be trusted.
  const cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess) {
    g_msg = std::string("an earlier CUDA error is pending: ") + cudaGetErrorString(pending);
    return LS_ERR_CUDA;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    if (e != cudaSuccess) cudaGetLastError();  // this call's own error
    g_msg = std::string("no usable current device: ") + cudaGetErrorString(e);
    return LS_ERR_CUDA;
  }
  double* q = nullptr;
  {
    // Once per device and context, with that device current: the device address of the
    // scratch (the first lookup may load this file's module and create the context).
    std::lock_guard<std::mutex> lk(g_mu);
    unsigned long long ctx = current_context_id();
    ScratchAddr& a = g_addr[dev];
    if (!a.ptr || ctx == 0 || a.ctx != ctx) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_q);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        a.ptr = nullptr;
        g_msg = std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
        return LS_ERR_CUDA;
      }
      a.ptr = static_cast<double*>(ptr);
      a.ctx = current_context_id();
    }
    q = a.ptr;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const lsq::CsrDev A{m, n, row_ptr, col, val};
  const lsq::CscDev At{m, n, col_ptr, row, cval};
  lsq::launch_spmv_csr(A, p, q, pow2_lanes((double)nnz / (double)m), 0, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_msg = std::string("launch of q = A p failed: ") + cudaGetErrorString(e);
    return LS_ERR_CUDA;
  }
  lsq::launch_spmv_csc(At, q, w, nullptr, lsq::DotSite{}, pow2_lanes((double)nnz / (double)n), 0, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_msg = std::string("launch of w = A^T q failed: ") + cudaGetErrorString(e);
    return LS_ERR_CUDA;
  }
  return LS_OK;
}
