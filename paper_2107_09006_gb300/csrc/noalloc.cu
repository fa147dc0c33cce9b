// Allocation-free normal-equations product w = A^T (A p).
//
// Some callers cannot call cudaMalloc: code that records its GPU work into a CUDA
// graph by stream capture (allocation calls are not capturable), code that runs inside
// a framework whose memory must all come from its own pool, and real-time loops that
// must not enter the CUDA memory allocator.  This entry point lets them apply the
// operator C = A^T A without the library allocating anything: the caller passes A in
// CSR and CSC form, p and w; the intermediate q = A p lives in a file-scope device
// array of fixed size, the same array for every call.
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

std::mutex g_mu;
double* g_q_addr[kMaxDevices] = {};

thread_local std::string g_msg;

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
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    g_msg = "no usable current device";
    return LS_ERR_CUDA;
  }
  double* q = nullptr;
  {
    // Once per device, with that device current: the device address of the scratch.
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_q_addr[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_q);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        g_msg = std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
        return LS_ERR_CUDA;
      }
      g_q_addr[dev] = static_cast<double*>(ptr);
    }
    q = g_q_addr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const lsq::CsrDev A{m, n, row_ptr, col, val};
  const lsq::CscDev At{m, n, col_ptr, row, cval};
  lsq::launch_spmv_csr(A, p, q, pow2_lanes((double)nnz / (double)m), 0, st);
  lsq::launch_spmv_csc(At, q, w, nullptr, lsq::DotSite{}, pow2_lanes((double)nnz / (double)n), 0, st);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_msg = std::string("launch failed: ") + cudaGetErrorString(e);
    return LS_ERR_CUDA;
  }
  return LS_OK;
}
