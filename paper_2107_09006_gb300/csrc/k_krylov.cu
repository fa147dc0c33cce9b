// Sparse products with A and A^T, the CG vector updates with deterministic fused
// reductions, the overlap scatter-add with coarse prolongation, the coarse GEMV and
// the adjoint-gradient kernel.  All FP64.
//
// Reductions: every kernel that produces a dot product writes one partial sum per
// block; the consumer re-reduces the P partials in a fixed order in every block, so
// results do not depend on scheduling and CUDA-graph replays are bit-reproducible.
#include "common.cuh"
#include "kernels.h"

namespace lsq {

namespace {

__device__ __forceinline__ unsigned seg_mask(int V) {
  const int lane = threadIdx.x & 31;
  return V == 32 ? 0xffffffffu : (((1u << V) - 1u) << (lane / V * V));
}

// y = A x, V lanes per row (rows of A are short: a few stored entries each).
template <int V>
__global__ void __launch_bounds__(kThreads) k_spmv_csr(CsrDev A, const double* __restrict__ x,
                                                       double* __restrict__ y) {
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int sub = threadIdx.x % V;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x / V;
  const unsigned mask = seg_mask(V);
  for (int64_t r = gt / V; r < A.m; r += stride) {
    double acc = 0.0;
    const int64_t e1 = A.row_ptr[r + 1];
    for (int64_t e = A.row_ptr[r] + sub; e < e1; e += V) acc += __ldg(A.val + e) * __ldg(x + __ldg(A.col + e));
#pragma unroll
    for (int o = V / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(mask, acc, o);
    if (sub == 0) y[r] = acc;
  }
}

// w = A^T q through the CSC copy; optional fused partial sums of d . w.
template <int V>
__global__ void __launch_bounds__(kThreads) k_spmv_csc(CscDev At, const double* __restrict__ q,
                                                       double* __restrict__ w, const double* __restrict__ d,
                                                       double* __restrict__ part) {
  __shared__ double red[kWarps];
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int sub = threadIdx.x % V;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x / V;
  const unsigned mask = seg_mask(V);
  double dacc = 0.0;
  for (int64_t j = gt / V; j < At.n; j += stride) {
    double acc = 0.0;
    const int64_t e1 = At.col_ptr[j + 1];
    for (int64_t e = At.col_ptr[j] + sub; e < e1; e += V) acc += __ldg(At.val + e) * __ldg(q + __ldg(At.row + e));
#pragma unroll
    for (int o = V / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(mask, acc, o);
    if (sub == 0) {
      w[j] = acc;
      dacc += (d ? d[j] : acc) * acc;
    }
  }
  if (part) {
    const double s = block_sum(dacc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(kThreads) k_cg_update(int64_t n, int P, const double* __restrict__ part_pw,
                                                        const double* __restrict__ part_rz,
                                                        const double* __restrict__ p, const double* __restrict__ w,
                                                        double* __restrict__ x, double* __restrict__ r,
                                                        double* __restrict__ r_old, double* __restrict__ part_rr,
                                                        double* scal, int* ctr, double* alpha_hist, int cap) {
  __shared__ double red[kWarps];
  const double pw = reduce_partials(part_pw, P, red);
  const double rz = reduce_partials(part_rz, P, red);
  const double alpha = rz / pw;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    scal[S_RZOLD] = rz;
    scal[S_ALPHA] = alpha;
    const int it = *ctr;
    if (it >= 0 && it < cap) alpha_hist[it] = alpha;
    if (!(pw > 0.0) || !isfinite(alpha)) scal[S_FLAG] = 1.0;
  }
  double acc = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    x[k] += alpha * p[k];
    double rk = r[k];
    if (r_old) r_old[k] = rk;
    rk -= alpha * w[k];
    r[k] = rk;
    acc += rk * rk;
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) part_rr[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_p_update(int64_t n, int P, const double* __restrict__ part_rz,
                                                       const double* __restrict__ part_rzo,
                                                       const double* __restrict__ part_rr, double* scal,
                                                       int* ctr, double* beta_hist, int cap,
                                                       const double* __restrict__ z, double* __restrict__ p,
                                                       int init) {
  __shared__ double red[kWarps];
  double beta = 0.0;
  if (!init) {
    const double rz_new = reduce_partials(part_rz, P, red);
    const double num = part_rzo ? rz_new - reduce_partials(part_rzo, P, red) : rz_new;
    beta = num / scal[S_RZOLD];
  }
  if (blockIdx.x == 0 && !init) {
    const double rr = reduce_partials(part_rr, P, red);
    if (threadIdx.x == 0) {
      scal[S_RR] = rr;
      scal[S_BETA] = beta;
      const int it = *ctr;
      if (it >= 0 && it < cap) beta_hist[it] = beta;
      *ctr = it + 1;
      if (!isfinite(beta) || !isfinite(rr)) scal[S_FLAG] = 1.0;
    }
  }
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    p[k] = init ? z[k] : z[k] + beta * p[k];
}

__global__ void __launch_bounds__(kThreads) k_dot(int64_t n, const double* __restrict__ a,
                                                  const double* __restrict__ b, double* __restrict__ part) {
  __shared__ double red[kWarps];
  double acc = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    acc += a[k] * b[k];
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_finish_sum(const double* __restrict__ part, int P, double* out) {
  __shared__ double red[kWarps];
  const double s = reduce_partials(part, P, red);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_axpby(int64_t n, double alpha, const double* __restrict__ a, double beta,
                        const double* __restrict__ b, double* __restrict__ out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = alpha * a[k] + (b ? beta * b[k] : 0.0);
}

__global__ void k_fill(int64_t n, double v, double* __restrict__ out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = v;
}

// z_j = sum over the copies of column j in the subdomains (ascending subdomain order)
//     + sum_t Zbar_{part[j]}[t, jj(j)] y0[coff + t]          (coarse prolongation)
__global__ void __launch_bounds__(kThreads) k_scatter(ScatterArgs a) {
  __shared__ double red[kWarps];
  double acc_rz = 0.0, acc_rzo = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.n; j += (int64_t)gridDim.x * blockDim.x) {
    double z = 0.0;
    if (a.add_coarse_only != 1) {
      for (int64_t e = a.map_ptr[j]; e < a.map_ptr[j + 1]; ++e) z += a.y[a.map_idx[e]];
    }
    if (a.coarse && a.add_coarse_only != 2) {
      const int i = a.part[j];
      const int c0 = a.coff[i], k = a.coff[i + 1] - c0;
      const int64_t nIi = a.nI[i];
      const double* Zi = a.Z + a.zoff[i] + a.jj_of[j];
      for (int t = 0; t < k; ++t) z += Zi[t * nIi] * a.y0[c0 + t];
    }
    a.z[j] = z;
    if (a.part_rz) {
      acc_rz += a.r[j] * z;
      if (a.r_old) acc_rzo += a.r_old[j] * z;
    }
  }
  if (a.part_rz) {
    const double s = block_sum(acc_rz, red);
    if (threadIdx.x == 0) a.part_rz[blockIdx.x] = s;
    if (a.r_old) {
      const double s2 = block_sum(acc_rzo, red);
      if (threadIdx.x == 0) a.part_rzo[blockIdx.x] = s2;
    }
  }
}

// y0 = X r0 for the dense n0 x n0 coarse inverse (one warp per row).
__global__ void __launch_bounds__(kThreads) k_gemv(int64_t n0, const double* __restrict__ X,
                                                   const double* __restrict__ r0, double* __restrict__ y0) {
  const int lane = threadIdx.x & 31;
  const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = wg; row < n0; row += nw) {
    const double* xr = X + row * n0;
    double acc = 0.0;
    for (int64_t c = lane; c < n0; c += 32) acc += __ldg(xr + c) * __ldg(r0 + c);
    acc = warp_sum(acc);
    if (lane == 0) y0[row] = acc;
  }
}

// g[e] (+)= rho_r lam_c - mu_r x_c for every stored entry e = (r, c) of A.
__global__ void __launch_bounds__(kThreads) k_grad_vals(CsrDev A, const double* __restrict__ rho,
                                                        const double* __restrict__ lam,
                                                        const double* __restrict__ mu,
                                                        const double* __restrict__ x, double* __restrict__ g,
                                                        int accumulate) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < A.m; r += (int64_t)gridDim.x * blockDim.x) {
    const double rr = rho[r], mr = mu[r];
    for (int64_t e = A.row_ptr[r]; e < A.row_ptr[r + 1]; ++e) {
      const int32_t c = A.col[e];
      const double v = rr * lam[c] - mr * x[c];
      g[e] = accumulate ? g[e] + v : v;
    }
  }
}

int grid_for(int64_t work, int per_block, int cap) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace

void launch_spmv_csr(const CsrDev& A, const double* x, double* y, int lanes, cudaStream_t st) {
  const int grid = grid_for(A.m * lanes, kThreads, 1 << 16);
  switch (lanes) {
    case 1: k_spmv_csr<1><<<grid, kThreads, 0, st>>>(A, x, y); break;
    case 2: k_spmv_csr<2><<<grid, kThreads, 0, st>>>(A, x, y); break;
    case 4: k_spmv_csr<4><<<grid, kThreads, 0, st>>>(A, x, y); break;
    case 8: k_spmv_csr<8><<<grid, kThreads, 0, st>>>(A, x, y); break;
    case 16: k_spmv_csr<16><<<grid, kThreads, 0, st>>>(A, x, y); break;
    default: k_spmv_csr<32><<<grid, kThreads, 0, st>>>(A, x, y); break;
  }
}

void launch_spmv_csc(const CscDev& At, const double* q, double* w, const double* d, double* part,
                     int P, int lanes, cudaStream_t st) {
  // With partials the grid is exactly P blocks (the consumer reduces P entries).
  const int grid = part ? P : grid_for(At.n * lanes, kThreads, 1 << 16);
  switch (lanes) {
    case 1: k_spmv_csc<1><<<grid, kThreads, 0, st>>>(At, q, w, d, part); break;
    case 2: k_spmv_csc<2><<<grid, kThreads, 0, st>>>(At, q, w, d, part); break;
    case 4: k_spmv_csc<4><<<grid, kThreads, 0, st>>>(At, q, w, d, part); break;
    case 8: k_spmv_csc<8><<<grid, kThreads, 0, st>>>(At, q, w, d, part); break;
    case 16: k_spmv_csc<16><<<grid, kThreads, 0, st>>>(At, q, w, d, part); break;
    default: k_spmv_csc<32><<<grid, kThreads, 0, st>>>(At, q, w, d, part); break;
  }
}

void launch_cg_update(int64_t n, int P, const double* part_pw, const double* part_rz, const double* p,
                      const double* w, double* x, double* r, double* r_old, double* part_rr,
                      double* scal, int* ctr, double* alpha_hist, int hist_cap, cudaStream_t st) {
  k_cg_update<<<P, kThreads, 0, st>>>(n, P, part_pw, part_rz, p, w, x, r, r_old, part_rr, scal, ctr,
                                      alpha_hist, hist_cap);
}

void launch_p_update(int64_t n, int P, const double* part_rz, const double* part_rzo,
                     const double* part_rr, double* scal, int* ctr, double* beta_hist, int hist_cap,
                     const double* z, double* p, int init, cudaStream_t st) {
  k_p_update<<<P, kThreads, 0, st>>>(n, P, part_rz, part_rzo, part_rr, scal, ctr, beta_hist, hist_cap, z,
                                     p, init);
}

void launch_dot(int64_t n, const double* a, const double* b, double* part, int P, cudaStream_t st) {
  k_dot<<<P, kThreads, 0, st>>>(n, a, b, part);
}

void launch_finish_sum(const double* part, int P, double* out, cudaStream_t st) {
  k_finish_sum<<<1, kThreads, 0, st>>>(part, P, out);
}

void launch_axpby(int64_t n, double alpha, const double* a, double beta, const double* b, double* out,
                  cudaStream_t st) {
  k_axpby<<<grid_for(n, kThreads, 4096), kThreads, 0, st>>>(n, alpha, a, beta, b, out);
}

void launch_fill(int64_t n, double v, double* out, cudaStream_t st) {
  k_fill<<<grid_for(n, kThreads, 4096), kThreads, 0, st>>>(n, v, out);
}

void launch_scatter(const ScatterArgs& a, cudaStream_t st) {
  k_scatter<<<a.P, kThreads, 0, st>>>(a);
}

void launch_gemv(int64_t n0, const double* X, const double* r0, double* y0, cudaStream_t st) {
  if (n0 <= 0) return;
  k_gemv<<<grid_for(n0 * 32, kThreads, 8192), kThreads, 0, st>>>(n0, X, r0, y0);
}

void launch_grad_vals(const CsrDev& A, const double* rho, const double* lam, const double* mu,
                      const double* x, double* g, int accumulate, cudaStream_t st) {
  k_grad_vals<<<grid_for(A.m, kThreads, 8192), kThreads, 0, st>>>(A, rho, lam, mu, x, g, accumulate);
}

}  // namespace lsq
