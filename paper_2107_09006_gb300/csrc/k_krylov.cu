// Sparse products with A and A^T, the CG vector updates, the overlap scatter-add with
// coarse prolongation, the coarse GEMV and the adjoint-gradient kernel.  All FP64.
//
// Reductions: a kernel that produces a dot product writes one partial sum per block;
// the last block to finish (an atomic ticket after a memory fence, no waiting) sums
// the partials in block order and stores the scalar into a slot of the device CG
// state.  The result does not depend on scheduling, so CUDA-graph replays are
// bit-reproducible, and consumers read one scalar.
#include "common.cuh"
#include "kernels.h"
#include "normal_tiles.h"

namespace lsq {

namespace {

__device__ __forceinline__ unsigned seg_mask(int V) {
  const int lane = threadIdx.x & 31;
  return V == 32 ? 0xffffffffu : (((1u << V) - 1u) << (lane / V * V));
}

// Block partials -> last block sums them in order -> *out (and a second sum if two).
__device__ __forceinline__ void finish_dots(double s1, double s2, bool two, const DotSite& d) {
  __shared__ double red[kWarps];
  __shared__ bool last;
  const double b1 = block_sum(s1, red);
  const double b2 = two ? block_sum(s2, red) : 0.0;
  if (threadIdx.x == 0) {
    d.parts[blockIdx.x] = b1;
    if (two) d.parts[d.stride + blockIdx.x] = b2;
    __threadfence();
    const unsigned t = atomicAdd(d.counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double a1 = 0.0, a2 = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
      a1 += ((volatile double*)d.parts)[k];
      if (two) a2 += ((volatile double*)d.parts)[d.stride + k];
    }
    a1 = block_sum(a1, red);
    if (two) a2 = block_sum(a2, red);
    if (threadIdx.x == 0) {
      d.out[0] = a1;
      if (two) d.out[d.out2] = a2;
      *d.counter = 0u;
    }
  }
}

// y = A x, V lanes per row.  Each lane group walks its row with stride V; rows of a
// few entries use small V so more rows are in flight per warp.
template <int V>
__global__ void __launch_bounds__(kThreads) k_spmv_csr(CsrDev A, const double* __restrict__ x,
                                                       double* __restrict__ y) {
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int sub = threadIdx.x % V;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x / V;
  const unsigned mask = seg_mask(V);
  for (int64_t r = gt / V; r < A.m; r += stride) {
    double acc = 0.0;
    const int64_t e0 = __ldg(A.row_ptr + r), e1 = __ldg(A.row_ptr + r + 1);
#pragma unroll 4
    for (int64_t e = e0 + sub; e < e1; e += V) acc += __ldg(A.val + e) * __ldg(x + __ldg(A.col + e));
#pragma unroll
    for (int o = V / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(mask, acc, o);
    if (sub == 0) y[r] = acc;
  }
}

// w = A^T q through the CSC copy; optionally d.w into the dot site (d = w if null).
template <int V>
__global__ void __launch_bounds__(kThreads) k_spmv_csc(CscDev At, const double* __restrict__ q,
                                                       double* __restrict__ w, const double* __restrict__ d,
                                                       DotSite ds) {
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int sub = threadIdx.x % V;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x / V;
  const unsigned mask = seg_mask(V);
  double dacc = 0.0;
  for (int64_t j = gt / V; j < At.n; j += stride) {
    double acc = 0.0;
    const int64_t e0 = __ldg(At.col_ptr + j), e1 = __ldg(At.col_ptr + j + 1);
#pragma unroll 4
    for (int64_t e = e0 + sub; e < e1; e += V) acc += __ldg(At.val + e) * __ldg(q + __ldg(At.row + e));
#pragma unroll
    for (int o = V / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(mask, acc, o);
    if (sub == 0) {
      w[j] = acc;
      dacc += (d ? d[j] : acc) * acc;
    }
  }
  if (ds.parts) finish_dots(dacc, 0.0, false, ds);
}

// Warp-stream product y = B x for a CSR matrix B (A itself, or A^T through the CSC copy):
// each warp takes R consecutive rows, loads all their entries coalesced (lanes stride the
// entry range, all loads independent), keeps the products in shared memory, then lane k
// sums row k in storage order.  Row blocks whose entries exceed CAP fall back to one
// warp per row.  Optional fused d . y as in k_spmv_csc.
template <int R, int CAP>
__global__ void __launch_bounds__(kThreads) k_spmv_stream(int64_t nrows, const int64_t* __restrict__ ptr,
                                                          const int32_t* __restrict__ idx,
                                                          const double* __restrict__ val,
                                                          const double* __restrict__ x, double* __restrict__ y,
                                                          const double* __restrict__ d, DotSite ds) {
  __shared__ double prod[kWarps][CAP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double* sm = prod[w];
  double dacc = 0.0;
  const int64_t nblk = (nrows + R - 1) / R;
  for (int64_t rb = (int64_t)blockIdx.x * kWarps + w; rb < nblk; rb += (int64_t)gridDim.x * kWarps) {
    const int64_t r0 = rb * R;
    const int64_t r = r0 + lane;
    const bool mine = lane < R && r < nrows;
    const int64_t plo = __ldg(ptr + (mine ? r : min(r0 + R, nrows)));
    const int64_t rend = min(r0 + R, nrows);
    const int64_t e1 = __ldg(ptr + rend);
    const int64_t e0 = __shfl_sync(0xffffffffu, plo, 0);
    const int64_t phi = __shfl_down_sync(0xffffffffu, plo, 1);
    const int64_t my_hi = (lane == R - 1 || r + 1 >= rend) ? e1 : phi;
    if (e1 - e0 <= CAP) {
#pragma unroll 4
      for (int64_t e = e0 + lane; e < e1; e += 32) sm[e - e0] = __ldg(val + e) * __ldg(x + __ldg(idx + e));
      __syncwarp();
      if (mine) {
        double s = 0.0;
        for (int64_t e = plo; e < my_hi; ++e) s += sm[e - e0];
        y[r] = s;
        dacc += (d ? d[r] : s) * s;
      }
      __syncwarp();
    } else {
      for (int64_t rr = r0; rr < rend; ++rr) {
        const int64_t a0 = __ldg(ptr + rr), a1 = __ldg(ptr + rr + 1);
        double s = 0.0;
        for (int64_t e = a0 + lane; e < a1; e += 32) s += __ldg(val + e) * __ldg(x + __ldg(idx + e));
        s = warp_sum(s);
        if (lane == 0) {
          y[rr] = s;
          dacc += (d ? d[rr] : s) * s;
        }
      }
    }
  }
  if (ds.parts) finish_dots(dacc, 0.0, false, ds);
}

// Sliced-ELL product: one warp per slice of 32 rows, lane l owns slice row l; every
// step k loads 32 consecutive (column, value) pairs, so there is no per-row pointer
// chase and the gathers of successive k are independent.
__global__ void __launch_bounds__(kThreads) k_spmv_sell(SellDev S, const double* __restrict__ x,
                                                        double* __restrict__ y, const double* __restrict__ d,
                                                        DotSite ds) {
  const int lane = threadIdx.x & 31;
  double dacc = 0.0;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < S.nslices;
       s += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t o = __ldg(S.off + s);
    const int W = (int)((__ldg(S.off + s + 1) - o) >> 5);
    const int r = __ldg(S.perm + s * 32 + lane);
    const int32_t* cp = S.col + o + lane;
    const double* vp = S.val + o + lane;
    double acc = 0.0;
#pragma unroll 8
    for (int k = 0; k < W; ++k) acc += __ldg(vp + 32 * k) * __ldg(x + __ldg(cp + 32 * k));
    if (r >= 0) {
      y[r] = acc;
      dacc += (d ? d[r] : acc) * acc;
    }
  }
  if (ds.parts) finish_dots(dacc, 0.0, false, ds);
}

// alpha = rz / pw; x += alpha p; r_old = r; r -= alpha w; rr = r.r
__global__ void __launch_bounds__(kThreads) k_cg_update(int64_t n, double* scal, const double* __restrict__ p,
                                                        const double* __restrict__ w, double* __restrict__ x,
                                                        double* __restrict__ r, double* __restrict__ r_old,
                                                        DotSite rr, int* ctr, double* alpha_hist, int cap) {
  const double rz = scal[S_RZ], pw = scal[S_PW];
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
  finish_dots(acc, 0.0, false, rr);
}

// beta = rz_new / rz_old (or (rz_new - rzo_new) / rz_old, flexible); p = z + beta p.
__global__ void __launch_bounds__(kThreads) k_p_update(int64_t n, double* scal, int* ctr, double* beta_hist,
                                                       int cap, const double* __restrict__ z, double* __restrict__ p,
                                                       int init, int flex) {
  double beta = 0.0;
  if (!init) {
    const double num = flex ? scal[S_RZ] - scal[S_RZO] : scal[S_RZ];
    beta = num / scal[S_RZOLD];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      scal[S_BETA] = beta;
      const int it = *ctr;
      if (it >= 0 && it < cap) beta_hist[it] = beta;
      *ctr = it + 1;
      scal[S_ITS] = (double)(it + 1);
      if (!isfinite(beta)) scal[S_FLAG] = 1.0;
    }
  }
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    p[k] = init ? z[k] : z[k] + beta * p[k];
}

__global__ void k_cg_continue(const double* scal, const int* ctr, int limit, cudaGraphConditionalHandle hnd) {
  const double rr = scal[S_RR], thr = scal[S_THR];
  bool go = scal[S_FLAG] == 0.0 && scal[S_ERR] == 0.0 && isfinite(rr) && *ctr < limit;
  if (thr > 0.0 && rr <= thr) go = false;
  cudaGraphSetConditional(hnd, go ? 1u : 0u);
}

__global__ void k_stamp(unsigned long long* stamps, const int* ctr, int cap, int k, int after) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  const int slot = *ctr - after;
  if (slot >= 0 && slot < cap) stamps[(int64_t)slot * 8 + k] = t;
}

__global__ void __launch_bounds__(kThreads) k_dot(int64_t n, const double* __restrict__ a,
                                                  const double* __restrict__ b, DotSite ds) {
  double acc = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    acc += a[k] * b[k];
  finish_dots(acc, 0.0, false, ds);
}

__global__ void k_axpby(int64_t n, double alpha, const double* __restrict__ a, double beta,
                        const double* __restrict__ b, double* __restrict__ out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = alpha * a[k] + (b ? beta * b[k] : 0.0);
}

__global__ void k_gather(int64_t n, const int32_t* __restrict__ idx, const double* __restrict__ src,
                         double* __restrict__ dst) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = src[idx[k]];
}

__global__ void k_gather64(int64_t n, const int64_t* __restrict__ idx, const double* __restrict__ src,
                           double* __restrict__ dst) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = idx[k];
    dst[k] = t >= 0 ? src[t] : 0.0;
  }
}

__global__ void k_scatter_idx(int64_t n, const int32_t* __restrict__ i32, const int64_t* __restrict__ i64,
                              const double* __restrict__ src, double* __restrict__ dst, int accumulate) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = i32 ? (int64_t)i32[k] : i64[k];
    dst[t] = accumulate ? dst[t] + src[k] : src[k];
  }
}

__global__ void k_fill(int64_t n, double v, double* __restrict__ out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = v;
}

// z_j = sum over the copies of column j in the subdomains (ascending subdomain order)
//     + sum_t Zbar_{part[j]}[t, jj(j)] y0[coff + t]          (coarse prolongation)
__global__ void __launch_bounds__(kThreads) k_scatter(ScatterArgs a) {
  double acc_rz = 0.0, acc_rzo = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.n; j += (int64_t)gridDim.x * blockDim.x) {
    double z = 0.0;
    if (a.add_coarse_only != 1) {
      for (int64_t e = a.map_ptr[j]; e < a.map_ptr[j + 1]; ++e)
        if (in_range(a.map_idx[e], a.total_local, a.err)) z += a.y[a.map_idx[e]];
    }
    if (a.coarse && a.add_coarse_only != 2) {
      const int i = a.part[j];
      const int c0 = a.coff[i], k = a.coff[i + 1] - c0;
      const int64_t nIi = a.nI[i];
      const double* Zi = a.Z + a.zoff[i] + a.jj_of[j];
      for (int t = 0; t < k; ++t) z += Zi[t * nIi] * a.y0[c0 + t];
    }
    a.z[j] = z;
    if (a.dots.parts) {
      acc_rz += a.r[j] * z;
      if (a.r_old) acc_rzo += a.r_old[j] * z;
    }
  }
  if (a.dots.parts) finish_dots(acc_rz, acc_rzo, a.r_old != nullptr, a.dots);
}

// r0[c0 + t] = sum_jj Zbar_i[t, jj] v[Omega_I,i[jj]] (one block per subdomain, one warp
// per coarse vector): the coarse restriction R_0 v on its own.
__global__ void __launch_bounds__(kThreads) k_restrict(const int64_t* __restrict__ int_off,
                                                       const int32_t* __restrict__ int_glob,
                                                       const int64_t* __restrict__ zoff,
                                                       const int32_t* __restrict__ coff, const double* __restrict__ Z,
                                                       const double* __restrict__ v, double* __restrict__ r0) {
  const int i = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c0 = coff[i], kk = coff[i + 1] - c0;
  const int64_t io = int_off[i];
  const int64_t nIi = int_off[i + 1] - io;
  const double* Zi = Z + zoff[i];
  for (int t = w; t < kk; t += kWarps) {
    double acc = 0.0;
    for (int64_t jj = lane; jj < nIi; jj += 32) acc += Zi[(int64_t)t * nIi + jj] * v[int_glob[io + jj]];
    acc = warp_sum(acc);
    if (lane == 0) r0[c0 + t] = acc;
  }
}

// z = a + b - c with the fused dots r.z (and r_old.z) of the preconditioned residual.
__global__ void __launch_bounds__(kThreads) k_combine3(int64_t n, const double* __restrict__ a,
                                                       const double* __restrict__ b, const double* __restrict__ c,
                                                       double* __restrict__ z, const double* __restrict__ r,
                                                       const double* __restrict__ r_old, DotSite ds) {
  double d1 = 0.0, d2 = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double v = a[k] + b[k] - c[k];
    z[k] = v;
    if (ds.parts) {
      d1 += r[k] * v;
      if (r_old) d2 += r_old[k] * v;
    }
  }
  if (ds.parts) finish_dots(d1, d2, r_old != nullptr, ds);
}

// The vector updates of one preconditioned LSQR step: v = t / alpha, q = s / alpha
// (q = M v), x += c1 w, w = v - c2 w.
__global__ void __launch_bounds__(kThreads) k_lsqr_step(int64_t n, double inv_alpha, double c1, double c2,
                                                        const double* __restrict__ t, const double* __restrict__ s,
                                                        double* __restrict__ v, double* __restrict__ q,
                                                        double* __restrict__ x, double* __restrict__ w) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double vk = t[k] * inv_alpha;
    v[k] = vk;
    q[k] = s[k] * inv_alpha;
    const double wk = w[k];
    x[k] += c1 * wk;
    w[k] = vk - c2 * wk;
  }
}

// RAS prolongation: z_j = a_j + y[own[j]] (a may be null), the local solution of the
// subdomain that owns column j only.
__global__ void __launch_bounds__(kThreads) k_ras_combine(int64_t n, const int64_t* __restrict__ own,
                                                          const double* __restrict__ y, const double* __restrict__ a,
                                                          double* __restrict__ z) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    z[j] = (a ? a[j] : 0.0) + y[own[j]];
}

// Per-block partial dots of the k columns of V (column-major, leading dimension ld)
// with w: part[c * gridDim.x + block] (one column after another, block-wide sums).
__global__ void __launch_bounds__(kThreads) k_multi_dot(int64_t n, const double* __restrict__ V, int64_t ld, int k,
                                                        const double* __restrict__ w, double* __restrict__ part) {
  __shared__ double red[kWarps];
  for (int c = 0; c < k; ++c) {
    double acc = 0.0;
    const double* v = V + (int64_t)c * ld;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
      acc += v[r] * w[r];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) part[(int64_t)c * gridDim.x + blockIdx.x] = acc;
  }
}

// out[c] = sum of column c's partials in block order (one block per column).
__global__ void __launch_bounds__(kThreads) k_multi_dot_finish(int nparts, const double* __restrict__ part,
                                                               double* __restrict__ out) {
  __shared__ double red[kWarps];
  const int c = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) acc += part[(int64_t)c * nparts + b];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) out[c] = acc;
}

// out += sign * V coef over the k columns of V (column-major, leading dimension ld).
__global__ void __launch_bounds__(kThreads) k_multi_axpy(int64_t n, const double* __restrict__ V, int64_t ld, int k,
                                                         const double* __restrict__ coef, double sign,
                                                         double* __restrict__ out) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < k; ++c) acc += V[(int64_t)c * ld + r] * coef[c];
    out[r] += sign * acc;
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

// One-pass normal product, part 1: one block per row tile (layout in normal_tiles.h).
// The tile's window of p is loaded into shared memory; each warp then takes row slices
// (32 rows, lane l row l, entry k of every lane in one coalesced load) and leaves
// s_j = a_j . p in shared memory; after a barrier each warp takes column slices (32
// window columns) and forms u_c = sum_j a_jc s_j over the tile's rows, written over the p
// window; the window goes to the tile's partial buffer.  Both sums run in storage
// order.  The two sweeps read each stored entry once and gather only from shared memory.
//
// The sweeps are bound by the latency of the entry loads: a warp takes P adjacent slices
// at a time and issues up to 8 entry loads of each before the first FMA, and it loads the
// slice offsets of its next group while the current group's entries are in flight.
// Configurations (option normal_kernel): 512 threads with P = 1, 2, 3, or 1,024 threads
// with P = 1.  Slices are stored heaviest first; each warp starts on the group of its
// index and then claims the next unclaimed group from a shared counter, so the warps
// of a sweep finish close together.

// One sweep over slices [s_begin, s_end): acc = sum_k val[.] * src[idx[.]] per lane; the
// result of slice s goes to dst[(s - s_begin) * 32 + lane] (cid == nullptr) or to
// dst[cid[s * 32 + lane]] (lanes with cid 0xFFFF write nothing).
template <int P, int NT>
__device__ __forceinline__ void normal_sweep(const int64_t* __restrict__ off, const uint16_t* __restrict__ idx,
                                             const double* __restrict__ val, const uint16_t* __restrict__ cid,
                                             int s_begin, int s_end, const double* src, int src_n, double* dst,
                                             int dst_n, int* claim, double* err) {
  const int lane = threadIdx.x & 31;
  const int ng = (s_end - s_begin + P - 1) / P;
  int64_t o[P + 1], no[P + 1];
  auto load_off = [&](int g, int64_t(&oo)[P + 1]) {
#pragma unroll
    for (int q = 0; q <= P; ++q) oo[q] = __ldg(off + min(s_begin + g * P + q, s_end));
  };
  int g = threadIdx.x >> 5;
  if (g < ng) load_off(g, o);
  while (g < ng) {
    int nxt = 0;
    if (lane == 0) nxt = atomicAdd(claim, 1);
    nxt = __shfl_sync(0xffffffffu, nxt, 0);
    int K[P], Kmax = 0;
#pragma unroll
    for (int q = 0; q < P; ++q) {
      K[q] = (int)((o[q + 1] - o[q]) >> 5);
      Kmax = max(Kmax, K[q]);
    }
    double acc[P];
#pragma unroll
    for (int q = 0; q < P; ++q) acc[q] = 0.0;
    const bool more = nxt < ng;
    for (int k0 = 0; k0 < Kmax || k0 == 0; k0 += 8) {
      int c[P][8];
      double v[P][8];
#pragma unroll
      for (int q = 0; q < P; ++q)
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const bool ok = k0 + u < K[q];
          const int64_t e = o[q] + lane + 32 * (k0 + u);
          c[q][u] = ok ? (int)__ldg(idx + e) : 0;
          v[q][u] = ok ? __ldg(val + e) : 0.0;
        }
      if (k0 == 0 && more) load_off(nxt, no);
#pragma unroll
      for (int q = 0; q < P; ++q)
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (k0 + u < K[q] && in_range(c[q][u], src_n, err)) acc[q] = fma(v[q][u], src[c[q][u]], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int s = s_begin + g * P + q;
      if (s >= s_end) break;
      if (!cid) {
        dst[(s - s_begin) * 32 + lane] = acc[q];
      } else {
        const int c = __ldg(cid + (int64_t)s * 32 + lane);
        if (c != 0xFFFF && in_range(c, dst_n, err)) dst[c] = acc[q];
      }
    }
    if (more) {
#pragma unroll
      for (int q = 0; q <= P; ++q) o[q] = no[q];
    }
    g = nxt;
  }
}

template <int P, int NT>
__global__ void __launch_bounds__(NT, 1) k_normal_tile(NormalTilesDev T, const double* __restrict__ p) {
  extern __shared__ __align__(16) double nsm[];
  __shared__ int claim[2];
  const int t = blockIdx.x;
  if (threadIdx.x == 0) claim[0] = claim[1] = NT / 32;
  const int64_t lo = __ldg(T.lo + t);
  const int W = __ldg(T.wid + t);
  const int a0 = __ldg(T.as0 + t), a1 = __ldg(T.as0 + t + 1);
  const int b0 = __ldg(T.bs0 + t), b1 = __ldg(T.bs0 + t + 1);
  double* pw = nsm;
  double* sv = nsm + ((W + 1) & ~1);
  for (int i = threadIdx.x; i < W; i += NT) pw[i] = __ldg(p + lo + i);
  __syncthreads();
  normal_sweep<P, NT>(T.aoff, T.acol, T.aval, nullptr, a0, a1, pw, W, sv, (a1 - a0) * 32, claim, T.err);
  __syncthreads();
  normal_sweep<P, NT>(T.boff, T.brow, T.bval, T.bcid, b0, b1, sv, (a1 - a0) * 32, pw, W, claim + 1, T.err);
  __syncthreads();
  double* out = T.part + __ldg(T.poff + t);
  for (int i = threadIdx.x; i < W; i += NT) out[i] = pw[i];
}

// Part 2: w_c = sum of the partial windows that hold column c, in tile order (the tiles
// to look at come from the table of each block of kNormalColBlock columns), with the
// fused d . w.
__global__ void __launch_bounds__(kThreads) k_normal_reduce(NormalTilesDev T, double* __restrict__ w,
                                                            const double* __restrict__ d, DotSite ds) {
  double dacc = 0.0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < T.n; c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = c / kNormalColBlock;
    const int t0 = __ldg(T.cb_t0 + b), t1 = __ldg(T.cb_t1 + b);
    double acc = 0.0;
    for (int t = t0; t <= t1; ++t) {
      const int64_t off = c - __ldg(T.lo + t);
      if (off >= 0 && off < __ldg(T.wid + t)) acc += T.part[__ldg(T.poff + t) + off];
    }
    w[c] = acc;
    dacc += (d ? d[c] : acc) * acc;
  }
  if (ds.parts) finish_dots(dacc, 0.0, false, ds);
}

int grid_for(int64_t work, int per_block, int cap) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace

void launch_spmv_csr(const CsrDev& A, const double* x, double* y, int lanes, int grid, cudaStream_t st) {
  if (lanes == -2) {
    if (grid <= 0) grid = grid_for(A.sell.nslices, kWarps, kMaxGrid);
    k_spmv_sell<<<grid, kThreads, 0, st>>>(A.sell, x, y, nullptr, DotSite{});
    return;
  }
  if (lanes < 0) {
    const int R = lanes == -3 ? 32 : 16;
    if (grid <= 0) grid = grid_for((A.m + R - 1) / R, kWarps, kMaxGrid);
    if (lanes == -3) k_spmv_stream<32, 512><<<grid, kThreads, 0, st>>>(A.m, A.row_ptr, A.col, A.val, x, y, nullptr, DotSite{});
    else k_spmv_stream<16, 768><<<grid, kThreads, 0, st>>>(A.m, A.row_ptr, A.col, A.val, x, y, nullptr, DotSite{});
    return;
  }
  if (grid <= 0) grid = grid_for(A.m * lanes, kThreads, kMaxGrid);
  switch (lanes) {
    case 1: k_spmv_csr<1><<<grid, kThreads, 0, st>>>(A, x, y); break;
    case 2: k_spmv_csr<2><<<grid, kThreads, 0, st>>>(A, x, y); break;
    case 4: k_spmv_csr<4><<<grid, kThreads, 0, st>>>(A, x, y); break;
    case 8: k_spmv_csr<8><<<grid, kThreads, 0, st>>>(A, x, y); break;
    case 16: k_spmv_csr<16><<<grid, kThreads, 0, st>>>(A, x, y); break;
    default: k_spmv_csr<32><<<grid, kThreads, 0, st>>>(A, x, y); break;
  }
}

void launch_spmv_csc(const CscDev& At, const double* q, double* w, const double* d, const DotSite& ds, int lanes,
                     int grid, cudaStream_t st) {
  if (lanes == -2) {
    if (grid <= 0) grid = grid_for(At.sell.nslices, kWarps, kMaxGrid);
    k_spmv_sell<<<grid, kThreads, 0, st>>>(At.sell, q, w, d, ds);
    return;
  }
  if (lanes < 0) {
    const int R = lanes == -3 ? 32 : 16;
    if (grid <= 0) grid = grid_for((At.n + R - 1) / R, kWarps, kMaxGrid);
    if (lanes == -3) k_spmv_stream<32, 512><<<grid, kThreads, 0, st>>>(At.n, At.col_ptr, At.row, At.val, q, w, d, ds);
    else k_spmv_stream<16, 768><<<grid, kThreads, 0, st>>>(At.n, At.col_ptr, At.row, At.val, q, w, d, ds);
    return;
  }
  if (grid <= 0) grid = grid_for(At.n * lanes, kThreads, kMaxGrid);
  switch (lanes) {
    case 1: k_spmv_csc<1><<<grid, kThreads, 0, st>>>(At, q, w, d, ds); break;
    case 2: k_spmv_csc<2><<<grid, kThreads, 0, st>>>(At, q, w, d, ds); break;
    case 4: k_spmv_csc<4><<<grid, kThreads, 0, st>>>(At, q, w, d, ds); break;
    case 8: k_spmv_csc<8><<<grid, kThreads, 0, st>>>(At, q, w, d, ds); break;
    case 16: k_spmv_csc<16><<<grid, kThreads, 0, st>>>(At, q, w, d, ds); break;
    default: k_spmv_csc<32><<<grid, kThreads, 0, st>>>(At, q, w, d, ds); break;
  }
}

bool normal_tiles_prepare(const NormalTilesDev& T) {
  const size_t bytes = (size_t)T.smem_doubles * sizeof(double);
  int dev = 0, cap = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
  // Each configuration's limit is the device's (less its static shared memory), not this
  // matrix's need: handles of other matrices share the kernels.
  auto allow = [&](const void* fn) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return false;
    const int dyn = cap - (int)fa.sharedSizeBytes;
    if (bytes > (size_t)dyn) return false;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) == cudaSuccess;
  };
  const bool ok = allow((const void*)k_normal_tile<1, 512>) && allow((const void*)k_normal_tile<2, 512>) &&
                  allow((const void*)k_normal_tile<3, 512>) && allow((const void*)k_normal_tile<1, 1024>);
  if (!ok) cudaGetLastError();  // a refused setting leaves no error behind: the two products run instead
  return ok;
}

void launch_normal_tiles(const NormalTilesDev& T, const double* v, double* w, const double* d, const DotSite& ds,
                         cudaStream_t st) {
  const size_t smem = (size_t)T.smem_doubles * sizeof(double);
  if (T.ntiles > 0) {
    switch (T.config) {
      case 2: k_normal_tile<2, 512><<<T.ntiles, 512, smem, st>>>(T, v); break;
      case 3: k_normal_tile<3, 512><<<T.ntiles, 512, smem, st>>>(T, v); break;
      case 4: k_normal_tile<1, 1024><<<T.ntiles, 1024, smem, st>>>(T, v); break;
      default: k_normal_tile<1, 512><<<T.ntiles, 512, smem, st>>>(T, v); break;
    }
  }
  k_normal_reduce<<<grid_for(T.n, kThreads, kVecGrid), kThreads, 0, st>>>(T, w, d, ds);
}

void launch_cg_update(int64_t n, double* scal, const double* p, const double* w, double* x, double* r, double* r_old,
                      const DotSite& rr, int* ctr, double* alpha_hist, int hist_cap, cudaStream_t st) {
  k_cg_update<<<grid_for(n, kThreads, kVecGrid), kThreads, 0, st>>>(n, scal, p, w, x, r, r_old, rr, ctr, alpha_hist,
                                                                    hist_cap);
}

void launch_p_update(int64_t n, double* scal, int* ctr, double* beta_hist, int hist_cap, const double* z, double* p,
                     int init, int flex, cudaStream_t st) {
  k_p_update<<<grid_for(n, kThreads, kVecGrid), kThreads, 0, st>>>(n, scal, ctr, beta_hist, hist_cap, z, p, init,
                                                                   flex);
}

void launch_cg_continue(const double* scal, const int* ctr, int limit, cudaGraphConditionalHandle hnd,
                        cudaStream_t st) {
  k_cg_continue<<<1, 1, 0, st>>>(scal, ctr, limit, hnd);
}

void launch_stamp(unsigned long long* stamps, const int* ctr, int cap, int k, int after, cudaStream_t st) {
  k_stamp<<<1, 1, 0, st>>>(stamps, ctr, cap, k, after);
}

void launch_dot(int64_t n, const double* a, const double* b, const DotSite& ds, cudaStream_t st) {
  k_dot<<<grid_for(n, kThreads, kVecGrid), kThreads, 0, st>>>(n, a, b, ds);
}

void launch_axpby(int64_t n, double alpha, const double* a, double beta, const double* b, double* out,
                  cudaStream_t st) {
  k_axpby<<<grid_for(n, kThreads, kVecGrid), kThreads, 0, st>>>(n, alpha, a, beta, b, out);
}

void launch_fill(int64_t n, double v, double* out, cudaStream_t st) {
  k_fill<<<grid_for(n, kThreads, kVecGrid), kThreads, 0, st>>>(n, v, out);
}

void launch_gather(int64_t n, const int32_t* idx, const double* src, double* dst, cudaStream_t st) {
  k_gather<<<grid_for(n, kThreads, kVecGrid), kThreads, 0, st>>>(n, idx, src, dst);
}

void launch_gather64(int64_t n, const int64_t* idx, const double* src, double* dst, cudaStream_t st) {
  if (n <= 0) return;
  k_gather64<<<grid_for(n, kThreads, kVecGrid), kThreads, 0, st>>>(n, idx, src, dst);
}

void launch_scatter_idx(int64_t n, const int32_t* idx32, const int64_t* idx64, const double* src, double* dst,
                        int accumulate, cudaStream_t st) {
  k_scatter_idx<<<grid_for(n, kThreads, kVecGrid), kThreads, 0, st>>>(n, idx32, idx64, src, dst, accumulate);
}

void launch_lsqr_step(int64_t n, double inv_alpha, double c1, double c2, const double* t, const double* s, double* v,
                      double* q, double* x, double* w, cudaStream_t st) {
  k_lsqr_step<<<grid_for(n, kThreads, kVecGrid), kThreads, 0, st>>>(n, inv_alpha, c1, c2, t, s, v, q, x, w);
}

void launch_ras_combine(int64_t n, const int64_t* own, const double* y, const double* a, double* z, cudaStream_t st) {
  k_ras_combine<<<grid_for(n, kThreads, kVecGrid), kThreads, 0, st>>>(n, own, y, a, z);
}

int multi_dot_grid(int64_t n) { return grid_for(n, kThreads * 4, kVecGrid); }

void launch_multi_dot(int64_t n, const double* V, int64_t ld, int k, const double* w, double* part, double* out,
                      cudaStream_t st) {
  const int g = multi_dot_grid(n);
  k_multi_dot<<<g, kThreads, 0, st>>>(n, V, ld, k, w, part);
  k_multi_dot_finish<<<k, kThreads, 0, st>>>(g, part, out);
}

void launch_multi_axpy(int64_t n, const double* V, int64_t ld, int k, const double* coef, double sign, double* out,
                       cudaStream_t st) {
  k_multi_axpy<<<grid_for(n, kThreads, kVecGrid), kThreads, 0, st>>>(n, V, ld, k, coef, sign, out);
}

void launch_restrict(int N, const int64_t* int_off, const int32_t* int_glob, const int64_t* zoff, const int32_t* coff,
                     const double* Z, const double* v, double* r0, cudaStream_t st) {
  k_restrict<<<N, kThreads, 0, st>>>(int_off, int_glob, zoff, coff, Z, v, r0);
}

void launch_combine3(int64_t n, const double* a, const double* b, const double* c, double* z, const double* r,
                     const double* r_old, const DotSite& ds, cudaStream_t st) {
  k_combine3<<<grid_for(n, kThreads, kVecGrid), kThreads, 0, st>>>(n, a, b, c, z, r, r_old, ds);
}

void launch_scatter(const ScatterArgs& a, cudaStream_t st) {
  k_scatter<<<grid_for(a.n, kThreads, kVecGrid), kThreads, 0, st>>>(a);
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
