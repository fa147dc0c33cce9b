// Local matrices in block-envelope storage: assembly of C_ii and C~_ii, the shifts of
// Section 4.1.2, batched Cholesky (one CTA per subdomain, left-looking over 32x32
// tiles) and the batched local solves of the preconditioner apply.
#include "band.cuh"
#include "tile.cuh"
#include "kernels.h"

namespace lsq {

namespace {

__device__ __forceinline__ int lower_bound_i32(const int32_t* a, int n, int32_t key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// One thread per local row k of subdomain i: row k of C_ii = sum over the rows r of A
// that touch column Omega_i[k] of a_{r,k} a_{r,q} (q in Omega_i, q <= k); the rows
// of Xi_i (those touching an interior column) also go to C~_ii (eq. (3.2)).
__global__ void __launch_bounds__(kThreads) k_assemble(BandPlan P, CsrDev A, CscDev At,
                                                       const int32_t* __restrict__ part, int64_t total,
                                                       double* __restrict__ C, double* __restrict__ Ct) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = P.row_sub[e];
    const int64_t o0 = P.om_off[i];
    const int ni = (int)(P.om_off[i + 1] - o0);
    const int k = (int)(e - o0);
    const int32_t* om = P.om_glob + o0;
    const int b = k >> 5, rr = k & 31;
    const int64_t bi = P.blk_off[i] + b;
    const int t0 = P.blk_tf[bi];
    const int width = (b - t0 + 1) * kT;
    const int64_t rowoff = P.blk_poff[bi] + (int64_t)rr * width - (int64_t)t0 * kT;
    const int32_t g = om[k];
    for (int64_t e2 = At.col_ptr[g]; e2 < At.col_ptr[g + 1]; ++e2) {
      const int32_t r = At.row[e2];
      const double arg = At.val[e2];
      const int64_t s0 = A.row_ptr[r], s1 = A.row_ptr[r + 1];
      bool inxi = false;
      for (int64_t s = s0; s < s1; ++s)
        if (part[A.col[s]] == i) { inxi = true; break; }
      for (int64_t s = s0; s < s1; ++s) {
        const int32_t c = A.col[s];
        const int q = lower_bound_i32(om, ni, c);
        if (q < ni && om[q] == c && q <= k) {
          const double v = arg * A.val[s];
          C[rowoff + q] += v;
          if (inxi) Ct[rowoff + q] += v;
        }
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_norms(BandPlan P, const double* __restrict__ C,
                                                    const double* __restrict__ Ct, double* cn2, double* ctn2) {
  __shared__ double red[kWarps];
  const int i = blockIdx.x;
  const int64_t o0 = P.om_off[i];
  const int ni = (int)(P.om_off[i + 1] - o0);
  const int64_t b0 = P.blk_off[i];
  const int nb = (int)(P.blk_off[i + 1] - b0);
  const uint8_t* isint = P.om_int + o0;
  double sc = 0.0, st = 0.0;
  for (int b = 0; b < nb; ++b) {
    const int t0 = P.blk_tf[b0 + b];
    const int width = (b - t0 + 1) * kT;
    const int64_t po = P.blk_poff[b0 + b];
    for (int e = threadIdx.x; e < kT * width; e += blockDim.x) {
      const int rr = e / width, cc = e - rr * width;
      const int p = b * kT + rr, q = t0 * kT + cc;
      if (p >= ni || q > p) continue;
      const double v = C[po + e], w = Ct[po + e];
      sc += v * v * (double)(isint[p] + (q < p ? isint[q] : 0));
      st += w * w * (q == p ? 1.0 : 2.0);
    }
  }
  const double s1 = block_sum(sc, red);
  const double s2 = block_sum(st, red);
  if (threadIdx.x == 0) { cn2[i] = s1; ctn2[i] = s2; }
}

// C_ii += delta I; eqs = diag^{-1/2}; C_ii <- diag(eqs) C_ii diag(eqs); B = C~_ii + s_i I.
// Padding rows (k >= n_i) become identity rows in both storages.
__global__ void __launch_bounds__(kThreads) k_prep(BandPlan P, double delta, const double* __restrict__ s,
                                                   double* __restrict__ C, double* __restrict__ eqs,
                                                   const double* __restrict__ Ct, double* __restrict__ B) {
  const int i = blockIdx.x;
  const int64_t o0 = P.om_off[i];
  const int ni = (int)(P.om_off[i + 1] - o0);
  const int64_t b0 = P.blk_off[i];
  const int nb = (int)(P.blk_off[i + 1] - b0);
  for (int k = threadIdx.x; k < nb * kT; k += blockDim.x) {
    const int b = k >> 5, rr = k & 31;
    const int t0 = P.blk_tf[b0 + b];
    const int width = (b - t0 + 1) * kT;
    const int64_t d = P.blk_poff[b0 + b] + (int64_t)rr * width + (width - kT) + rr;
    if (k < ni) {
      const double c = C[d] + delta;
      C[d] = c;
      eqs[o0 + k] = c > 0.0 ? 1.0 / sqrt(c) : 1.0;
    } else {
      C[d] = 1.0;
    }
  }
  __syncthreads();
  const double si = s[i];
  for (int b = 0; b < nb; ++b) {
    const int t0 = P.blk_tf[b0 + b];
    const int width = (b - t0 + 1) * kT;
    const int64_t po = P.blk_poff[b0 + b];
    for (int e = threadIdx.x; e < kT * width; e += blockDim.x) {
      const int rr = e / width, cc = e - rr * width;
      const int p = b * kT + rr, q = t0 * kT + cc;
      double bv = Ct[po + e];
      if (p < ni && q < ni) {
        C[po + e] *= eqs[o0 + p] * eqs[o0 + q];
        if (p == q) bv += si;
      } else if (p == q) {
        bv = 1.0;
      } else {
        bv = 0.0;
        C[po + e] = 0.0;
      }
      B[po + e] = bv;
    }
  }
}

// Left-looking tiled Cholesky of every subdomain's block-envelope matrix, in place.
// dinv: scratch of 1024 doubles per block row holding the inverse diagonal tiles.
__global__ void __launch_bounds__(kThreads) k_band_cholesky(BandPlan P, double* __restrict__ F,
                                                            double* __restrict__ idiag, double* __restrict__ dinv,
                                                            int* __restrict__ status) {
  __shared__ double S[kT * 33], Pm[kT * 33], Qm[kT * 33];
  __shared__ int fail;
  const int i = blockIdx.x;
  const int64_t b0 = P.blk_off[i];
  const int nb = (int)(P.blk_off[i + 1] - b0);
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int b = 0; b < nb; ++b) {
    const int tb = P.blk_tf[b0 + b];
    const int wb = (b - tb + 1) * kT;
    double* panb = F + P.blk_poff[b0 + b];
    for (int c = tb; c <= b; ++c) {
      const int tc = P.blk_tf[b0 + c];
      const int wc = (c - tc + 1) * kT;
      const double* panc = F + P.blk_poff[b0 + c];
      load_tile(S, panb, wb, (c - tb) * kT);
      __syncthreads();
      for (int k = max(tb, tc); k < c; ++k) {
        load_tile(Pm, panb, wb, (k - tb) * kT);
        load_tile(Qm, panc, wc, (k - tc) * kT);
        __syncthreads();
        tile_mm<false, true>(S, Pm, Qm, -1);
        __syncthreads();
      }
      if (c < b) {
        // L(b,c) = S L(c,c)^{-T} = S * (L(c,c)^{-1})^T
        const double* dv = dinv + (b0 + c) * (int64_t)(kT * kT);
        for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) Qm[(e >> 5) * 33 + (e & 31)] = dv[e];
        for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) Pm[(e >> 5) * 33 + (e & 31)] = S[(e >> 5) * 33 + (e & 31)];
        __syncthreads();
        tile_mm<false, true>(S, Pm, Qm, 0);
        __syncthreads();
      } else {
        tile_potrf_inv(S, Qm, &fail, b * kT);
        double* dv = dinv + (b0 + b) * (int64_t)(kT * kT);
        for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) dv[e] = Qm[(e >> 5) * 33 + (e & 31)];
        if (threadIdx.x < kT) idiag[b0 * kT + b * kT + threadIdx.x] = Qm[threadIdx.x * 33 + threadIdx.x];
        // zero the strict upper part of the diagonal tile
        for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) {
          const int a = e >> 5, l = e & 31;
          if (l > a) S[a * 33 + l] = 0.0;
        }
        __syncthreads();
      }
      store_tile(S, panb, wb, (c - tb) * kT);
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) status[i] = fail;
}

__global__ void k_convert_f32(int64_t n, const double* __restrict__ src, float* __restrict__ dst) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = (float)src[k];
}

// One CTA per block row: per 32x32 tile, scale = max |entry| (1 if the tile is zero)
// and the BF16 values entry / scale.
__global__ void __launch_bounds__(kThreads) k_convert_bf16(const int64_t* __restrict__ poff, const double* __restrict__ src,
                                                           __nv_bfloat16* __restrict__ dst, float* __restrict__ tsc) {
  __shared__ double red[kWarps];
  const int64_t g = blockIdx.x;
  const int64_t po = poff[g];
  const int width = (int)((poff[g + 1] - po) / kT);
  const int ntile = width / kT;
  for (int t = 0; t < ntile; ++t) {
    double mx = 0.0;
    for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) {
      const int rr = e >> 5, cc = e & 31;
      mx = fmax(mx, fabs(src[po + (int64_t)rr * width + t * kT + cc]));
    }
    // block max through the sum helper on a one-hot trick is not possible; do it directly
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    double m = 0.0;
    for (int k = 0; k < kWarps; ++k) m = fmax(m, red[k]);
    const double sc = m > 0.0 ? m : 1.0;
    if (threadIdx.x == 0) tsc[po / 1024 + t] = (float)sc;
    for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) {
      const int rr = e >> 5, cc = e & 31;
      const int64_t idx = po + (int64_t)rr * width + t * kT + cc;
      dst[idx] = __float2bfloat16_rn((float)(src[idx] / sc));
    }
  }
}

// One CTA per subdomain: gather r(Omega_i), optional coarse restriction
// r0_i = Zbar_i^T r(Omega_I,i), then C_ii^{-1} through the (equilibrated) factor.
template <class TF, class TA>
__global__ void __launch_bounds__(kThreads) k_local_solve(LocalArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int i = blockIdx.x;
  const int64_t o0 = a.om_off[i];
  const int ni = (int)(a.om_off[i + 1] - o0);
  const int64_t b0 = a.blk_off[i];
  const int nb = (int)(a.blk_off[i + 1] - b0);
  TA* v = reinterpret_cast<TA*>(smem_raw);
  TA* dt = v + nb * kT;
  TA* tmp = dt + kT * 33;
  for (int k = threadIdx.x; k < nb * kT; k += blockDim.x)
    v[k] = k < ni ? (TA)(a.r[a.om_glob[o0 + k]] * a.eqs[o0 + k]) : (TA)0;
  if (a.coarse) {
    const int c0 = a.coff[i], kk = a.coff[i + 1] - c0;
    const int64_t io = a.int_off[i];
    const int nIi = (int)(a.int_off[i + 1] - io);
    const double* Zi = a.Z + a.zoff[i];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int t = w; t < kk; t += kWarps) {
      double acc = 0.0;
      for (int jj = lane; jj < nIi; jj += 32) acc += Zi[(int64_t)t * nIi + jj] * a.r[a.int_glob[io + jj]];
      acc = warp_sum(acc);
      if (lane == 0) a.r0[c0 + t] = acc;
    }
  }
  __syncthreads();
  BandRef B{a.blk_tf + b0, a.blk_poff + b0, nb};
  const TF* fac = reinterpret_cast<const TF*>(a.fac);
  const TA* idg = reinterpret_cast<const TA*>(a.idiag) + b0 * kT;
  band_forward<TF, TA>(fac, a.tsc, idg, B, v, dt, tmp);
  band_backward<TF, TA>(fac, a.tsc, idg, B, v, dt, tmp);
  for (int k = threadIdx.x; k < ni; k += blockDim.x) a.y[o0 + k] = (double)v[k] * a.eqs[o0 + k];
}

int grid_for(int64_t work, int cap) {
  int64_t g = (work + kThreads - 1) / kThreads;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

void launch_assemble(const BandPlan& P, const CsrDev& A, const CscDev& At, const int32_t* part,
                     int64_t total_local, double* Cst, double* Ctst, cudaStream_t st) {
  k_assemble<<<grid_for(total_local, 1 << 15), kThreads, 0, st>>>(P, A, At, part, total_local, Cst, Ctst);
}

void launch_norms(const BandPlan& P, const double* Cst, const double* Ctst, double* cn2, double* ctn2,
                  cudaStream_t st) {
  k_norms<<<P.N, kThreads, 0, st>>>(P, Cst, Ctst, cn2, ctn2);
}

void launch_prep(const BandPlan& P, double delta, const double* s, double* Cst, double* eqs,
                 const double* Ctst, double* Bst, cudaStream_t st) {
  k_prep<<<P.N, kThreads, 0, st>>>(P, delta, s, Cst, eqs, Ctst, Bst);
}

void launch_band_cholesky(const BandPlan& P, double* F, double* idiag, double* dinv, int* status,
                               cudaStream_t st) {
  k_band_cholesky<<<P.N, kThreads, 0, st>>>(P, F, idiag, dinv, status);
}

void launch_convert_f32(int64_t n, const double* src, float* dst, cudaStream_t st) {
  k_convert_f32<<<grid_for(n, 8192), kThreads, 0, st>>>(n, src, dst);
}

void launch_convert_bf16(int64_t nblocks, const int64_t* poff, const double* src, __nv_bfloat16* dst,
                              float* tsc, cudaStream_t st) {
  k_convert_bf16<<<(unsigned)nblocks, kThreads, 0, st>>>(poff, src, dst, tsc);
}

size_t local_solve_smem(int prec, int max_nb) {
  const size_t es = prec == 0 ? sizeof(double) : sizeof(float);
  return es * ((size_t)max_nb * kT + kT * 33 + kT);
}

void launch_local_solve(int prec, int N, int max_nb, const LocalArgs& a, cudaStream_t st) {
  // The opt-in shared-memory limit is raised only when a larger size is first needed,
  // so launches inside a stream capture make no attribute calls.
  static size_t raised[3] = {0, 0, 0};
  const size_t sm = local_solve_smem(prec, max_nb);
  const bool raise = sm > 48 * 1024 && sm > raised[prec];
  if (prec == 0) {
    if (raise) cudaFuncSetAttribute(k_local_solve<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_local_solve<double, double><<<N, kThreads, sm, st>>>(a);
  } else if (prec == 1) {
    if (raise) cudaFuncSetAttribute(k_local_solve<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_local_solve<float, float><<<N, kThreads, sm, st>>>(a);
  } else {
    if (raise) cudaFuncSetAttribute(k_local_solve<__nv_bfloat16, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_local_solve<__nv_bfloat16, float><<<N, kThreads, sm, st>>>(a);
  }
  if (raise) raised[prec] = sm;
}

}  // namespace lsq
