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
__global__ void __launch_bounds__(kThreads) k_prep(BandPlan P, const double* __restrict__ dsub, const double* __restrict__ s,
                                                   double* __restrict__ C, double* __restrict__ eqs,
                                                   const double* __restrict__ Ct, double* __restrict__ B) {
  const int i = blockIdx.x;
  const double delta = dsub[i];
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

void launch_prep(const BandPlan& P, const double* dsub, const double* s, double* Cst, double* eqs,
                 const double* Ctst, double* Bst, cudaStream_t st) {
  k_prep<<<P.N, kThreads, 0, st>>>(P, dsub, s, Cst, eqs, Ctst, Bst);
}

void launch_band_cholesky(const BandPlan& P, double* F, double* idiag, double* dinv, int* status,
                               cudaStream_t st) {
  k_band_cholesky<<<P.N, kThreads, 0, st>>>(P, F, idiag, dinv, status);
}

}  // namespace lsq
