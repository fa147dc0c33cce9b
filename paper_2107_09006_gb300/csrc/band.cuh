// Block-envelope ("tiled skyline") storage of one local matrix and the CTA-wide
// triangular solves and symmetric products on it.
//
// Subdomain i's local matrix (size n_i, padded to nb*32 with identity rows) is kept
// in ascending global column order.  Block row b (rows [32b, 32b+32)) stores the
// tiles [tf_b, b] of its lower triangle as one row-major 32 x width panel,
// width = (b - tf_b + 1) * 32; tf_b is the first tile column that any row of the
// block couples to, so the Cholesky factor's fill stays inside the same panels.
// The inverse diagonal of the factor is kept apart (idiag) so the diagonal-tile
// substitutions multiply instead of divide.  BF16 storage carries one FP32 scale
// per 32x32 tile (tile id = panel offset / 1024 + tile column within the panel).
#pragma once
#include "common.cuh"

namespace lsq {

template <class TF> struct Load;
template <> struct Load<double> {
  static __device__ __forceinline__ double get(const double* p, int64_t k) { return p[k]; }
};
template <> struct Load<float> {
  static __device__ __forceinline__ float get(const float* p, int64_t k) { return __ldg(p + k); }
};
template <> struct Load<__nv_bfloat16> {
  static __device__ __forceinline__ float get(const __nv_bfloat16* p, int64_t k) {
    return __bfloat162float(p[k]);
  }
};

struct BandRef {
  const int32_t* tf;    // first tile column of each block row of this subdomain
  const int64_t* poff;  // element offset of each panel
  int nb;               // block rows
};

// Solve L y = v in place (v: nb*32 entries, shared or global memory).
// dt: 32*33 scratch, tmp: 32 scratch, both shared.  All threads of the CTA call it.
template <class TF, class TA>
__device__ void band_forward(const TF* __restrict__ fac, const float* __restrict__ tsc,
                             const TA* __restrict__ idiag, BandRef B, TA* v, TA* dt, TA* tmp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int b = 0; b < B.nb; ++b) {
    const int t0 = B.tf[b];
    const int width = (b - t0 + 1) * kT;
    const int offw = width - kT;
    const int64_t po = B.poff[b];
    const TF* pan = fac + po;
    const TA* vw = v + t0 * kT;
    // the warp's four rows in one pass (four independent loads per column step; each
    // row's sum keeps its order)
    const TF* row0 = pan + (int64_t)(w * 4) * width;
    TA acc[4] = {0, 0, 0, 0};
    if (tsc) {
      int tcol = 0;
      for (int c = lane; c < offw; c += 32, ++tcol) {
        const TA x = vw[c], sc = (TA)tsc[po / 1024 + tcol];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += sc * (Load<TF>::get(row0 + (int64_t)q * width, c) * x);
      }
    } else {
      for (int c = lane; c < offw; c += 32) {
        const TA x = vw[c];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += Load<TF>::get(row0 + (int64_t)q * width, c) * x;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const TA sum = warp_sum(acc[q]);
      if (lane == 0) tmp[w * 4 + q] = v[b * kT + w * 4 + q] - sum;
    }
    const TA dsc = tsc ? (TA)tsc[po / 1024 + (b - t0)] : (TA)1;
    for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) {
      const int rr = e >> 5, cc = e & 31;
      dt[rr * 33 + cc] = dsc * Load<TF>::get(pan, (int64_t)rr * width + offw + cc);
    }
    __syncthreads();
    if (w == 0) {
      TA y = tmp[lane];
      const TA id = idiag[b * kT + lane];
      for (int c = 0; c < kT; ++c) {
        const TA xc = __shfl_sync(0xffffffffu, y * id, c);
        if (lane > c) y -= dt[lane * 33 + c] * xc;
      }
      v[b * kT + lane] = y * id;
    }
    __syncthreads();
  }
}

// Solve L^T x = v in place.
template <class TF, class TA>
__device__ void band_backward(const TF* __restrict__ fac, const float* __restrict__ tsc,
                              const TA* __restrict__ idiag, BandRef B, TA* v, TA* dt, TA* tmp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int b = B.nb - 1; b >= 0; --b) {
    const int t0 = B.tf[b];
    const int width = (b - t0 + 1) * kT;
    const int offw = width - kT;
    const int64_t po = B.poff[b];
    const TF* pan = fac + po;
    const TA dsc = tsc ? (TA)tsc[po / 1024 + (b - t0)] : (TA)1;
    for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) {
      const int rr = e >> 5, cc = e & 31;
      dt[rr * 33 + cc] = dsc * Load<TF>::get(pan, (int64_t)rr * width + offw + cc);
    }
    __syncthreads();
    if (w == 0) {
      TA y = v[b * kT + lane];
      const TA id = idiag[b * kT + lane];
      for (int r = kT - 1; r >= 0; --r) {
        const TA xr = __shfl_sync(0xffffffffu, y * id, r);
        if (lane < r) y -= dt[r * 33 + lane] * xr;
      }
      y *= id;
      tmp[lane] = y;
      v[b * kT + lane] = y;
    }
    __syncthreads();
    TA* vw = v + t0 * kT;
    for (int c = threadIdx.x; c < offw; c += blockDim.x) {
      TA acc = 0;
#pragma unroll 8
      for (int rr = 0; rr < kT; ++rr) acc += Load<TF>::get(pan, (int64_t)rr * width + c) * tmp[rr];
      if (tsc) acc *= (TA)tsc[po / 1024 + (c >> 5)];
      vw[c] -= acc;
    }
    __syncthreads();
  }
}

// y += C x for the symmetric matrix whose lower triangle is stored (FP64, setup only).
template <class TA>
__device__ void band_symv(const double* __restrict__ fac, BandRef B, const TA* x, TA* y) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int b = 0; b < B.nb; ++b) {
    const int t0 = B.tf[b];
    const int width = (b - t0 + 1) * kT;
    const int offw = width - kT;
    const double* pan = fac + B.poff[b];
    const TA* xw = x + t0 * kT;
    // the warp's four rows in one pass (row rr sums columns c <= offw + rr, in order)
    const double* row0 = pan + (int64_t)(w * 4) * width;
    TA acc[4] = {0, 0, 0, 0};
    for (int c = lane; c <= offw + w * 4 + 3; c += 32) {
      const TA xc = xw[c];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (c <= offw + w * 4 + q) acc[q] += row0[(int64_t)q * width + c] * xc;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const TA sum = warp_sum(acc[q]);
      if (lane == 0) y[b * kT + w * 4 + q] += sum;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < width; c += blockDim.x) {
      TA acc = 0;
      if (c < offw) {
#pragma unroll 8
        for (int rr = 0; rr < kT; ++rr) acc += pan[(int64_t)rr * width + c] * x[b * kT + rr];
      } else {
        for (int rr = c - offw + 1; rr < kT; ++rr) acc += pan[(int64_t)rr * width + c] * x[b * kT + rr];
      }
      y[t0 * kT + c] += acc;
    }
    __syncthreads();
  }
}

}  // namespace lsq
