// FP64 32x32 tile helpers for the setup factorizations (CTA of 256 threads; tiles
// live in shared memory with a row pitch of 33 to spread banks).
#pragma once
#include "common.cuh"

namespace lsq {

// S = / += / -= op(P) op(Q) with op(P)[i][l] = tP ? P[l][i] : P[i][l] and
// op(Q)[l][j] = tQ ? Q[j][l] : Q[l][j]; mode 0 assigns, +1 adds, -1 subtracts.
// Each thread owns row t/8 and four consecutive columns.
template <bool tP, bool tQ>
__device__ __forceinline__ void tile_mm(double* S, const double* P, const double* Q, int mode) {
  const int t = threadIdx.x;
  const int i = t >> 3, j0 = (t & 7) * 4;
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll 8
  for (int l = 0; l < kT; ++l) {
    const double p = tP ? P[l * 33 + i] : P[i * 33 + l];
    a0 += p * (tQ ? Q[(j0 + 0) * 33 + l] : Q[l * 33 + j0 + 0]);
    a1 += p * (tQ ? Q[(j0 + 1) * 33 + l] : Q[l * 33 + j0 + 1]);
    a2 += p * (tQ ? Q[(j0 + 2) * 33 + l] : Q[l * 33 + j0 + 2]);
    a3 += p * (tQ ? Q[(j0 + 3) * 33 + l] : Q[l * 33 + j0 + 3]);
  }
  double* s = S + i * 33 + j0;
  if (mode == 0) { s[0] = a0; s[1] = a1; s[2] = a2; s[3] = a3; }
  else if (mode > 0) { s[0] += a0; s[1] += a1; s[2] += a2; s[3] += a3; }
  else { s[0] -= a0; s[1] -= a1; s[2] -= a2; s[3] -= a3; }
}

__device__ __forceinline__ void load_tile(double* dst, const double* src, int64_t ld, int64_t col0) {
  for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) {
    const int rr = e >> 5, cc = e & 31;
    dst[rr * 33 + cc] = src[(int64_t)rr * ld + col0 + cc];
  }
}

__device__ __forceinline__ void store_tile(const double* src, double* dst, int64_t ld, int64_t col0) {
  for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) {
    const int rr = e >> 5, cc = e & 31;
    dst[(int64_t)rr * ld + col0 + cc] = src[rr * 33 + cc];
  }
}

// Unblocked Cholesky of the 32x32 tile in S (lower triangle used); on a pivot that is
// not positive and finite records 1 + (row0 + row) in *fail (first failure only) and
// continues with pivot 1.  Then Q = L^{-1} (lower), S's strict upper part is zeroed.
__device__ __forceinline__ void tile_potrf_inv(double* S, double* Q, int* fail, int row0) {
  const int t = threadIdx.x;
  for (int j = 0; j < kT; ++j) {
    if (t == 0) {
      double d = S[j * 33 + j];
      if (!(d > 0.0) || !isfinite(d)) {
        if (*fail == 0) *fail = row0 + j + 1;
        d = 1.0;
      }
      S[j * 33 + j] = sqrt(d);
    }
    __syncthreads();
    if (t > j && t < kT) S[t * 33 + j] /= S[j * 33 + j];
    __syncthreads();
    for (int e = t; e < kT * kT; e += blockDim.x) {
      const int a = e >> 5, l = e & 31;
      if (a > j && l > j && l <= a) S[a * 33 + l] -= S[a * 33 + j] * S[l * 33 + j];
    }
    __syncthreads();
  }
  if (t < kT) {
    const int j = t;  // column j of L^{-1}
    for (int a = 0; a < kT; ++a) Q[a * 33 + j] = 0.0;
    Q[j * 33 + j] = 1.0 / S[j * 33 + j];
    for (int a = j + 1; a < kT; ++a) {
      double acc = 0.0;
      for (int l = j; l < a; ++l) acc += S[a * 33 + l] * Q[l * 33 + j];
      Q[a * 33 + j] = -acc / S[a * 33 + a];
    }
  }
  __syncthreads();
  for (int e = t; e < kT * kT; e += blockDim.x) {
    const int a = e >> 5, l = e & 31;
    if (l > a) S[a * 33 + l] = 0.0;
  }
  __syncthreads();
}

}  // namespace lsq
