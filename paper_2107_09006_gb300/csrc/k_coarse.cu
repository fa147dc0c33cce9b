// Coarse operator of Algorithm 1: W_i = A(Xi_i, Omega_I,i) Zbar_i, the blocks
// C_00(i, j) = W_i(shared rows)^T W_j(shared rows) + delta [i == j] Zbar_i^T Zbar_i
// (so that C_00 = (A R_0^T)^T (A R_0^T) + delta R_0 R_0^T), and the dense FP64
// Cholesky factorization of C_00 followed by its explicit inverse (used by the
// per-iteration coarse solve as one dense product).
#include "kernels.h"
#include "tile.cuh"

namespace lsq {

namespace {

__global__ void __launch_bounds__(kThreads) k_coarse_w(const int64_t* __restrict__ xi_off, const int32_t* __restrict__ xi,
                                                       const int32_t* __restrict__ coff, const int64_t* __restrict__ woff,
                                                       const int64_t* __restrict__ zoff, const int32_t* __restrict__ nI,
                                                       CsrDev A, const int32_t* __restrict__ part,
                                                       const int32_t* __restrict__ jj_of, const double* __restrict__ Z,
                                                       double* __restrict__ W, int64_t total, const int32_t* __restrict__ xi_sub) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = xi_sub[e];
    const int k = coff[i + 1] - coff[i];
    if (k == 0) continue;
    const int64_t a = e - xi_off[i];
    const int32_t r = xi[e];
    const int64_t nIi = nI[i];
    const double* Zi = Z + zoff[i];
    double* Wr = W + woff[i] + a * k;
    for (int t = 0; t < k; ++t) {
      double acc = 0.0;
      for (int64_t s = A.row_ptr[r]; s < A.row_ptr[r + 1]; ++s) {
        const int32_t c = A.col[s];
        if (part[c] == i) acc += A.val[s] * Zi[t * nIi + jj_of[c]];
      }
      Wr[t] = acc;
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_coarse_pairs(const int32_t* __restrict__ pi, const int32_t* __restrict__ pj,
                                                           const int64_t* __restrict__ poff, const int32_t* __restrict__ ppi,
                                                           const int32_t* __restrict__ ppj, const int32_t* __restrict__ coff,
                                                           const int64_t* __restrict__ woff, const int64_t* __restrict__ zoff,
                                                           const int32_t* __restrict__ nI, const double* __restrict__ W,
                                                           const double* __restrict__ Z, const double* __restrict__ dsub,
                                                           CoarseBlocks cb, double* __restrict__ C00) {
  const int p = blockIdx.x;
  const int i = pi[p], j = pj[p];
  const int q = cb.prob_of_sub[i];  // i and j belong to the same problem
  const int64_t ld = cb.ld[q];
  double* Cq = C00 + cb.base[q];
  const int ci = coff[i] - cb.c0[q], ki = coff[i + 1] - coff[i];
  const int cj = coff[j] - cb.c0[q], kj = coff[j + 1] - coff[j];
  const double delta = dsub[i];
  if (ki == 0 || kj == 0) return;
  const double* Wi = W + woff[i];
  const double* Wj = W + woff[j];
  for (int e = threadIdx.x; e < ki * kj; e += blockDim.x) {
    const int t = e / kj, u = e % kj;
    double acc = 0.0;
    for (int64_t s = poff[p]; s < poff[p + 1]; ++s) acc += Wi[(int64_t)ppi[s] * ki + t] * Wj[(int64_t)ppj[s] * kj + u];
    if (i == j && delta != 0.0) {
      const int64_t n = nI[i];
      const double* Zi = Z + zoff[i];
      double zz = 0.0;
      for (int64_t q = 0; q < n; ++q) zz += Zi[t * n + q] * Zi[u * n + q];
      acc += delta * zz;
    }
    Cq[(int64_t)(ci + t) * ld + cj + u] = acc;
    if (i != j) Cq[(int64_t)(cj + u) * ld + ci + t] = acc;
  }
}

// ---- dense tiled Cholesky and inverse (n a multiple of 32, row-major, ld = n) ----

__global__ void __launch_bounds__(kThreads) k_potrf_tile(double* A, int64_t n, int k, double* dinv, int* status) {
  __shared__ double S[kT * 33], Q[kT * 33];
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  double* Akk = A + (int64_t)k * kT * n + (int64_t)k * kT;
  load_tile(S, Akk, n, 0);
  __syncthreads();
  tile_potrf_inv(S, Q, &fail, k * kT);
  store_tile(S, Akk, n, 0);
  for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) dinv[(int64_t)k * kT * kT + e] = Q[(e >> 5) * 33 + (e & 31)];
  if (threadIdx.x == 0 && fail && *status == 0) *status = fail;
}

// L(i,k) = A(i,k) L(k,k)^{-T} for the tiles below the diagonal.
__global__ void __launch_bounds__(kThreads) k_trsm_col(double* A, int64_t n, int k, const double* dinv) {
  __shared__ double S[kT * 33], P[kT * 33], Q[kT * 33];
  const int i = k + 1 + blockIdx.x;
  double* Aik = A + (int64_t)i * kT * n + (int64_t)k * kT;
  load_tile(P, Aik, n, 0);
  for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) Q[(e >> 5) * 33 + (e & 31)] = dinv[(int64_t)k * kT * kT + e];
  __syncthreads();
  tile_mm<false, true>(S, P, Q, 0);
  __syncthreads();
  store_tile(S, Aik, n, 0);
}

// A(i,j) -= L(i,k) L(j,k)^T for k < j <= i.
__global__ void __launch_bounds__(kThreads) k_syrk_update(double* A, int64_t n, int k, int nt) {
  __shared__ double S[kT * 33], P[kT * 33], Q[kT * 33];
  // blockIdx.x enumerates the lower-triangular pairs (i, j) of the trailing nt-k-1 tiles
  const int m = nt - k - 1;
  int rem = blockIdx.x, ii = 0;
  while (rem >= ii + 1) { rem -= ii + 1; ++ii; }
  const int i = k + 1 + ii, j = k + 1 + rem;
  if (ii >= m) return;
  double* Aij = A + (int64_t)i * kT * n + (int64_t)j * kT;
  load_tile(S, Aij, n, 0);
  load_tile(P, A + (int64_t)i * kT * n + (int64_t)k * kT, n, 0);
  load_tile(Q, A + (int64_t)j * kT * n + (int64_t)k * kT, n, 0);
  __syncthreads();
  tile_mm<false, true>(S, P, Q, -1);
  __syncthreads();
  store_tile(S, Aij, n, 0);
}

// Y = L^{-1} (lower), one CTA per tile column j: Y(j,j) = L(j,j)^{-1};
// Y(i,j) = -L(i,i)^{-1} sum_{k=j}^{i-1} L(i,k) Y(k,j).
__global__ void __launch_bounds__(kThreads) k_trtri_col(const double* L, double* Y, int64_t n, int nt, const double* dinv) {
  __shared__ double S[kT * 33], P[kT * 33], Q[kT * 33];
  const int j = blockIdx.x;
  for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) S[(e >> 5) * 33 + (e & 31)] = dinv[(int64_t)j * kT * kT + e];
  __syncthreads();
  store_tile(S, Y + (int64_t)j * kT * n + (int64_t)j * kT, n, 0);
  __syncthreads();
  for (int i = j + 1; i < nt; ++i) {
    for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) S[(e >> 5) * 33 + (e & 31)] = 0.0;
    __syncthreads();
    for (int k = j; k < i; ++k) {
      load_tile(P, L + (int64_t)i * kT * n + (int64_t)k * kT, n, 0);
      load_tile(Q, Y + (int64_t)k * kT * n + (int64_t)j * kT, n, 0);
      __syncthreads();
      tile_mm<false, false>(S, P, Q, 1);
      __syncthreads();
    }
    for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) P[(e >> 5) * 33 + (e & 31)] = dinv[(int64_t)i * kT * kT + e];
    __syncthreads();
    tile_mm<false, false>(Q, P, S, 0);  // Q = Linv(i,i) * S
    __syncthreads();
    for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) Q[(e >> 5) * 33 + (e & 31)] = -Q[(e >> 5) * 33 + (e & 31)];
    __syncthreads();
    store_tile(Q, Y + (int64_t)i * kT * n + (int64_t)j * kT, n, 0);
    __syncthreads();
  }
}

// X(i,j) = sum_{k >= i} Y(k,i)^T Y(k,j) for i >= j (Y lower), written to both halves.
__global__ void __launch_bounds__(kThreads) k_lauum(const double* Y, double* X, int64_t n, int nt) {
  __shared__ double S[kT * 33], P[kT * 33], Q[kT * 33];
  int rem = blockIdx.x, i = 0;
  while (rem >= i + 1) { rem -= i + 1; ++i; }
  const int j = rem;
  for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) S[(e >> 5) * 33 + (e & 31)] = 0.0;
  __syncthreads();
  for (int k = i; k < nt; ++k) {
    load_tile(P, Y + (int64_t)k * kT * n + (int64_t)i * kT, n, 0);
    load_tile(Q, Y + (int64_t)k * kT * n + (int64_t)j * kT, n, 0);
    __syncthreads();
    tile_mm<true, false>(S, P, Q, 1);
    __syncthreads();
  }
  store_tile(S, X + (int64_t)i * kT * n + (int64_t)j * kT, n, 0);
  if (i != j) {
    for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) {
      const int rr = e >> 5, cc = e & 31;
      X[(int64_t)(j * kT + rr) * n + i * kT + cc] = S[cc * 33 + rr];
    }
  }
}

int grid_for(int64_t work, int cap) {
  int64_t g = (work + kThreads - 1) / kThreads;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

void launch_coarse_w(int N, const int64_t* xi_off, const int32_t* xi, const int32_t* coff, const int64_t* woff,
                     const int64_t* zoff, const int32_t* nI, const CsrDev& A, const int32_t* part,
                     const int32_t* jj_of, const double* Z, double* W, int64_t total_xi, const int32_t* xi_sub,
                     cudaStream_t st) {
  (void)N;
  k_coarse_w<<<grid_for(total_xi, 1 << 15), kThreads, 0, st>>>(xi_off, xi, coff, woff, zoff, nI, A, part, jj_of, Z,
                                                               W, total_xi, xi_sub);
}

void launch_coarse_pairs(int npairs, const int32_t* pi, const int32_t* pj, const int64_t* poff, const int32_t* ppi,
                         const int32_t* ppj, const int32_t* coff, const int64_t* woff, const int64_t* zoff,
                         const int32_t* nI, const double* W, const double* Z, const double* dsub,
                         const CoarseBlocks& cb, double* C00, cudaStream_t st) {
  if (npairs <= 0) return;
  k_coarse_pairs<<<npairs, kThreads, 0, st>>>(pi, pj, poff, ppi, ppj, coff, woff, zoff, nI, W, Z, dsub, cb, C00);
}

// A (n x n, n a multiple of 32) is replaced by A^{-1}; Y is an n x n scratch; dinv is
// an (n/32) * 1024 scratch.  *status (device) receives 0 or 1 + the failing row.
void dense_spd_inverse(int64_t n, double* A, double* Y, double* dinv, int* status, cudaStream_t st) {
  const int nt = (int)(n / kT);
  for (int k = 0; k < nt; ++k) {
    k_potrf_tile<<<1, kThreads, 0, st>>>(A, n, k, dinv, status);
    const int m = nt - k - 1;
    if (m > 0) {
      k_trsm_col<<<m, kThreads, 0, st>>>(A, n, k, dinv);
      k_syrk_update<<<m * (m + 1) / 2, kThreads, 0, st>>>(A, n, k, nt);
    }
  }
  cudaMemsetAsync(Y, 0, sizeof(double) * n * n, st);
  k_trtri_col<<<nt, kThreads, 0, st>>>(A, Y, n, nt, dinv);
  k_lauum<<<nt * (nt + 1) / 2, kThreads, 0, st>>>(Y, A, n, nt);
}

}  // namespace lsq
