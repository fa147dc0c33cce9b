// Device eigen setup: for every subdomain, the largest eigenpairs of the shifted
// local pencil  D_i C_ii D_i v = lambda (C~_ii + s I) v  (eq. (3.4)).
//
// With C~_ii + s I = L L^T, the pencil is the symmetric standard problem
// T u = lambda u, T = L^{-1} D_i C_ii D_i L^{-T}, v = L^{-T} u (so v is
// (C~_ii + s I)-normalised).  Each CTA runs a thick-restart Lanczos (Krylov-Schur
// form) on its subdomain: full re-orthogonalisation in two Gram-Schmidt passes,
// Rayleigh-Ritz on the projected matrix by parallel cyclic Jacobi, restart on the
// best `keep` Ritz vectors.  Only products and solves are needed (Remark 3.2):
// D C_ii D x = D (C~_ii (D x)) + delta D x, since the interior block of C~_ii equals
// that of C_ii = A(:,Omega)^T A(:,Omega) + delta I.  Every loop is bounded by
// maxit; a subdomain that does not converge reports status 2.
#include "band.cuh"
#include "kernels.h"

namespace lsq {

namespace {

constexpr int kMaxK = 160;  // largest Lanczos basis handled

__device__ __forceinline__ double hash_unit(uint32_t a, uint32_t b) {
  // splitmix-style integer hash of (a, b) mapped to [-1, 1)
  uint64_t z = ((uint64_t)a << 32) ^ (uint64_t)b ^ 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

struct Shared {
  double* x1;  // operator work vector (nb*32)
  double* x2;  // operator output / new Lanczos vector (nb*32)
  double* dt;  // 32*33
  double* tmp; // 32
  double* hs;  // kMaxK projection coefficients
  double* h2;  // kMaxK
  double* cs;  // kMaxK/2 Jacobi cosines
  double* sn;  // kMaxK/2 Jacobi sines
  int* pp; int* qq; int* ord;
  double* red; // kWarps
};

// x2 = T x1, destroying x1: x1 <- L^{-T} x1; x2 = D (C~ (D x1)) + delta D x1; x2 <- L^{-1} x2.
__device__ void apply_T(const EigArgs& a, BandRef B, const uint8_t* isint, int ni, int npad, Shared& s) {
  band_backward<double, double>(a.Bfac, nullptr, a.Bidiag + (int64_t)(B.poff - a.P.blk_poff) * kT, B,
                                s.x1, s.dt, s.tmp);
  for (int k = threadIdx.x; k < npad; k += blockDim.x) {
    const double d = (k < ni && isint[k]) ? 1.0 : 0.0;
    s.x1[k] *= d;
    s.x2[k] = 0.0;
  }
  __syncthreads();
  band_symv<double>(a.Ct, B, s.x1, s.x2);
  for (int k = threadIdx.x; k < npad; k += blockDim.x) {
    const double d = (k < ni && isint[k]) ? 1.0 : 0.0;
    s.x2[k] = d * (s.x2[k] + a.delta[blockIdx.x] * s.x1[k]);
  }
  __syncthreads();
  band_forward<double, double>(a.Bfac, nullptr, a.Bidiag + (int64_t)(B.poff - a.P.blk_poff) * kT, B,
                               s.x2, s.dt, s.tmp);
}

// h[t] = V_t . x for t < nv (one warp per t, two vectors per warp at a time for more
// loads in flight; each sum keeps its order).
__device__ void project(const double* V, int64_t vs, int nv, const double* x, int npad, double* h) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t = w; t < nv; t += 2 * kWarps) {
    const int t2 = t + kWarps;
    const double* vt = V + t * vs;
    const double* vu = V + (int64_t)min(t2, nv - 1) * vs;
    double acc = 0.0, acc2 = 0.0;
#pragma unroll 4
    for (int k = lane; k < npad; k += 32) {
      const double xk = x[k];
      acc += vt[k] * xk;
      acc2 += vu[k] * xk;
    }
    acc = warp_sum(acc);
    acc2 = warp_sum(acc2);
    if (lane == 0) {
      h[t] = acc;
      if (t2 < nv) h[t2] = acc2;
    }
  }
  __syncthreads();
}

// x -= sum_t V_t h[t]
__device__ void subtract(const double* V, int64_t vs, int nv, const double* h, double* x, int npad) {
  for (int k = threadIdx.x; k < npad; k += blockDim.x) {
    double acc = 0.0;
#pragma unroll 8
    for (int t = 0; t < nv; ++t) acc += V[t * vs + k] * h[t];
    x[k] -= acc;
  }
  __syncthreads();
}

__device__ double norm2(const double* x, int npad, double* red) {
  double acc = 0.0;
  for (int k = threadIdx.x; k < npad; k += blockDim.x) acc += x[k] * x[k];
  return sqrt(block_sum(acc, red));
}

// Eigen-decomposition of the symmetric n x n matrix H (leading block of a K x K
// buffer, upper triangle valid on entry) by parallel cyclic Jacobi (round-robin
// pairs).  On exit diag(H) holds the eigenvalues, S (K x K) the eigenvectors as
// columns, and s.ord the indices sorted by descending eigenvalue.
__device__ void jacobi(double* H, double* S, int K, int n, Shared& s) {
  const int np = n + (n & 1);  // even size; the extra index is an isolated zero
  for (int e = threadIdx.x; e < np * np; e += blockDim.x) {
    const int r = e / np, c = e % np;
    if (r > c && r < n) H[r * K + c] = H[c * K + r];
    if (r >= n || c >= n) H[r * K + c] = 0.0;
    S[r * K + c] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int half = np / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int e = threadIdx.x; e < np * np; e += blockDim.x) {
      const int r = e / np, c = e % np;
      const double v = H[r * K + c];
      if (r != c) off += v * v; else dia += v * v;
    }
    off = block_sum(off, s.red);
    dia = block_sum(dia, s.red);
    if (off <= 1e-30 * (dia + off) || off == 0.0) break;
    for (int round = 0; round < np - 1; ++round) {
      for (int k = threadIdx.x; k < half; k += blockDim.x) {
        int p, q;
        if (k == 0) { p = round; q = np - 1; }
        else { p = (round + k) % (np - 1); q = (round - k + np - 1) % (np - 1); }
        if (p > q) { const int t = p; p = q; q = t; }
        const double apq = H[p * K + q];
        double c = 1.0, sn = 0.0;
        if (apq != 0.0) {
          const double app = H[p * K + p], aqq = H[q * K + q];
          const double th = (aqq - app) / (2.0 * apq);
          const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
          c = 1.0 / sqrt(1.0 + t * t);
          sn = t * c;
        }
        s.pp[k] = p; s.qq[k] = q; s.cs[k] = c; s.sn[k] = sn;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < half * np; e += blockDim.x) {
        const int k = e / np, col = e % np;
        const int p = s.pp[k], q = s.qq[k];
        const double c = s.cs[k], sn = s.sn[k];
        const double hp = H[p * K + col], hq = H[q * K + col];
        H[p * K + col] = c * hp - sn * hq;
        H[q * K + col] = sn * hp + c * hq;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < half * np; e += blockDim.x) {
        const int k = e / np, row = e % np;
        const int p = s.pp[k], q = s.qq[k];
        const double c = s.cs[k], sn = s.sn[k];
        const double hp = H[row * K + p], hq = H[row * K + q];
        H[row * K + p] = c * hp - sn * hq;
        H[row * K + q] = sn * hp + c * hq;
        const double sp = S[row * K + p], sq = S[row * K + q];
        S[row * K + p] = c * sp - sn * sq;
        S[row * K + q] = sn * sp + c * sq;
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const double th = H[t * K + t];
    int rank = 0;
    for (int u = 0; u < n; ++u) {
      const double tu = H[u * K + u];
      if (tu > th || (tu == th && u < t)) ++rank;
    }
    s.ord[rank] = t;
  }
  __syncthreads();
}

// Vout_t = sum_s Vin_s S[s][ord[t]] for t < cnt.
__device__ void rotate(const double* Vin, double* Vout, int64_t vs, int nv, const double* S, int K,
                       const int* ord, int cnt, int npad) {
  for (int k = threadIdx.x; k < npad; k += blockDim.x) {
    for (int t = 0; t < cnt; ++t) {
      const int col = ord[t];
      double acc = 0.0;
      for (int s2 = 0; s2 < nv; ++s2) acc += Vin[s2 * vs + k] * S[s2 * K + col];
      Vout[t * vs + k] = acc;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads) k_lanczos(EigArgs a, int use_smem) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int i = blockIdx.x;
  const int64_t o0 = a.P.om_off[i];
  const int ni = (int)(a.P.om_off[i + 1] - o0);
  const int64_t b0 = a.P.blk_off[i];
  const int nb = (int)(a.P.blk_off[i + 1] - b0);
  const int npad = nb * kT;
  const uint8_t* isint = a.P.om_int + o0;
  BandRef B{a.P.blk_tf + b0, a.P.blk_poff + b0, nb};
  const int K = a.Kmax;
  const int64_t vs = a.vstride;

  Shared s;
  double* base = reinterpret_cast<double*>(smem_raw);
  int off = 0;
  if (use_smem) {
    s.x1 = base; s.x2 = base + npad; off = 2 * (int)a.vstride;
  } else {
    s.x1 = a.vec + (int64_t)i * 2 * vs; s.x2 = s.x1 + vs;
  }
  s.dt = base + off; off += kT * 33;
  s.tmp = base + off; off += kT;
  s.hs = base + off; off += kMaxK;
  s.h2 = base + off; off += kMaxK;
  s.cs = base + off; off += kMaxK / 2;
  s.sn = base + off; off += kMaxK / 2;
  s.red = base + off; off += kWarps;
  int* ib = reinterpret_cast<int*>(base + off);
  s.pp = ib; s.qq = ib + kMaxK / 2; s.ord = ib + kMaxK;

  double* V = a.V + (int64_t)i * K * vs;
  double* W = a.V2 + (int64_t)i * K * vs;
  double* H = a.H + (int64_t)i * K * K;
  double* S = a.S + (int64_t)i * K * K;
  const int kw = min(a.kwant_cap, ni);
  const int Keff = min(K, ni);
  const int keep = max(kw, min(a.keep, Keff - 1));

  // deterministic start vector
  for (int k = threadIdx.x; k < npad; k += blockDim.x) V[k] = k < ni ? hash_unit(i, k) + 0.5 : 0.0;
  __syncthreads();
  {
    const double nv0 = norm2(V, npad, s.red);
    for (int k = threadIdx.x; k < npad; k += blockDim.x) V[k] /= nv0;
    __syncthreads();
  }
  int nV = 1, steps = 0, status = 0, nconv = 0, fresh = 1;
  double beta = 0.0;
  for (;;) {
    // expand the newest vector: x2 = T V[nV-1], orthogonalised against V[0..nV)
    const double* vj = V + (int64_t)(nV - 1) * vs;
    for (int k = threadIdx.x; k < npad; k += blockDim.x) s.x1[k] = vj[k];
    __syncthreads();
    apply_T(a, B, isint, ni, npad, s);
    ++steps;
    project(V, vs, nV, s.x2, npad, s.hs);
    subtract(V, vs, nV, s.hs, s.x2, npad);
    project(V, vs, nV, s.x2, npad, s.h2);
    subtract(V, vs, nV, s.h2, s.x2, npad);
    for (int t = threadIdx.x; t < nV; t += blockDim.x) H[t * K + (nV - 1)] = s.hs[t] + s.h2[t];
    double hn = 0.0;
    for (int t = 0; t < nV; ++t) hn += (s.hs[t] + s.h2[t]) * (s.hs[t] + s.h2[t]);
    beta = norm2(s.x2, npad, s.red);
    const bool breakdown = !(beta > 1e-12 * sqrt(hn + beta * beta));
    if (nV < Keff && steps < a.maxit) {
      double* vn = V + (int64_t)nV * vs;
      if (!breakdown) {
        for (int k = threadIdx.x; k < npad; k += blockDim.x) vn[k] = s.x2[k] / beta;
      } else {
        // invariant subspace: continue with a fresh vector orthogonal to V
        for (int k = threadIdx.x; k < npad; k += blockDim.x)
          s.x2[k] = k < ni ? hash_unit(i + 7919u * (uint32_t)(fresh + 1), k) : 0.0;
        ++fresh;
        __syncthreads();
        project(V, vs, nV, s.x2, npad, s.hs);
        subtract(V, vs, nV, s.hs, s.x2, npad);
        project(V, vs, nV, s.x2, npad, s.h2);
        subtract(V, vs, nV, s.h2, s.x2, npad);
        const double nn = norm2(s.x2, npad, s.red);
        for (int k = threadIdx.x; k < npad; k += blockDim.x) vn[k] = s.x2[k] / nn;
        beta = 0.0;
      }
      __syncthreads();
      ++nV;
      continue;
    }
    if (breakdown) beta = 0.0;
    // Rayleigh-Ritz on the nV x nV projected matrix
    __syncthreads();
    jacobi(H, S, K, nV, s);
    nconv = 0;
    const int kk = min(kw, nV);
    {
      const double th0 = fabs(H[s.ord[0] * K + s.ord[0]]);
      for (int t = 0; t < kk; ++t) {
        const double res = beta * fabs(S[(nV - 1) * K + s.ord[t]]);
        if (res <= a.tol * fmax(th0, 1e-300)) ++nconv; else break;
      }
    }
    const bool done = (nconv >= kk) || (nV >= ni) || (steps >= a.maxit);
    const int cnt = done ? kk : keep;
    rotate(V, W, vs, nV, S, K, s.ord, cnt, npad);
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) s.hs[t] = H[s.ord[t] * K + s.ord[t]];
    __syncthreads();
    { double* tsw = V; V = W; W = tsw; }
    if (done) {
      if (nconv < kk && nV < ni) status = 2;
      for (int t = threadIdx.x; t < kk; t += blockDim.x) a.lam[(int64_t)i * a.kwant_cap + t] = s.hs[t];
      // the caller expects the Ritz vectors in its V region
      if (V != a.V + (int64_t)i * K * vs) {
        double* dst = a.V + (int64_t)i * K * vs;
        for (int64_t e = threadIdx.x; e < (int64_t)kk * vs; e += blockDim.x) dst[e] = V[e];
      }
      break;
    }
    // restart: H = diag(theta_0..theta_{keep-1}); the residual direction becomes V[keep]
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) H[e] = 0.0;
    __syncthreads();
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) H[t * K + t] = s.hs[t];
    double* vn = V + (int64_t)cnt * vs;
    if (beta > 0.0) {
      for (int k = threadIdx.x; k < npad; k += blockDim.x) vn[k] = s.x2[k] / beta;
      __syncthreads();
    } else {
      for (int k = threadIdx.x; k < npad; k += blockDim.x)
        s.x2[k] = k < ni ? hash_unit(i + 7919u * (uint32_t)(fresh + 1), k) : 0.0;
      ++fresh;
      __syncthreads();
      project(V, vs, cnt, s.x2, npad, s.hs);
      subtract(V, vs, cnt, s.hs, s.x2, npad);
      project(V, vs, cnt, s.x2, npad, s.h2);
      subtract(V, vs, cnt, s.h2, s.x2, npad);
      const double nn = norm2(s.x2, npad, s.red);
      for (int k = threadIdx.x; k < npad; k += blockDim.x) vn[k] = s.x2[k] / nn;
      __syncthreads();
    }
    nV = cnt + 1;
  }
  if (threadIdx.x == 0) {
    a.nconv[i] = nconv;
    a.steps[i] = steps;
    a.status[i] = status;
  }
}

// Z_i[t, :] = interior entries of L^{-T} U_t (U_t = Ritz vector t in V).
__global__ void __launch_bounds__(kThreads) k_eigvec(EigArgs a, const int32_t* __restrict__ coff,
                                                     const int64_t* __restrict__ zoff,
                                                     const int64_t* __restrict__ int_off,
                                                     const int32_t* __restrict__ int_loc, double* __restrict__ Z,
                                                     int use_smem) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int i = blockIdx.x;
  const int64_t b0 = a.P.blk_off[i];
  const int nb = (int)(a.P.blk_off[i + 1] - b0);
  const int npad = nb * kT;
  const int64_t vs = a.vstride;
  double* base = reinterpret_cast<double*>(smem_raw);
  double* x1 = use_smem ? base : a.vec + (int64_t)i * 2 * vs;
  double* dt = base + (use_smem ? 2 * vs : 0);
  double* tmp = dt + kT * 33;
  BandRef B{a.P.blk_tf + b0, a.P.blk_poff + b0, nb};
  const double* V = a.V + (int64_t)i * a.Kmax * vs;
  const int k = coff[i + 1] - coff[i];
  const int64_t io = int_off[i];
  const int nIi = (int)(int_off[i + 1] - io);
  for (int t = 0; t < k; ++t) {
    for (int e = threadIdx.x; e < npad; e += blockDim.x) x1[e] = V[t * vs + e];
    __syncthreads();
    band_backward<double, double>(a.Bfac, nullptr, a.Bidiag + b0 * kT, B, x1, dt, tmp);
    for (int jj = threadIdx.x; jj < nIi; jj += blockDim.x) Z[zoff[i] + (int64_t)t * nIi + jj] = x1[int_loc[io + jj]];
    __syncthreads();
  }
}

}  // namespace

size_t lanczos_smem(int max_nb) {
  const size_t vec = 2 * (size_t)max_nb * kT * sizeof(double);
  const size_t rest = (kT * 33 + kT + 2 * kMaxK + kMaxK + kWarps) * sizeof(double) + 2 * kMaxK * sizeof(int);
  return vec + rest;
}

void launch_lanczos(const EigArgs& a, cudaStream_t st) {
  const size_t full = lanczos_smem((int)(a.vstride / kT));
  const int use = full <= 200 * 1024;
  const size_t sm = use ? full : lanczos_smem(0);
  cudaFuncSetAttribute(k_lanczos, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_lanczos<<<a.P.N, kThreads, sm, st>>>(a, use);
}

void launch_eigvec(const EigArgs& a, const int32_t* coff, const int64_t* zoff, const int64_t* int_off,
                   const int32_t* int_loc, double* Z, cudaStream_t st) {
  const size_t full = (2 * (size_t)a.vstride + kT * 33 + kT) * sizeof(double);
  const int use = full <= 200 * 1024;
  const size_t sm = use ? full : (kT * 33 + kT) * sizeof(double);
  cudaFuncSetAttribute(k_eigvec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_eigvec<<<a.P.N, kThreads, sm, st>>>(a, coff, zoff, int_off, int_loc, Z, use);
}

}  // namespace lsq
