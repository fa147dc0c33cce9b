// Multi right-hand-side kernels: R <= 32 right-hand sides advance together through one
// launch of every kernel, and with a batched handle several independent problems
// share the launches as well.
//
// Block vectors are interleaved: entry (j, k) of an n x R block sits at j * R + k, so
// the R values of one column are contiguous (256 bytes for R = 32) and one warp reads
// them with one coalesced access.  A warp's lanes are split into groups of Rp lanes
// (R rounded up to a power of two); lane k of a group serves right-hand side k.
//
// Reductions run per chunk, a range of at most 256 columns inside one problem: each
// chunk writes its partial sums to part[c * 32 + k]; one finishing block per problem
// adds its chunks' partials in chunk order, so every (problem, right-hand side) scalar
// is reproducible bit for bit across runs and graph replays.
//
// The local solves stream every factor tile once per apply for all R right-hand
// sides: one CTA per subdomain (taken from a work queue, largest first) walks the
// tiles front to back (forward sweep) and back to front (backward sweep) through a
// ring of shared-memory stages filled by bulk asynchronous copies; the R solution
// columns of the tiles in the envelope window stay in a shared-memory ring of tiles.
#include "common.cuh"
#include "kernels.h"

namespace lsq {

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void bar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ bool bar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

constexpr long long kSpinCycles = 4000000000ll;  // about two seconds at GB300 clocks

struct Lanes {
  int g, k, G;
  __device__ explicit Lanes(int Rp) {
    const int lane = threadIdx.x & 31;
    g = lane / Rp;
    k = lane % Rp;
    G = 32 / Rp;
  }
};

// Per-rhs total of v over the lane groups and warps of the block -> out[k], k < R.
__device__ void chunk_total(double v, int Rp, int R, double* red, double* out) {
  for (int o = Rp; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane < Rp) red[w * 32 + lane] = v;
  __syncthreads();
  if ((int)threadIdx.x < R) {
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < kWarps; ++u) s += red[u * 32 + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// ---- sparse products ------------------------------------------------------------------

// Y = A X for R right-hand sides (A in CSR; one lane group per row).
__global__ void __launch_bounds__(kThreads) k_b_spmm_csr(int64_t m, const int64_t* __restrict__ rp,
                                                         const int32_t* __restrict__ col,
                                                         const double* __restrict__ val,
                                                         const double* __restrict__ X, double* __restrict__ Y,
                                                         int R, int Rp) {
  const Lanes L(Rp);
  const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if (L.k >= R) return;
  for (int64_t r = wg * L.G + L.g; r < m; r += nw * L.G) {
    const int64_t e0 = rp[r], e1 = rp[r + 1];
    double a0 = 0.0, a1 = 0.0;
    int64_t e = e0;
    for (; e + 1 < e1; e += 2) {
      const int32_t c0 = col[e], c1 = col[e + 1];
      const double v0 = val[e], v1 = val[e + 1];
      a0 += v0 * X[(int64_t)c0 * R + L.k];
      a1 += v1 * X[(int64_t)c1 * R + L.k];
    }
    if (e < e1) a0 += val[e] * X[(int64_t)col[e] * R + L.k];
    Y[r * R + L.k] = a0 + a1;
  }
}

// W = A^T Q (A^T in CSC, one lane group per column) and, with part, the per-chunk
// partials of D . W (D == nullptr: W . W).
__global__ void __launch_bounds__(kThreads) k_b_spmm_csc(BChunks ch, const int64_t* __restrict__ cp,
                                                         const int32_t* __restrict__ row,
                                                         const double* __restrict__ val,
                                                         const double* __restrict__ Q, double* __restrict__ W,
                                                         int R, int Rp, const double* __restrict__ D,
                                                         double* __restrict__ part) {
  __shared__ double red[kWarps * 32];
  const Lanes L(Rp);
  const int w = threadIdx.x >> 5;
  for (int64_t c = blockIdx.x; c < ch.n; c += gridDim.x) {
    const int64_t s = ch.start[c], e = ch.start[c + 1];
    double d = 0.0;
    if (L.k < R) {
      for (int64_t j = s + w * L.G + L.g; j < e; j += kWarps * L.G) {
        const int64_t t0 = cp[j], t1 = cp[j + 1];
        double a0 = 0.0, a1 = 0.0;
        int64_t t = t0;
        for (; t + 1 < t1; t += 2) {
          const int32_t r0 = row[t], r1 = row[t + 1];
          a0 += val[t] * Q[(int64_t)r0 * R + L.k];
          a1 += val[t + 1] * Q[(int64_t)r1 * R + L.k];
        }
        if (t < t1) a0 += val[t] * Q[(int64_t)row[t] * R + L.k];
        const double acc = a0 + a1;
        W[j * R + L.k] = acc;
        d += (D ? D[j * R + L.k] : acc) * acc;
      }
    }
    if (part) chunk_total(d, Rp, R, red, part + c * 32);
  }
}

// ---- CG vector kernels ----------------------------------------------------------------

// X += alpha P; Rold = R (if given); R -= alpha W; partials of R . R.
__global__ void __launch_bounds__(kThreads) k_b_update(BChunks ch, int R, int Rp, const double* __restrict__ alpha,
                                                       const double* __restrict__ P, const double* __restrict__ W,
                                                       double* __restrict__ X, double* __restrict__ Rv,
                                                       double* __restrict__ Rold, double* __restrict__ part) {
  __shared__ double red[kWarps * 32];
  const Lanes L(Rp);
  const int w = threadIdx.x >> 5;
  for (int64_t c = blockIdx.x; c < ch.n; c += gridDim.x) {
    const int64_t s = ch.start[c], e = ch.start[c + 1];
    double d = 0.0;
    if (L.k < R) {
      const double a = alpha[(int64_t)ch.prob[c] * R + L.k];
      for (int64_t j = s + w * L.G + L.g; j < e; j += kWarps * L.G) {
        const int64_t x = j * R + L.k;
        X[x] += a * P[x];
        double r = Rv[x];
        if (Rold) Rold[x] = r;
        r -= a * W[x];
        Rv[x] = r;
        d += r * r;
      }
    }
    chunk_total(d, Rp, R, red, part + c * 32);
  }
}

// P = Z + beta P (init: P = Z).
__global__ void __launch_bounds__(kThreads) k_b_pupdate(BChunks ch, int R, int Rp, const double* __restrict__ beta,
                                                        const double* __restrict__ Z, double* __restrict__ P,
                                                        int init) {
  const Lanes L(Rp);
  const int w = threadIdx.x >> 5;
  if (L.k >= R) return;
  for (int64_t c = blockIdx.x; c < ch.n; c += gridDim.x) {
    const int64_t s = ch.start[c], e = ch.start[c + 1];
    const double b = init ? 0.0 : beta[(int64_t)ch.prob[c] * R + L.k];
    for (int64_t j = s + w * L.G + L.g; j < e; j += kWarps * L.G) {
      const int64_t x = j * R + L.k;
      P[x] = init ? Z[x] : Z[x] + b * P[x];
    }
  }
}

// Finishing block per problem: sums the chunk partials (in chunk order) and applies
// the CG scalar step of `mode` to every right-hand side of the problem.
__global__ void __launch_bounds__(kThreads) k_b_finish(const int64_t* __restrict__ pc_off,
                                                       const double* __restrict__ part,
                                                       const double* __restrict__ part2, int R, BScal s, int mode,
                                                       int flex) {
  __shared__ double red[kWarps][32], red2[kWarps][32];
  __shared__ int cnt;
  const int q = blockIdx.x;
  const int w = threadIdx.x >> 5, k = threadIdx.x & 31;
  const int64_t c0 = pc_off[q], c1 = pc_off[q + 1];
  double a = 0.0, b = 0.0;
  if (k < R) {
    for (int64_t c = c0 + w; c < c1; c += kWarps) {
      a += part[c * 32 + k];
      if (part2) b += part2[c * 32 + k];
    }
  }
  red[w][k] = a;
  red2[w][k] = b;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  if ((int)threadIdx.x < R) {
    double x = 0.0, y = 0.0;
#pragma unroll
    for (int u = 0; u < kWarps; ++u) {
      x += red[u][k];
      y += red2[u][k];
    }
    const int64_t i = (int64_t)q * R + k;
    const int act = s.act[i];
    switch (mode) {
      case kFinGG: s.gg[i] = x; break;
      case kFinTT: s.tt[i] = x; break;
      case kFinAlpha: {
        const double al = act ? s.rzold[i] / x : 0.0;
        s.alpha[i] = al;
        if (act && (!(x > 0.0) || !isfinite(al))) s.stat[1] = 1;
        break;
      }
      case kFinRR: {
        s.rr[i] = x;
        if (!isfinite(x)) s.stat[1] = 1;
        if (act) {
          s.its[i] += 1;
          const int still = x > s.thr2[i] ? 1 : 0;
          s.act[i] = still;
          if (still) atomicAdd(&cnt, 1);
        }
        break;
      }
      case kFinBeta0: s.rzold[i] = x; s.beta[i] = 0.0; break;
      default: {  // kFinBeta
        const double bt = act ? (flex ? x - y : x) / s.rzold[i] : 0.0;
        s.beta[i] = bt;
        s.rzold[i] = x;
        if (act && !isfinite(bt)) s.stat[1] = 1;
        break;
      }
    }
  }
  __syncthreads();
  if (mode == kFinRR && threadIdx.x == 0 && cnt) atomicAdd(&s.stat[0], cnt);
}

// Z = sum over the copies of every column in the subdomains of Y (local solutions)
//   + coarse prolongation; partials of R . Z and (flexible) Rold . Z.
__global__ void __launch_bounds__(kThreads) k_b_scatter(BChunks ch, BScatterArgs a) {
  __shared__ double red[kWarps * 32];
  const Lanes L(a.Rp);
  const int R = a.R;
  const int w = threadIdx.x >> 5;
  for (int64_t c = blockIdx.x; c < ch.n; c += gridDim.x) {
    const int64_t s = ch.start[c], e = ch.start[c + 1];
    double d1 = 0.0, d2 = 0.0;
    if (L.k < R) {
      for (int64_t j = s + w * L.G + L.g; j < e; j += kWarps * L.G) {
        double z = 0.0;
        for (int64_t t = a.map_ptr[j]; t < a.map_ptr[j + 1]; ++t) z += a.Y[a.map_idx[t] * R + L.k];
        if (a.coarse && a.ZT) {
          const int i = a.part[j];
          const int cc = a.coff[i], kk = a.coff[i + 1] - cc, kp = (kk + 3) & ~3;
          const float4* z4 = reinterpret_cast<const float4*>(a.ZT + a.zt_off[i] + (int64_t)a.jj_of[j] * kp);
          const float* y0 = a.Y0f + (int64_t)cc * R + L.k;
          float zc = 0.f;
          for (int t4 = 0; 4 * t4 < kk; ++t4) {
            const float4 zz = z4[t4];
            const int t = 4 * t4;
            zc += zz.x * y0[(int64_t)t * R];
            if (t + 1 < kk) zc += zz.y * y0[(int64_t)(t + 1) * R];
            if (t + 2 < kk) zc += zz.z * y0[(int64_t)(t + 2) * R];
            if (t + 3 < kk) zc += zz.w * y0[(int64_t)(t + 3) * R];
          }
          z += (double)zc;
        } else if (a.coarse) {
          const int i = a.part[j];
          const int cc = a.coff[i], kk = a.coff[i + 1] - cc;
          const int64_t nIi = a.nI[i];
          const double* Zi = a.Z + a.zoff[i] + a.jj_of[j];
          for (int t = 0; t < kk; ++t) z += Zi[t * nIi] * a.Y0[(int64_t)(cc + t) * R + L.k];
        }
        const int64_t x = j * R + L.k;
        a.Zout[x] = z;
        d1 += a.Rv[x] * z;
        if (a.Rold) d2 += a.Rold[x] * z;
      }
    }
    chunk_total(d1, a.Rp, R, red, a.part1 + c * 32);
    if (a.Rold) chunk_total(d2, a.Rp, R, red, a.part2 + c * 32);
  }
}

// R0[(c0 + t), k] = sum_jj Zbar_i[t, jj] R[Omega_I,i[jj], k] (one block per subdomain).
__global__ void __launch_bounds__(kThreads) k_b_restrict(int R, int Rp, const int64_t* __restrict__ int_off,
                                                         const int32_t* __restrict__ int_glob,
                                                         const int64_t* __restrict__ zoff,
                                                         const int32_t* __restrict__ coff, const double* __restrict__ Z,
                                                         const double* __restrict__ Rv, double* __restrict__ R0) {
  const int i = blockIdx.x;
  const Lanes L(Rp);
  const int w = threadIdx.x >> 5;
  const int cc = coff[i], kk = coff[i + 1] - cc;
  const int64_t io = int_off[i];
  const int nIi = (int)(int_off[i + 1] - io);
  const double* Zi = Z + zoff[i];
  for (int tb = 0; tb < kk; tb += 4 * kWarps) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int jj = L.g; jj < nIi; jj += L.G) {
      const double rv = L.k < R ? Rv[(int64_t)int_glob[io + jj] * R + L.k] : 0.0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int t = tb + w + kWarps * u;
        if (t < kk) acc[u] += Zi[(int64_t)t * nIi + jj] * rv;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      double v = acc[u];
      for (int o = Rp; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      const int t = tb + w + kWarps * u;
      if (t < kk && L.g == 0 && L.k < R) R0[(int64_t)(cc + t) * R + L.k] = v;
    }
  }
}

// FP32 transposed copy of the coarse basis: ZT[zt_off[i] + jj * kp + t] = Zbar_i[t, jj]
// (kp = k_i rounded up to 4, so one interior column's k_i values are 16-byte aligned).
__global__ void __launch_bounds__(kThreads) k_b_ztrans(const int64_t* __restrict__ int_off,
                                                       const int64_t* __restrict__ zoff,
                                                       const int32_t* __restrict__ coff,
                                                       const int64_t* __restrict__ zt_off,
                                                       const double* __restrict__ Z, float* __restrict__ ZT) {
  const int i = blockIdx.x;
  const int kk = coff[i + 1] - coff[i], kp = (kk + 3) & ~3;
  const int64_t nIi = int_off[i + 1] - int_off[i];
  for (int64_t e = threadIdx.x; e < nIi * kp; e += blockDim.x) {
    const int64_t jj = e / kp;
    const int t = (int)(e % kp);
    ZT[zt_off[i] + e] = t < kk ? (float)Z[zoff[i] + (int64_t)t * nIi + jj] : 0.f;
  }
}

// FP32 restriction R0[(c0 + t), k] = sum_jj ZT[jj, t] R[Omega_I,i[jj], k] for the mixed
// forms: warps split the interior columns, lane k keeps 32 coarse sums in registers,
// the warps' sums meet in shared memory.
__global__ void __launch_bounds__(kThreads) k_b_restrict32(int R, const int64_t* __restrict__ int_off,
                                                           const int32_t* __restrict__ int_glob,
                                                           const int32_t* __restrict__ coff,
                                                           const int64_t* __restrict__ zt_off,
                                                           const float* __restrict__ ZT,
                                                           const double* __restrict__ Rv, double* __restrict__ R0) {
  __shared__ float red[kWarps][32][33];
  const int i = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int cc = coff[i], kk = coff[i + 1] - cc, kp = (kk + 3) & ~3;
  const int64_t io = int_off[i];
  const int nIi = (int)(int_off[i + 1] - io);
  const float* Zi = ZT + zt_off[i];
  for (int tb = 0; tb < kk; tb += 32) {
    const int tn = min(32, kk - tb);
    float acc[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) acc[t] = 0.f;
    for (int jj = w; jj < nIi; jj += kWarps) {
      const float rv = lane < R ? (float)Rv[(int64_t)int_glob[io + jj] * R + lane] : 0.f;
      const float4* z4 = reinterpret_cast<const float4*>(Zi + (int64_t)jj * kp + tb);
#pragma unroll
      for (int t4 = 0; t4 < 8; ++t4) {
        if (4 * t4 < tn) {
          const float4 z = z4[t4];
          acc[4 * t4 + 0] += z.x * rv; acc[4 * t4 + 1] += z.y * rv;
          acc[4 * t4 + 2] += z.z * rv; acc[4 * t4 + 3] += z.w * rv;
        }
      }
    }
#pragma unroll
    for (int t = 0; t < 32; ++t) red[w][t][lane] = acc[t];
    __syncthreads();
    for (int e = threadIdx.x; e < tn * 32; e += blockDim.x) {
      const int t = e >> 5, k = e & 31;
      float s = 0.f;
#pragma unroll
      for (int u = 0; u < kWarps; ++u) s += red[u][t][k];
      if (k < R) R0[(int64_t)(cc + tb + t) * R + k] = (double)s;
    }
    __syncthreads();
  }
}

// Y0 = C00_q^{-1} R0 on every problem's dense block; one block per (problem, 32-row tile).
__global__ void __launch_bounds__(kThreads) k_b_coarse(int R, const int32_t* __restrict__ ct_prob,
                                                       const int32_t* __restrict__ ct_row, CoarseBlocks cb,
                                                       const int32_t* __restrict__ n0q, const double* __restrict__ Xinv,
                                                       const double* __restrict__ R0, double* __restrict__ Y0,
                                                       float* __restrict__ Y0f) {
  const int q = ct_prob[blockIdx.x], rt = ct_row[blockIdx.x];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane >= R) return;
  const int64_t ld = cb.ld[q];
  const int c0 = cb.c0[q], nq = n0q[q];
  const double* X = Xinv + cb.base[q];
  const int rbase = rt * 32 + 4 * w;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int c = 0; c < nq; ++c) {
    const double rv = R0[(int64_t)(c0 + c) * R + lane];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] += X[(int64_t)(rbase + u) * ld + c] * rv;
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
    if (rbase + u < nq) {
      Y0[(int64_t)(c0 + rbase + u) * R + lane] = acc[u];
      if (Y0f) Y0f[(int64_t)(c0 + rbase + u) * R + lane] = (float)acc[u];
    }
}

// ---- layout conversions ---------------------------------------------------------------

// Bb[r', k] = Bu[k * m + perm[r']] (caller's column-major right-hand sides -> interleaved
// rows of the row-reordered matrix).
__global__ void __launch_bounds__(kThreads) k_b_load_rows(int64_t m, int R, int Rp, const int32_t* __restrict__ perm,
                                                          const double* __restrict__ Bu, double* __restrict__ Bb) {
  const Lanes L(Rp);
  const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if (L.k >= R) return;
  for (int64_t r = wg * L.G + L.g; r < m; r += nw * L.G) Bb[r * R + L.k] = Bu[(int64_t)L.k * m + perm[r]];
}

// Xu[k * n + j] = Xb[j * R + k] (interleaved -> column-major), 32 columns per tile.
__global__ void __launch_bounds__(kThreads) k_b_store_cols(int64_t n, int R, const double* __restrict__ Xb,
                                                           double* __restrict__ Xu) {
  __shared__ double t[32][33];
  for (int64_t j0 = (int64_t)blockIdx.x * 32; j0 < n; j0 += (int64_t)gridDim.x * 32) {
    const int cols = (int)(n - j0 < 32 ? n - j0 : 32);
    for (int e = threadIdx.x; e < cols * R; e += blockDim.x) t[e / R][e % R] = Xb[j0 * R + e];
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * R; e += blockDim.x) {
      const int k = e / 32, jj = e % 32;
      if (jj < cols) Xu[(int64_t)k * n + j0 + jj] = t[jj][k];
    }
    __syncthreads();
  }
}

// Xb[j * R + k] = Xu[k * n + j] (caller's column-major n-vectors -> interleaved), 32
// columns per tile.
__global__ void __launch_bounds__(kThreads) k_b_load_cols(int64_t n, int R, const double* __restrict__ Xu,
                                                          double* __restrict__ Xb) {
  __shared__ double t[32][33];
  for (int64_t j0 = (int64_t)blockIdx.x * 32; j0 < n; j0 += (int64_t)gridDim.x * 32) {
    const int cols = (int)(n - j0 < 32 ? n - j0 : 32);
    for (int e = threadIdx.x; e < 32 * R; e += blockDim.x) {
      const int k = e / 32, jj = e % 32;
      if (jj < cols) t[jj][k] = Xu[(int64_t)k * n + j0 + jj];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < cols * R; e += blockDim.x) Xb[j0 * R + e] = t[e / R][e % R];
    __syncthreads();
  }
}

// Yu[k * m + perm[r']] = Yb[r' * R + k] (interleaved rows of the row-reordered matrix ->
// the caller's column-major m-vectors).
__global__ void __launch_bounds__(kThreads) k_b_store_rows(int64_t m, int R, int Rp, const int32_t* __restrict__ perm,
                                                           const double* __restrict__ Yb, double* __restrict__ Yu) {
  const Lanes L(Rp);
  const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if (L.k >= R) return;
  for (int64_t r = wg * L.G + L.g; r < m; r += nw * L.G) Yu[(int64_t)L.k * m + perm[r]] = Yb[r * R + L.k];
}

// W = G - W with the per-chunk partials of W . W (the residual of C x = g when W = C x;
// with W = 0 beforehand it copies G and gives ||G||^2).
__global__ void __launch_bounds__(kThreads) k_b_resid(BChunks ch, int R, int Rp, const double* __restrict__ G,
                                                      double* __restrict__ W, double* __restrict__ part) {
  __shared__ double red[kWarps * 32];
  const Lanes L(Rp);
  const int w = threadIdx.x >> 5;
  for (int64_t c = blockIdx.x; c < ch.n; c += gridDim.x) {
    const int64_t s = ch.start[c], e = ch.start[c + 1];
    double d = 0.0;
    if (L.k < R) {
      for (int64_t j = s + w * L.G + L.g; j < e; j += kWarps * L.G) {
        const int64_t x = j * R + L.k;
        const double v = G[x] - W[x];
        W[x] = v;
        d += v * v;
      }
    }
    chunk_total(d, Rp, R, red, part + c * 32);
  }
}

// Gradient on the stored entries, summed over the right-hand sides: for entry e of row
// r' of the row-reordered matrix (column c), out[entmap[e]] = sum_k rho[r', k] lam[c, k]
// - (A lam)[r', k] x[c, k]; one warp per row, lane k per right-hand side.
__global__ void __launch_bounds__(kThreads) k_b_grad_vals(int64_t m, const int64_t* __restrict__ rp,
                                                          const int32_t* __restrict__ col,
                                                          const int64_t* __restrict__ entmap, int R,
                                                          const double* __restrict__ rho,
                                                          const double* __restrict__ lam,
                                                          const double* __restrict__ Al,
                                                          const double* __restrict__ X, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = wg; r < m; r += nw) {
    const double rr = lane < R ? rho[r * R + lane] : 0.0;
    const double ar = lane < R ? Al[r * R + lane] : 0.0;
    for (int64_t e = rp[r]; e < rp[r + 1]; ++e) {
      const int64_t c = col[e];
      double v = lane < R ? rr * lam[c * R + lane] - ar * X[c * R + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) out[entmap[e]] = v;
    }
  }
}

__global__ void k_b_sub(int64_t len, const double* __restrict__ a, double* __restrict__ b) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x)
    b[e] = a[e] - b[e];
}

// ---- multi right-hand-side local solves -------------------------------------------------

template <class TF> struct Ld4;
template <> struct Ld4<float> {
  static __device__ __forceinline__ void f(const float* p, float& a, float& b, float& c, float& d) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = v.x; b = v.y; c = v.z; d = v.w;
  }
};
template <> struct Ld4<__nv_bfloat16> {
  static __device__ __forceinline__ void f(const __nv_bfloat16* p, float& a, float& b, float& c, float& d) {
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    a = __uint_as_float(v.x << 16); b = __uint_as_float(v.x & 0xffff0000u);
    c = __uint_as_float(v.y << 16); d = __uint_as_float(v.y & 0xffff0000u);
  }
};
template <> struct Ld4<double> {
  static __device__ __forceinline__ void f(const double* p, double& a, double& b, double& c, double& d) {
    const double2 u = *reinterpret_cast<const double2*>(p);
    const double2 v = *reinterpret_cast<const double2*>(p + 2);
    a = u.x; b = u.y; c = v.x; d = v.y;
  }
};

// acc[u] += sc * sum_c T[c*32 + r0 + u] V[c*32 + lane]     (T column-major: T(r, c))
template <class TF, class TA>
__device__ __forceinline__ void tile_colmajor(const TF* T, const TA* V, TA acc[4], TA sc, int r0, int lane) {
  TA s0 = 0, s1 = 0, s2 = 0, s3 = 0;
#pragma unroll 8
  for (int c = 0; c < kT; ++c) {
    const TA v = V[c * kT + lane];
    TA l0, l1, l2, l3;
    Ld4<TF>::f(T + c * kT + r0, l0, l1, l2, l3);
    s0 += l0 * v; s1 += l1 * v; s2 += l2 * v; s3 += l3 * v;
  }
  acc[0] += sc * s0; acc[1] += sc * s1; acc[2] += sc * s2; acc[3] += sc * s3;
}

// acc[u] = sc * sum_q T[(r0 + u)*32 + q] V[q*32 + lane]    (the transposed product)
template <class TF, class TA>
__device__ __forceinline__ void tile_transposed(const TF* T, const TA* V, TA acc[4], TA sc, int r0, int lane) {
  TA s[4] = {0, 0, 0, 0};
#pragma unroll 2
  for (int q = 0; q < kT; q += 4) {
    const TA v0 = V[(q + 0) * kT + lane], v1 = V[(q + 1) * kT + lane];
    const TA v2 = V[(q + 2) * kT + lane], v3 = V[(q + 3) * kT + lane];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      TA l0, l1, l2, l3;
      Ld4<TF>::f(T + (r0 + u) * kT + q, l0, l1, l2, l3);
      s[u] += l0 * v0 + l1 * v1 + l2 * v2 + l3 * v3;
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) acc[u] = sc * s[u];
}

template <class TF, class TA>
__global__ void __launch_bounds__(kThreads, 1) k_b_local(BLocalArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int ES = sizeof(TF);
  constexpr int S = kBlockRingBytes / (kT * kT * ES);  // factor tiles in flight
  TF* fring = reinterpret_cast<TF*>(smem);
  TA* vring = reinterpret_cast<TA*>(smem + kBlockRingBytes);
  TA* tin = vring + (size_t)a.ring * kT * kT;
  uint64_t* bars = reinterpret_cast<uint64_t*>(tin + kT * kT);
  int* sh = reinterpret_cast<int*>(bars + S);  // sh[0]: subdomain, sh[1]: abort
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int r0 = 4 * w;
  const int R = a.R, RING = a.ring;
  const TF* fac = reinterpret_cast<const TF*>(a.fac);
  TA* spill = reinterpret_cast<TA*>(a.Vg);
  if (tid == 0) {
    for (int s = 0; s < S; ++s) bar_init(&bars[s], 1);
    sh[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t q = 0;       // tiles consumed by this CTA so far (every thread)
  uint32_t issued = 0;  // tiles issued so far (thread 0)
  for (;;) {
    if (tid == 0) {
      const unsigned t = atomicAdd(a.qctr, 1u);
      sh[0] = t < (unsigned)a.N ? a.order[t] : -1;
    }
    __syncthreads();
    const int i = sh[0];
    if (i < 0) break;
    const int64_t o0 = a.om_off[i];
    const int ni = (int)(a.om_off[i + 1] - o0);
    const int64_t b0 = a.blk_off[i];
    const int nb = (int)(a.blk_off[i + 1] - b0);
    const int32_t* tf = a.blk_tf + b0;
    const int64_t T0 = a.blk_poff[b0] / (kT * kT);
    const int64_t ntile = a.blk_poff[b0 + nb] / (kT * kT) - T0;
    // tile sequence: forward T0 .. T0+ntile-1, then backward T0+ntile-1 .. T0
    int64_t pnext = 0;
    auto issue = [&]() {
      const int64_t tile = pnext < ntile ? T0 + pnext : T0 + 2 * ntile - 1 - pnext;
      const int stage = (int)(issued % S);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bar_expect_tx(&bars[stage], kT * kT * ES);
      copy_g2s(fring + (size_t)stage * kT * kT, fac + tile * kT * kT, kT * kT * ES, &bars[stage]);
      ++pnext;
      ++issued;
    };
    if (tid == 0 && !a.stall)  // (a.stall, a test hook: no copies, so every wait runs out)
      while (pnext < 2 * ntile && issued < q + S) issue();
    auto wait_tile = [&]() -> const TF* {
      const int stage = (int)(q % S);
      const uint32_t parity = (q / S) & 1u;
      if (!bar_try_wait(&bars[stage], parity)) {
        const long long t0 = clock64();
        bool ok = false;
        while (!(ok = bar_try_wait(&bars[stage], parity)))
          if (clock64() - t0 > kSpinCycles) break;
        if (!ok) sh[1] = 1;
      }
      return fring + (size_t)stage * kT * kT;
    };
    // every thread is done with the current stage: hand it back to the producer
    // (on a give-up q keeps pointing at the tile that was waited for, so the final
    // drain covers it)
    auto release = [&]() -> bool {
      __syncthreads();
      if (sh[1]) return false;
      ++q;
      if (tid == 0 && !a.stall && pnext < 2 * ntile) issue();
      return true;
    };
    auto tile_scale = [&](uint32_t seq) -> TA {
      if (!a.tsc) return (TA)1;
      const int64_t tile = seq < ntile ? T0 + seq : T0 + 2 * ntile - 1 - seq;
      return (TA)a.tsc[tile];
    };
    bool ok = true;
    uint32_t seq = 0;  // position in this subdomain's tile sequence
    // forward sweep: v_b = L_bb^{-1} (r_b - sum_t L_bt v_t)
    for (int b = 0; b < nb && ok; ++b) {
      for (int e = tid; e < kT * kT; e += kThreads) {
        const int rr = e >> 5, k = e & 31, l = b * kT + rr;
        TA v = 0;
        if (l < ni && k < R && in_range(a.om_glob[o0 + l], a.n_cols, a.err))
          v = (TA)(a.Rv[(int64_t)a.om_glob[o0 + l] * R + k] * a.eqs[o0 + l]);
        tin[e] = v;
      }
      __syncthreads();
      TA acc[4] = {0, 0, 0, 0};
      const int tfb = tf[b];  // a register: the barriers in release() would force reloads
      for (int t = tfb; t < b && ok; ++t) {
        const TF* T = wait_tile();
        tile_colmajor<TF, TA>(T, vring + (size_t)(t % RING) * kT * kT, acc, tile_scale(seq), r0, lane);
        ++seq;
        ok = release();
      }
      if (!ok) break;
      const TF* D = wait_tile();
#pragma unroll
      for (int u = 0; u < 4; ++u) tin[(r0 + u) * kT + lane] -= acc[u];
      __syncthreads();
      TA y[4] = {0, 0, 0, 0};
      tile_colmajor<TF, TA>(D, tin, y, tile_scale(seq), r0, lane);
      ++seq;
      TA* vb = vring + (size_t)(b % RING) * kT * kT;
#pragma unroll
      for (int u = 0; u < 4; ++u) vb[(r0 + u) * kT + lane] = y[u];
      if (b < nb - RING) {
        TA* sp = spill + (size_t)(b0 + b) * kT * kT;
#pragma unroll
        for (int u = 0; u < 4; ++u) sp[(r0 + u) * kT + lane] = y[u];
      }
      ok = release();
    }
    // backward sweep: x_b = L_bb^{-T} v_b, then v_t -= L_bt^T x_b for the window tiles
    for (int b = nb - 1; b >= 0 && ok; --b) {
      const TF* D = wait_tile();
      TA x[4];
      tile_transposed<TF, TA>(D, vring + (size_t)(b % RING) * kT * kT, x, tile_scale(seq), r0, lane);
      ++seq;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        tin[(r0 + u) * kT + lane] = x[u];
        const int l = b * kT + r0 + u;
        if (l < ni && lane < R) a.Y[(o0 + l) * R + lane] = (double)x[u] * a.eqs[o0 + l];
      }
      ok = release();
      const int tfb = tf[b];
      for (int t = b - 1; t >= tfb && ok; --t) {
        const TF* T = wait_tile();
        TA sdec[4];
        tile_transposed<TF, TA>(T, tin, sdec, tile_scale(seq), r0, lane);
        ++seq;
        TA* vt = vring + (size_t)(t % RING) * kT * kT;
#pragma unroll
        for (int u = 0; u < 4; ++u) vt[(r0 + u) * kT + lane] -= sdec[u];
        ok = release();
      }
      if (ok && b - RING >= 0) {
        const TA* sp = spill + (size_t)(b0 + b - RING) * kT * kT;
        TA* vb = vring + (size_t)(b % RING) * kT * kT;
        for (int e = tid; e < kT * kT; e += kThreads) vb[e] = sp[e];
        __syncthreads();
      }
    }
    if (!ok) break;
  }
  if (sh[1]) {
    if (tid == 0) {
      if (a.err[0] == 0.0) a.err[0] = kErrTimeout;
      // bounded drain of the copies still in flight before the shared memory is released
      for (uint32_t qq = q; qq < issued; ++qq) {
        const long long t0 = clock64();
        while (!bar_try_wait(&bars[qq % S], (qq / S) & 1u))
          if (clock64() - t0 > kSpinCycles) break;
      }
    }
  }
}

// ---- tensor-core local solves (FP32 factors) ------------------------------------------
// Each 32 x 32 block step is a product of a factor tile (or its transpose) with the
// 32 x R solution tile, done as 2 x 4 warp tiles of m16n8k8 TF32 MMAs: warp w owns the
// output rows [16 (w / 4), +16) and right-hand sides [8 (w % 4), +8).  The solution
// operand is split into a TF32 head and a TF32 tail (two MMAs), which keeps it at
// about FP32 accuracy; the factor is TF32 (stored pre-rounded).  Factor and solution
// tiles are row-major with the swizzle (r, c) -> 32 r + (c xor s(r)), s(r) = 8 (r % 4) +
// 4 ((r / 4) % 2): the fragments of T, of T^T and of the solution tile then all hit 32
// distinct banks, and each fragment address is a per-thread offset (TcOff) plus a
// multiple of 256.

__device__ __forceinline__ int swz(int r, int c) { return r * kT + (c ^ (8 * (r & 3) + 4 * ((r >> 2) & 1))); }

// Fragment offsets of one thread (lane = 4 g + t of warp (mb, nb)):
//   a[ks][j]  T(16 mb + g, 8 ks + t + 4 j)                 (+256: row + 8)
//   t[h][j]   T(8 ks + t + 4 j, 16 mb + g + 8 h) - 256 ks
//   b[j]      V(8 ks + t + 4 j, 8 nb + g) - 256 ks
//   o[h]      output pair (16 mb + g + 8 h, 8 nb + 2 t + {0, 1})
struct TcOff {
  int a[4][2], t[2][2], b[2], o[2];
};

__device__ __forceinline__ TcOff tc_offsets(int mb, int nb, int g, int t) {
  TcOff f;
  const int gb = (g >> 2) & 1, g3 = g & 3, r0 = 16 * mb + g;
#pragma unroll
  for (int ks = 0; ks < 4; ++ks)
#pragma unroll
    for (int j = 0; j < 2; ++j) f.a[ks][j] = r0 * 32 + t + 8 * (ks ^ g3) + 4 * (j ^ gb);
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int j = 0; j < 2; ++j) f.t[h][j] = 32 * t + 128 * j + 8 * ((2 * mb + h) ^ t) + 4 * (gb ^ j) + g3;
#pragma unroll
  for (int j = 0; j < 2; ++j) f.b[j] = 32 * t + 128 * j + 8 * (nb ^ t) + 4 * (gb ^ j) + g3;
#pragma unroll
  for (int h = 0; h < 2; ++h) f.o[h] = (r0 + 8 * h) * 32 + 8 * (nb ^ g3) + ((2 * t) ^ (4 * gb));
  return f;
}

__device__ __forceinline__ uint32_t tf32_bits(float x) {
  uint32_t y;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void mma_tf32(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// c += op(T) V on the warp's 16 x 8 output block; op(T) = T or T^T.  The head and
// tail products go to two accumulators (two independent MMA chains), summed at the end.
template <bool TRANS>
__device__ __forceinline__ void tile_mma(const float* T, const float* V, float c[4], const TcOff& f) {
  float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    uint32_t a[4];
    if (!TRANS) {
      a[0] = __float_as_uint(T[f.a[ks][0]]);
      a[1] = __float_as_uint(T[f.a[ks][0] + 256]);
      a[2] = __float_as_uint(T[f.a[ks][1]]);
      a[3] = __float_as_uint(T[f.a[ks][1] + 256]);
    } else {
      a[0] = __float_as_uint(T[256 * ks + f.t[0][0]]);
      a[1] = __float_as_uint(T[256 * ks + f.t[1][0]]);
      a[2] = __float_as_uint(T[256 * ks + f.t[0][1]]);
      a[3] = __float_as_uint(T[256 * ks + f.t[1][1]]);
    }
    const float v0 = V[256 * ks + f.b[0]], v1 = V[256 * ks + f.b[1]];
    const uint32_t h0 = tf32_bits(v0), h1 = tf32_bits(v1);
    const uint32_t l0 = tf32_bits(v0 - __uint_as_float(h0)), l1 = tf32_bits(v1 - __uint_as_float(h1));
    mma_tf32(c, a, h0, h1);
    mma_tf32(d, a, l0, l1);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) c[u] += d[u];
}

// The warp's accumulator elements: (row, col) of c[2 h + j] = (16 mb + g + 8 h, 8 nb + 2 t + j).
__device__ __forceinline__ float2* frag_ptr(float* tile, const TcOff& f, int h) {
  return reinterpret_cast<float2*>(tile + f.o[h]);
}

__global__ void __launch_bounds__(kThreads, 1) k_b_local_tc(BLocalArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int S = kBlockRingBytes / (kT * kT * 4);
  float* fring = reinterpret_cast<float*>(smem);
  float* vring = reinterpret_cast<float*>(smem + kBlockRingBytes);
  float* tin = vring + (size_t)a.ring * kT * kT;
  uint64_t* bars = reinterpret_cast<uint64_t*>(tin + kT * kT);
  int* sh = reinterpret_cast<int*>(bars + S);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int mb = w >> 2, nb = w & 3, g = lane >> 2, t4 = lane & 3;
  const TcOff off = tc_offsets(mb, nb, g, t4);
  const int R = a.R, RING = a.ring;
  const float* fac = reinterpret_cast<const float*>(a.fac);
  float* spill = reinterpret_cast<float*>(a.Vg);
  if (tid == 0) {
    for (int s = 0; s < S; ++s) bar_init(&bars[s], 1);
    sh[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t q = 0, issued = 0;
  for (;;) {
    if (tid == 0) {
      const unsigned tk = atomicAdd(a.qctr, 1u);
      sh[0] = tk < (unsigned)a.N ? a.order[tk] : -1;
    }
    __syncthreads();
    const int i = sh[0];
    if (i < 0) break;
    const int64_t o0 = a.om_off[i];
    const int ni = (int)(a.om_off[i + 1] - o0);
    const int64_t b0 = a.blk_off[i];
    const int nbk = (int)(a.blk_off[i + 1] - b0);
    const int32_t* tf = a.blk_tf + b0;
    const int64_t T0 = a.blk_poff[b0] / (kT * kT);
    const int64_t ntile = a.blk_poff[b0 + nbk] / (kT * kT) - T0;
    int64_t pnext = 0;
    auto issue = [&]() {
      const int64_t tile = pnext < ntile ? T0 + pnext : T0 + 2 * ntile - 1 - pnext;
      const int stage = (int)(issued % S);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bar_expect_tx(&bars[stage], kT * kT * 4);
      copy_g2s(fring + (size_t)stage * kT * kT, fac + tile * kT * kT, kT * kT * 4, &bars[stage]);
      ++pnext;
      ++issued;
    };
    if (tid == 0 && !a.stall)  // (a.stall, a test hook: no copies, so every wait runs out)
      while (pnext < 2 * ntile && issued < q + S) issue();
    // tile q + off of the sequence (off = 0, 1; both are in flight: S >= 2)
    auto wait_tile = [&](uint32_t off) -> const float* {
      const int stage = (int)((q + off) % S);
      const uint32_t parity = ((q + off) / S) & 1u;
      if (!bar_try_wait(&bars[stage], parity)) {
        const long long c0 = clock64();
        bool ok = false;
        while (!(ok = bar_try_wait(&bars[stage], parity)))
          if (clock64() - c0 > kSpinCycles) break;
        if (!ok) sh[1] = 1;
      }
      return fring + (size_t)stage * kT * kT;
    };
    // (on a give-up q keeps pointing at the tile that was waited for, so the final
    // drain covers it)
    auto release = [&](uint32_t used) -> bool {
      __syncthreads();
      if (sh[1]) return false;
      q += used;
      if (tid == 0 && !a.stall)
        while (pnext < 2 * ntile && issued < q + S) issue();
      return true;
    };
    bool ok = true;
    // this thread's 4 entries (rows e / 32, rhs e % 32, e = tid + 256 u) of block row b's
    // gathered right-hand side, loaded one block row ahead
    float pre[4];
    auto fetch_rhs = [&](int b) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = tid + kThreads * u, rr = e >> 5, k = e & 31, l = b * kT + rr;
        pre[u] = (l < ni && k < R && in_range(a.om_glob[o0 + l], a.n_cols, a.err))
                     ? (float)(a.Rv[(int64_t)a.om_glob[o0 + l] * R + k] * a.eqs[o0 + l])
                     : 0.f;
      }
    };
    fetch_rhs(0);
    // first tile column of the next block row, loaded one block row ahead (in a register:
    // the barriers of release() would otherwise force a reload on the dependency chain)
    int tf_next = tf[0];
    // forward sweep
    for (int b = 0; b < nbk && ok; ++b) {
      const int tfb = tf_next;
      if (b + 1 < nbk) tf_next = tf[b + 1];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = tid + kThreads * u;
        tin[swz(e >> 5, e & 31)] = pre[u];
      }
      if (b + 1 < nbk) fetch_rhs(b + 1);
      __syncthreads();
      // panel tiles two at a time (independent products, one barrier per pair)
      float c[4] = {0.f, 0.f, 0.f, 0.f}, c2[4] = {0.f, 0.f, 0.f, 0.f};
      int t = tfb;
      for (; t + 1 < b && ok; t += 2) {
        const float* T1 = wait_tile(0);
        const float* T2 = wait_tile(1);
        tile_mma<false>(T1, vring + (size_t)(t % RING) * kT * kT, c, off);
        tile_mma<false>(T2, vring + (size_t)((t + 1) % RING) * kT * kT, c2, off);
        ok = release(2);
      }
      if (ok && t < b) {
        const float* T = wait_tile(0);
        tile_mma<false>(T, vring + (size_t)(t % RING) * kT * kT, c, off);
        ok = release(1);
      }
      if (!ok) break;
#pragma unroll
      for (int u = 0; u < 4; ++u) c[u] += c2[u];
      const float* D = wait_tile(0);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float2* p = frag_ptr(tin, off, h);
        float2 v = *p;
        v.x -= c[2 * h];
        v.y -= c[2 * h + 1];
        *p = v;
      }
      __syncthreads();
      float y[4] = {0.f, 0.f, 0.f, 0.f};
      tile_mma<false>(D, tin, y, off);
      float* vb = vring + (size_t)(b % RING) * kT * kT;
#pragma unroll
      for (int h = 0; h < 2; ++h) *frag_ptr(vb, off, h) = make_float2(y[2 * h], y[2 * h + 1]);
      if (b < nbk - RING) {
        float* sp = spill + (size_t)(b0 + b) * kT * kT;
#pragma unroll
        for (int h = 0; h < 2; ++h) *frag_ptr(sp, off, h) = make_float2(y[2 * h], y[2 * h + 1]);
      }
      ok = release(1);
    }
    // backward sweep; tf and the equilibration scales of this thread's output rows are
    // loaded one block row ahead
    auto fetch_scales = [&](int b, double sc[2]) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int l = b * kT + mb * 16 + g + 8 * h;
        sc[h] = l < ni ? a.eqs[o0 + l] : 0.0;
      }
    };
    double sc_next[2];
    if (nbk > 0) {
      tf_next = tf[nbk - 1];
      fetch_scales(nbk - 1, sc_next);
    }
    for (int b = nbk - 1; b >= 0 && ok; --b) {
      const int tfb = tf_next;
      const double scb[2] = {sc_next[0], sc_next[1]};
      if (b > 0) {
        tf_next = tf[b - 1];
        fetch_scales(b - 1, sc_next);
      }
      // the forward values of tile b - RING, which takes slot b % RING after this step
      float4 refill = make_float4(0.f, 0.f, 0.f, 0.f);
      if (b - RING >= 0) refill = reinterpret_cast<const float4*>(spill + (size_t)(b0 + b - RING) * kT * kT)[tid];
      const float* D = wait_tile(0);
      float x[4] = {0.f, 0.f, 0.f, 0.f};
      tile_mma<true>(D, vring + (size_t)(b % RING) * kT * kT, x, off);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        *frag_ptr(tin, off, h) = make_float2(x[2 * h], x[2 * h + 1]);
        const int l = b * kT + mb * 16 + g + 8 * h;
        const int k = nb * 8 + 2 * t4;
        if (l < ni) {
          const double sc = scb[h];
          if (k < R) a.Y[(o0 + l) * R + k] = (double)x[2 * h] * sc;
          if (k + 1 < R) a.Y[(o0 + l) * R + k + 1] = (double)x[2 * h + 1] * sc;
        }
      }
      ok = release(1);
      // window updates v_t -= L_bt^T x_b, two tiles (two different slots) per barrier
      auto update = [&](const float* T, int tt) {
        float s4[4] = {0.f, 0.f, 0.f, 0.f};
        tile_mma<true>(T, tin, s4, off);
        float* vt = vring + (size_t)(tt % RING) * kT * kT;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float2* p = frag_ptr(vt, off, h);
          float2 v = *p;
          v.x -= s4[2 * h];
          v.y -= s4[2 * h + 1];
          *p = v;
        }
      };
      int t = b - 1;
      for (; t - 1 >= tfb && ok; t -= 2) {
        const float* T1 = wait_tile(0);
        const float* T2 = wait_tile(1);
        update(T1, t);
        update(T2, t - 1);
        ok = release(2);
      }
      if (ok && t >= tfb) {
        update(wait_tile(0), t);
        ok = release(1);
      }
      if (ok && b - RING >= 0) {
        reinterpret_cast<float4*>(vring + (size_t)(b % RING) * kT * kT)[tid] = refill;
        __syncthreads();
      }
    }
    if (!ok) break;
  }
  if (sh[1]) {
    if (tid == 0) {
      if (a.err[0] == 0.0) a.err[0] = kErrTimeout;
      for (uint32_t qq = q; qq < issued; ++qq) {
        const long long c0 = clock64();
        while (!bar_try_wait(&bars[qq % S], (qq / S) & 1u))
          if (clock64() - c0 > kSpinCycles) break;
      }
    }
  }
}

// FP32 solve storage (column-major tiles) -> TF32-rounded swizzled row-major tiles.
__global__ void k_b_swizzle(int64_t nelem, const float* __restrict__ src, float* __restrict__ dst) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nelem; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t tile = e >> 10;
    const int r = (int)(e & 31), c = (int)((e >> 5) & 31);  // source element (c * 32 + r)
    dst[(tile << 10) + swz(r, c)] = __uint_as_float(tf32_bits(src[e]));
  }
}

int grid_rows(int64_t rows, int G) {
  const int64_t warps = (rows + G - 1) / G;
  const int64_t g = (warps + kWarps - 1) / kWarps;
  return (int)(g < 1 ? 1 : (g > 16384 ? 16384 : g));
}

int grid_chunks(int64_t n) { return (int)(n < 1 ? 1 : (n > 1 << 30 ? 1 << 30 : n)); }

int pow2_at_least(int R) {
  int p = 1;
  while (p < R) p <<= 1;
  return p;
}

// Raises the kernel's dynamic shared-memory limit when a larger ring needs it (the
// first call for a handle comes from setup, outside any stream capture).
template <class TF, class TA>
void raise_smem(size_t sm) {
  static size_t raised = 0;
  if (sm > 48 * 1024 && sm > raised) {
    cudaFuncSetAttribute(k_b_local<TF, TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    raised = sm;
  }
}

template <class TF, class TA>
void local_impl(const BLocalArgs& a, int grid, cudaStream_t st) {
  const size_t sm = block_local_smem(sizeof(TF), sizeof(TA), a.ring);
  raise_smem<TF, TA>(sm);
  k_b_local<TF, TA><<<grid, kThreads, sm, st>>>(a);
}

template <class TF, class TA>
int local_occ(int ring) {
  const size_t sm = block_local_smem(sizeof(TF), sizeof(TA), ring);
  raise_smem<TF, TA>(sm);
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_b_local<TF, TA>, kThreads, sm) != cudaSuccess) occ = 0;
  return occ;
}

}  // namespace

size_t block_local_smem(int fac_bytes, int arith_bytes, int ring) {
  (void)fac_bytes;
  const int S = kBlockRingBytes / (kT * kT * fac_bytes);
  return (size_t)kBlockRingBytes + (size_t)(ring + 1) * kT * kT * arith_bytes + (size_t)S * 8 + 16;
}

int block_local_occupancy(int prec, int ring) {
  if (prec == 0) return local_occ<double, double>(ring);
  if (prec == 1) return local_occ<float, float>(ring);
  return local_occ<__nv_bfloat16, float>(ring);
}

void launch_b_local(int prec, const BLocalArgs& a, int grid, cudaStream_t st) {
  cudaMemsetAsync(a.qctr, 0, sizeof(unsigned), st);
  if (prec == 0) local_impl<double, double>(a, grid, st);
  else if (prec == 1) local_impl<float, float>(a, grid, st);
  else local_impl<__nv_bfloat16, float>(a, grid, st);
}

int block_local_tc_occupancy(int ring) {
  const size_t sm = block_local_smem(4, 4, ring);
  static size_t raised = 0;
  if (sm > 48 * 1024 && sm > raised) {
    cudaFuncSetAttribute(k_b_local_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    raised = sm;
  }
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_b_local_tc, kThreads, sm) != cudaSuccess) occ = 0;
  return occ;
}

void launch_b_local_tc(const BLocalArgs& a, int grid, cudaStream_t st) {
  cudaMemsetAsync(a.qctr, 0, sizeof(unsigned), st);
  k_b_local_tc<<<grid, kThreads, block_local_smem(4, 4, a.ring), st>>>(a);
}

void launch_b_swizzle(int64_t nelem, const float* src, float* dst, cudaStream_t st) {
  int64_t g = (nelem + kThreads - 1) / kThreads;
  if (g > 8192) g = 8192;
  if (g < 1) g = 1;
  k_b_swizzle<<<(int)g, kThreads, 0, st>>>(nelem, src, dst);
}

void launch_b_spmm_csr(const CsrDev& A, const double* X, double* Y, int R, cudaStream_t st) {
  const int Rp = pow2_at_least(R);
  k_b_spmm_csr<<<grid_rows(A.m, 32 / Rp), kThreads, 0, st>>>(A.m, A.row_ptr, A.col, A.val, X, Y, R, Rp);
}

void launch_b_spmm_csc(const BChunks& ch, const CscDev& At, const double* Q, double* W, int R, const double* D,
                       double* part, cudaStream_t st) {
  k_b_spmm_csc<<<grid_chunks(ch.n), kThreads, 0, st>>>(ch, At.col_ptr, At.row, At.val, Q, W, R, pow2_at_least(R), D,
                                                      part);
}

void launch_b_update(const BChunks& ch, int R, const double* alpha, const double* P, const double* W, double* X,
                     double* Rv, double* Rold, double* part, cudaStream_t st) {
  k_b_update<<<grid_chunks(ch.n), kThreads, 0, st>>>(ch, R, pow2_at_least(R), alpha, P, W, X, Rv, Rold, part);
}

void launch_b_pupdate(const BChunks& ch, int R, const double* beta, const double* Z, double* P, int init,
                      cudaStream_t st) {
  k_b_pupdate<<<grid_chunks(ch.n), kThreads, 0, st>>>(ch, R, pow2_at_least(R), beta, Z, P, init);
}

void launch_b_finish(int nprob, const int64_t* pc_off, const double* part, const double* part2, int R,
                     const BScal& s, int mode, int flex, cudaStream_t st) {
  k_b_finish<<<nprob, kThreads, 0, st>>>(pc_off, part, part2, R, s, mode, flex);
}

void launch_b_scatter(const BChunks& ch, const BScatterArgs& a, cudaStream_t st) {
  k_b_scatter<<<grid_chunks(ch.n), kThreads, 0, st>>>(ch, a);
}

void launch_b_restrict(int N, int R, const int64_t* int_off, const int32_t* int_glob, const int64_t* zoff,
                       const int32_t* coff, const double* Z, const double* Rv, double* R0, cudaStream_t st) {
  k_b_restrict<<<N, kThreads, 0, st>>>(R, pow2_at_least(R), int_off, int_glob, zoff, coff, Z, Rv, R0);
}

void launch_b_coarse(int ntiles, int R, const int32_t* ct_prob, const int32_t* ct_row, const CoarseBlocks& cb,
                     const int32_t* n0q, const double* Xinv, const double* R0, double* Y0, float* Y0f,
                     cudaStream_t st) {
  if (ntiles <= 0) return;
  k_b_coarse<<<ntiles, kThreads, 0, st>>>(R, ct_prob, ct_row, cb, n0q, Xinv, R0, Y0, Y0f);
}

void launch_b_ztrans(int N, const int64_t* int_off, const int64_t* zoff, const int32_t* coff, const int64_t* zt_off,
                     const double* Z, float* ZT, cudaStream_t st) {
  k_b_ztrans<<<N, kThreads, 0, st>>>(int_off, zoff, coff, zt_off, Z, ZT);
}

void launch_b_restrict32(int N, int R, const int64_t* int_off, const int32_t* int_glob, const int32_t* coff,
                         const int64_t* zt_off, const float* ZT, const double* Rv, double* R0, cudaStream_t st) {
  k_b_restrict32<<<N, kThreads, 0, st>>>(R, int_off, int_glob, coff, zt_off, ZT, Rv, R0);
}

void launch_b_load_rows(int64_t m, int R, const int32_t* perm, const double* Bu, double* Bb, cudaStream_t st) {
  const int Rp = pow2_at_least(R);
  k_b_load_rows<<<grid_rows(m, 32 / Rp), kThreads, 0, st>>>(m, R, Rp, perm, Bu, Bb);
}

void launch_b_store_cols(int64_t n, int R, const double* Xb, double* Xu, cudaStream_t st) {
  const int64_t tiles = (n + 31) / 32;
  k_b_store_cols<<<(int)(tiles > 65536 ? 65536 : tiles), kThreads, 0, st>>>(n, R, Xb, Xu);
}

void launch_b_load_cols(int64_t n, int R, const double* Xu, double* Xb, cudaStream_t st) {
  const int64_t tiles = (n + 31) / 32;
  k_b_load_cols<<<(int)(tiles > 65536 ? 65536 : tiles), kThreads, 0, st>>>(n, R, Xu, Xb);
}

void launch_b_store_rows(int64_t m, int R, const int32_t* perm, const double* Yb, double* Yu, cudaStream_t st) {
  const int Rp = pow2_at_least(R);
  k_b_store_rows<<<grid_rows(m, 32 / Rp), kThreads, 0, st>>>(m, R, Rp, perm, Yb, Yu);
}

void launch_b_resid(const BChunks& ch, int R, const double* G, double* W, double* part, cudaStream_t st) {
  k_b_resid<<<grid_chunks(ch.n), kThreads, 0, st>>>(ch, R, pow2_at_least(R), G, W, part);
}

void launch_b_grad_vals(const CsrDev& A, const int64_t* entmap, int R, const double* rho, const double* lam,
                        const double* Al, const double* X, double* out, cudaStream_t st) {
  k_b_grad_vals<<<grid_rows(A.m, 1), kThreads, 0, st>>>(A.m, A.row_ptr, A.col, entmap, R, rho, lam, Al, X, out);
}

void launch_b_sub(int64_t len, const double* a, double* b, cudaStream_t st) {
  int64_t g = (len + kThreads - 1) / kThreads;
  if (g > 4864) g = 4864;
  if (g < 1) g = 1;
  k_b_sub<<<(int)g, kThreads, 0, st>>>(len, a, b);
}

}  // namespace lsq
