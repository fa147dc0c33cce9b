// Batched local solves of the preconditioner apply: y_i = C_ii^{-1} R_i r for every
// subdomain in one launch (one CTA per subdomain), plus the fused coarse restriction
// r0_i = Zbar_i^T r(Omega_I,i).
//
// Solve storage.  The factor L_i of the (equilibrated) C_ii is kept block row by
// block row (32 rows each); block row b is one contiguous segment of width columns
// of 32 entries (column-major): first the off-diagonal panel L(b, tf_b .. b-1)
// (offw = width - 32 columns), then the inverse of the diagonal tile L(b,b)^{-1}.
// With the inverse tile, each block step is two dense products:
//   forward  v_b <- L_bb^{-1} (v_b - L_off v_window)
//   backward x_b  = L_bb^{-T} v_b ;  v_window -= L_off^T x_b
// Streaming.  Each CTA reads its segments through a ring of 16 KB shared-memory
// stages filled by bulk asynchronous copies (cp.async.bulk + mbarrier): the forward
// sweep reads the subdomain's storage front to back, the backward sweep back to
// front (each segment's chunks from its end, so the inverse tile arrives first).
// The copies run ahead of the dependency chain of the block steps.  Every wait on a
// stage is bounded; on timeout the kernel sets the error slot and returns.
#include "common.cuh"
#include "kernels.h"

namespace lsq {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

template <class TF> struct Val;
template <> struct Val<double> { static __device__ __forceinline__ double f(double x) { return x; } };
template <> struct Val<float> { static __device__ __forceinline__ float f(float x) { return x; } };
template <> struct Val<__nv_bfloat16> {
  static __device__ __forceinline__ float f(__nv_bfloat16 x) { return __bfloat162float(x); }
};

// Two configurations: 256 threads with 16 KB stages (two CTAs per SM: many subdomains)
// and 512 threads with 32 KB stages (one CTA per SM: subdomains that each have an SM to
// themselves, where one CTA's own issue rate bounds the solve; twice the warps to hide
// the latency of its dependent steps and twice the columns per stage over which the
// per-stage bookkeeping is spread).
constexpr int kStageStd = 16384, kStageFat = 32768;
constexpr long long kWaitCycles = 4000000000ll;  // about two seconds at GB300 clocks

// Byte offset of the local vector v in shared memory: after the ring, the reduction
// buffers and the barriers, rounded up to 16 bytes (vector reads of v).
template <class TA, int S, int NT, int SB>
__host__ __device__ constexpr size_t v_offset() {
  return ((size_t)S * SB + (NT + 64) * sizeof(TA) + (S + 1) * sizeof(uint64_t) + 15) / 16 * 16;
}

// Order of the chunks one CTA consumes: forward sweep, blocks ascending, each segment's
// chunks from its start; backward sweep, blocks descending, each segment's chunks from
// its end.  Chunk k of a segment (counted from its end) covers the columns
// [max(0, width - (k+1) CC), width - k CC).
struct ChunkIter {
  int sweep, b, k, nb;
  const int32_t* tf;
  int CC;
  __device__ int width(int bb) const { return (bb - tf[bb] + 1) * kT; }
  __device__ int nchunks(int bb) const { return (width(bb) + CC - 1) / CC; }
  __device__ void start(const int32_t* tf_, int nb_, int cc) {
    tf = tf_; nb = nb_; CC = cc; sweep = 0; b = 0; k = nchunks(0) - 1;
  }
  __device__ bool done() const { return sweep == 1 && b < 0; }
  __device__ void next() {
    if (sweep == 0) {
      if (k > 0) { --k; return; }
      if (++b < nb) { k = nchunks(b) - 1; return; }
      sweep = 1; b = nb - 1; k = 0;
      return;
    }
    if (k + 1 < nchunks(b)) { ++k; return; }
    --b; k = 0;
  }
};

template <class TF, class TA, int S, int NT, int SB>
__global__ void __launch_bounds__(NT, NT <= 256 ? 2 : 1) k_local_solve(LocalArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int NW = NT / 32;                   // warps
  constexpr int ES = sizeof(TF);
  constexpr int CC = SB / (kT * ES);            // columns per stage
  constexpr int CHUNK = CC * kT;                // elements per stage
  constexpr int G = NT / CC;                    // row groups of the backward panel update
  constexpr int RG = kT / G;                    // rows per group
  constexpr bool kSplit = (ES == 8);            // spread the 32x32 products over the warps
  constexpr bool kVec = (sizeof(TA) == 4);      // FP32 arithmetic: vectorised inner loops
  constexpr int CPW = CC / NW;                  // forward: contiguous columns per warp
  constexpr int XG = 16 / ES;                   // rows per 16-byte read of a column
  constexpr int DC = kT / NW;                   // FP64 diagonal products: columns per warp
  static_assert(G * CC == NT && G * RG == kT, "stage geometry");
  static_assert(!kVec || (CPW % 4 == 0 && CC <= NT), "vectorised geometry");
  static_assert(DC * NW == kT && (DC & (DC - 1)) == 0, "diagonal split");
  TF* ring = reinterpret_cast<TF*>(smem_raw);
  TA* red = reinterpret_cast<TA*>(smem_raw + S * SB);
  TA* tv = red + NW * 32;
  TA* xv = tv + 32;
  uint64_t* bars = reinterpret_cast<uint64_t*>(xv + 32);
  int* abort_flag = reinterpret_cast<int*>(bars + S);
  TA* v = reinterpret_cast<TA*>(smem_raw + v_offset<TA, S, NT, SB>());  // 16-byte aligned

  const int i = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t o0 = a.om_off[i];
  const int ni = (int)(a.om_off[i + 1] - o0);
  const int64_t b0 = a.blk_off[i];
  const int nb = (int)(a.blk_off[i + 1] - b0);
  const TF* fac = reinterpret_cast<const TF*>(a.fac);
  if (nb == 0) return;  // (the host rejects empty subdomains; kept as a guard)
  // The block metadata (first tile column and storage offset of every block row) lives
  // in shared memory behind v: it is read at every stage and block-row transition, and
  // a global round trip there would sit on the dependency chain.
  int64_t* poff = reinterpret_cast<int64_t*>(v + (size_t)nb * kT);  // 16-byte aligned
  int32_t* tf = reinterpret_cast<int32_t*>(poff + nb);
  for (int k = tid; k < nb; k += blockDim.x) {
    poff[k] = a.blk_poff[b0 + k];
    tf[k] = a.blk_tf[b0 + k];
  }

  ChunkIter prod, cons;
  int issued = 0;  // chunks issued so far (issuing thread)
  // The copies are issued by the last warp: warp 0 carries the diagonal products of the
  // dependency chain, while the last warp's columns of a stage are most often the
  // diagonal tile's, which the panel products skip.
  const bool issuer = tid == NT - 32;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();  // barriers initialised, block metadata staged
  auto issue = [&](int stage) {
    const int wd = prod.width(prod.b);
    const int hi = wd - prod.k * CC;
    const int lo = max(0, hi - CC);
    const uint32_t bytes = (uint32_t)((hi - lo) * kT * ES);
    if (!in_range(poff[prod.b] + (int64_t)hi * kT - 1, a.fac_elems, a.err) || !in_range(poff[prod.b], a.fac_elems, a.err)) {
      *abort_flag = 1;  // (bounds-checked build: the copy is not issued; its wait gives up)
      prod.next();
      ++issued;
      return;
    }
    fence_proxy_async();
    mbar_expect_tx(&bars[stage], bytes);
    bulk_g2s(ring + stage * CHUNK, fac + poff[prod.b] + (int64_t)lo * kT, bytes, &bars[stage]);
    prod.next();
    ++issued;
  };
  // (a.stall, a test hook: no copy is issued, every wait below runs out after its bound
  // and the CTA takes the error path with nothing in flight)
  if (issuer && !a.stall) {
    prod.start(tf, nb, CC);
    for (int s = 0; s < S - 1 && !prod.done(); ++s) issue(s);
  }
  // gather r(Omega_i), scaled by the equilibration, while the first stages load
  for (int k = tid; k < nb * kT; k += blockDim.x)
    v[k] = (k < ni && in_range(a.om_glob[o0 + k], a.n_cols, a.err)) ? (TA)(a.r[a.om_glob[o0 + k]] * a.eqs[o0 + k])
                                                                     : (TA)0;
  if (a.coarse) {
    const int c0 = a.coff[i], kk = a.coff[i + 1] - c0;
    const int64_t io = a.int_off[i];
    const int nIi = (int)(a.int_off[i + 1] - io);
    const double* Zi = a.Z + a.zoff[i];
    for (int t = w; t < kk; t += NW) {
      double acc = 0.0;
      for (int jj = lane; jj < nIi; jj += 32) acc += Zi[(int64_t)t * nIi + jj] * a.r[a.int_glob[io + jj]];
      acc = warp_sum(acc);
      if (lane == 0) a.r0[c0 + t] = acc;
    }
  }
  __syncthreads();

  cons.start(tf, nb, CC);
  TA acc = 0;
  TA acc4[4] = {0, 0, 0, 0};                        // FP64: four independent FMA chains
  TA xr[kT];                                        // rotated copy of x_b (vectorised path)
  // this thread's skew of 16-byte groups: consecutive threads read consecutive columns
  // (32 x ES bytes each), so eight threads of a quarter-warp hit eight distinct 16-byte
  // bank groups (BF16: two columns per 128 bytes, so the skew advances every other thread)
  const int rot = kVec ? ((ES == 2 ? tid >> 1 : tid) & (kT / XG - 1)) : 0;
  int q = 0;
  while (!cons.done()) {
    const int stage = q % S;
    if (issuer && !a.stall && !prod.done()) issue((q + S - 1) % S);
    {
      const uint32_t parity = (uint32_t)((q / S) & 1);
      if (!mbar_try_wait(&bars[stage], parity)) {
        const long long t0 = clock64();
        bool ok = false;
        while (!(ok = mbar_try_wait(&bars[stage], parity)))
          if (clock64() - t0 > kWaitCycles) break;
        if (!ok) *abort_flag = 1;
      }
    }
    const TF* ch = ring + stage * CHUNK;
    const int b = cons.b;
    const int t0 = tf[b];
    const int wd = (b - t0 + 1) * kT;
    const int offw = wd - kT;
    const int hi = wd - cons.k * CC;
    const int lo = max(0, hi - CC);
    const int phi = min(hi, offw);  // panel columns of this chunk: [lo, phi)
    const float* sc = a.tsc ? a.tsc + poff[b] / 1024 : nullptr;
    if (cons.sweep == 0) {
      if (cons.k == cons.nchunks(b) - 1) {
        acc = 0;
        acc4[0] = acc4[1] = acc4[2] = acc4[3] = 0;
      }
      TA* vw = v + t0 * kT;
      if constexpr (kVec) {
        // warp w takes the contiguous columns [c0, c0 + CPW) of the chunk (one BF16 tile)
        const int c0 = lo + w * CPW;
        if (c0 < phi) {
          const TF* colp = ch + (c0 - lo) * kT + lane;
          TA s0 = 0, s1 = 0;
          if (c0 + CPW <= phi) {
#pragma unroll
            for (int j = 0; j < CPW; j += 4) {
              const float4 v4 = *reinterpret_cast<const float4*>(vw + c0 + j);
              s0 += Val<TF>::f(colp[(j + 0) * kT]) * v4.x;
              s1 += Val<TF>::f(colp[(j + 1) * kT]) * v4.y;
              s0 += Val<TF>::f(colp[(j + 2) * kT]) * v4.z;
              s1 += Val<TF>::f(colp[(j + 3) * kT]) * v4.w;
            }
          } else {
            for (int c = c0; c < phi; ++c) s0 += Val<TF>::f(colp[(c - c0) * kT]) * vw[c];
          }
          acc += sc ? (s0 + s1) * (TA)sc[c0 >> 5] : (s0 + s1);
        }
      } else {
        // FP64: warp w takes the contiguous columns [c0, c0 + CPW) of the chunk, the
        // window entries read two at a time, four independent FMA chains (the FP64 units
        // are few, so a single dependent chain per thread leaves them idle)
        const int c0 = lo + w * CPW;
        const TF* colp = ch + (c0 - lo) * kT + lane;
        if (c0 + CPW <= phi) {
#pragma unroll
          for (int j = 0; j < CPW; j += 2) {
            const double2 v2 = *reinterpret_cast<const double2*>(vw + c0 + j);
            acc4[(j >> 1) & 3] += Val<TF>::f(colp[j * kT]) * v2.x;
            acc4[((j >> 1) + 2) & 3] += Val<TF>::f(colp[(j + 1) * kT]) * v2.y;
          }
        } else if (c0 < phi) {
#pragma unroll
          for (int j = 0; j < CPW; ++j)
            if (c0 + j < phi) acc4[j & 3] += Val<TF>::f(colp[j * kT]) * vw[c0 + j];
        }
      }
      if (cons.k == 0) {
        if constexpr (!kVec) acc = (acc4[0] + acc4[1]) + (acc4[2] + acc4[3]);
        red[w * 32 + lane] = acc;
        __syncthreads();
        const TF* D = ch + (offw - lo) * kT;  // inverse tile, column-major
        const TA dsc = sc ? (TA)sc[offw >> 5] : (TA)1;
        if (w == 0) {
          TA s = 0;
#pragma unroll
          for (int u = 0; u < NW; ++u) s += red[u * 32 + lane];
          tv[lane] = v[b * kT + lane] - s;
          __syncwarp();
          if (!kSplit) {
            TA x0 = 0, x1 = 0;  // two FMA chains
#pragma unroll 8
            for (int c = 0; c < kT; c += 2) {
              x0 += Val<TF>::f(D[c * kT + lane]) * tv[c];
              x1 += Val<TF>::f(D[(c + 1) * kT + lane]) * tv[c + 1];
            }
            v[b * kT + lane] = (x0 + x1) * dsc;
          }
        }
        if (kSplit) {  // FP64: the 32x32 product spread over the warps (the FP64 pipe is narrow)
          // (the sums above stay on warp 0: FP64 additions with few active lanes would
          // occupy the FP64 units like full-warp ones)
          __syncthreads();
          TA x = 0;
#pragma unroll
          for (int c = DC * w; c < DC * w + DC; ++c) x += Val<TF>::f(D[c * kT + lane]) * tv[c];
          red[w * 32 + lane] = x;
          __syncthreads();
          if (w == 0) {
            TA s = 0;
#pragma unroll
            for (int u = 0; u < NW; ++u) s += red[u * 32 + lane];
            v[b * kT + lane] = s * dsc;
          }
        }
      }
    } else {
      if (cons.k == 0) {
        const TF* D = ch + (offw - lo) * kT;
        const TA dsc = sc ? (TA)sc[offw >> 5] : (TA)1;
        if (!kSplit) {
          if (w == 0) tv[lane] = v[b * kT + lane];
          __syncthreads();
          if (w == 0) {
            TA x0 = 0, x1 = 0;  // two FMA chains
#pragma unroll 8
            for (int u = 0; u < kT; u += 2) {
              const int r0 = (u + lane) & 31, r1 = (u + 1 + lane) & 31;  // skewed walk: no bank conflicts
              x0 += Val<TF>::f(D[lane * kT + r0]) * tv[r0];
              x1 += Val<TF>::f(D[lane * kT + r1]) * tv[r1];
            }
            TA x = (x0 + x1) * dsc;
            xv[lane] = x;
            v[b * kT + lane] = x;
          }
        } else {
          // (v_b is final: the last panel update reaching it ended with the previous stage)
          TA x = 0;
#pragma unroll
          for (int u = 0; u < DC; ++u) {
            const int r = DC * w + ((u + lane) & (DC - 1));
            x += Val<TF>::f(D[lane * kT + r]) * v[b * kT + r];
          }
          red[w * 32 + lane] = x;
          __syncthreads();
          if (w == 0) {
            TA s = 0;
#pragma unroll
            for (int u = 0; u < NW; ++u) s += red[u * 32 + lane];
            s *= dsc;
            xv[lane] = s;
            v[b * kT + lane] = s;
          }
        }
        __syncthreads();
        if constexpr (kVec) {
          // this thread's copy of x_b, rotated like its skewed column reads (16-byte reads)
#pragma unroll
          for (int g = 0; g < kT / XG; ++g)
#pragma unroll
            for (int h = 0; h < XG; h += 4) {
              const float4 t = *reinterpret_cast<const float4*>(xv + ((g + rot) & (kT / XG - 1)) * XG + h);
              xr[g * XG + h] = t.x; xr[g * XG + h + 1] = t.y; xr[g * XG + h + 2] = t.z; xr[g * XG + h + 3] = t.w;
            }
        }
      }
      // v_window -= L_off^T x_b
      TA* vw = v + t0 * kT;
      if constexpr (kVec) {
        // one thread per column; 16-byte reads walk the column in a rotated order
        const int c = lo + tid;
        if (tid < CC && c < phi) {
          const TF* col = ch + (c - lo) * kT;
          TA s = 0;
          if constexpr (ES == 4) {
            const float4* c4 = reinterpret_cast<const float4*>(col);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const float4 u = c4[(k + rot) & 7];
              s += u.x * xr[4 * k] + u.y * xr[4 * k + 1] + u.z * xr[4 * k + 2] + u.w * xr[4 * k + 3];
            }
          } else {
            const uint4* c8 = reinterpret_cast<const uint4*>(col);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint4 u = c8[(k + rot) & 3];
              const uint32_t wds[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
              for (int h = 0; h < 4; ++h) {
                s += __uint_as_float(wds[h] << 16) * xr[8 * k + 2 * h];
                s += __uint_as_float(wds[h] & 0xffff0000u) * xr[8 * k + 2 * h + 1];
              }
            }
          }
          if (sc) s *= (TA)sc[c >> 5];
          vw[c] -= s;
        }
      } else {
      // FP64: four row groups of 8 rows per column, their partial sums added by the
      // first group through shared memory (fewer FP64 additions than a shuffle tree: the
      // FP64 units are this kernel's bottleneck)
      const int cl = tid % CC, g = tid / CC;
      const int c = lo + cl;
      TA s = 0;
      if (c < phi) {
        const TF* col = ch + cl * kT + g * RG;
        TA s1 = 0;  // two FMA chains
#pragma unroll
        for (int u = 0; u < RG; u += 2) {
          const int r0 = (u + c) & (RG - 1), r1 = (u + 1 + c) & (RG - 1);
          s += Val<TF>::f(col[r0]) * xv[g * RG + r0];
          s1 += Val<TF>::f(col[r1]) * xv[g * RG + r1];
        }
        s += s1;
        if (sc) s *= (TA)sc[c >> 5];
      }
      red[g * CC + cl] = s;
      __syncthreads();
      if (g == 0 && c < phi) {
        TA t = 0;
#pragma unroll
        for (int u = 0; u < G; ++u) t += red[u * CC + cl];
        vw[c] -= t;
      }
      }
    }
    __syncthreads();
    if (*abort_flag) break;
    cons.next();
    ++q;
  }
  if (*abort_flag) {
    if (issuer) {
      if (a.err[0] == 0.0) a.err[0] = kErrTimeout;
      // bounded drain of the copies still in flight before the CTA's shared memory is released
      for (int qq = q; qq < issued; ++qq) {
        const long long t0 = clock64();
        while (!mbar_try_wait(&bars[qq % S], (uint32_t)((qq / S) & 1)))
          if (clock64() - t0 > kWaitCycles) break;
      }
    }
    return;
  }
  for (int k = tid; k < ni; k += blockDim.x) a.y[o0 + k] = (double)v[k] * a.eqs[o0 + k];
}

// Block-envelope factor (row-major panels, diagonal tile last) + inverse diagonal
// tiles (row-major, FP64) -> solve storage of the given precision (see above).
template <class TF>
__global__ void __launch_bounds__(kThreads) k_to_solve_layout(const int64_t* __restrict__ poff,
                                                              const double* __restrict__ L,
                                                              const double* __restrict__ dinv, TF* __restrict__ dst,
                                                              float* __restrict__ tsc) {
  (void)tsc;
  const int64_t g = blockIdx.x;
  const int64_t po = poff[g];
  const int width = (int)((poff[g + 1] - po) / kT);
  const int offw = width - kT;
  for (int64_t e = threadIdx.x; e < (int64_t)width * kT; e += blockDim.x) {
    const int c = (int)(e >> 5), r = (int)(e & 31);
    const double val = c < offw ? L[po + (int64_t)r * width + c] : dinv[g * 1024 + r * 32 + (c - offw)];
    dst[po + e] = (TF)val;
  }
}

template <>
__global__ void __launch_bounds__(kThreads) k_to_solve_layout<__nv_bfloat16>(const int64_t* __restrict__ poff,
                                                                             const double* __restrict__ L,
                                                                             const double* __restrict__ dinv,
                                                                             __nv_bfloat16* __restrict__ dst,
                                                                             float* __restrict__ tsc) {
  __shared__ double red[kWarps];
  const int64_t g = blockIdx.x;
  const int64_t po = poff[g];
  const int width = (int)((poff[g + 1] - po) / kT);
  const int offw = width - kT;
  auto src = [&](int c, int r) -> double {
    return c < offw ? L[po + (int64_t)r * width + c] : dinv[g * 1024 + r * 32 + (c - offw)];
  };
  for (int t = 0; t < width / kT; ++t) {
    double mx = 0.0;
    for (int e = threadIdx.x; e < 1024; e += blockDim.x) mx = fmax(mx, fabs(src(t * kT + (e >> 5), e & 31)));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    double m = 0.0;
    for (int k = 0; k < kWarps; ++k) m = fmax(m, red[k]);
    const double sc = m > 0.0 ? m : 1.0;
    if (threadIdx.x == 0) tsc[po / 1024 + t] = (float)sc;
    for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
      const int c = t * kT + (e >> 5), r = e & 31;
      dst[po + (int64_t)c * kT + r] = __float2bfloat16_rn((float)(src(c, r) / sc));
    }
    __syncthreads();
  }
}

template <class TF, class TA, int S, int NT, int SB>
size_t smem_bytes(int max_nb) {
  return v_offset<TA, S, NT, SB>() + (size_t)max_nb * (kT * sizeof(TA) + sizeof(int64_t) + sizeof(int32_t));
}

template <class TF, class TA, int S, int NT, int SB>
void launch_impl(int N, int max_nb, const LocalArgs& a, cudaStream_t st) {
  static size_t raised = 0;
  const size_t sm = smem_bytes<TF, TA, S, NT, SB>(max_nb);
  if (sm > 48 * 1024 && sm > raised) {
    cudaFuncSetAttribute(k_local_solve<TF, TA, S, NT, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    raised = sm;
  }
  k_local_solve<TF, TA, S, NT, SB><<<N, NT, sm, st>>>(a);
}

}  // namespace

// Configuration 1 (256 threads, 16 KB stages): as deep a ring as two CTAs per SM allow
// (228 KB per SM) for subdomains of up to 181 block rows.  Configuration 2 (512
// threads, 32 KB stages, one CTA per SM): four stages (two for FP64, whose local vector
// is twice as large).
size_t local_solve_smem(int prec, int max_nb, int config) {
  if (config == 2) {
    if (prec == 0) return smem_bytes<double, double, 2, 512, kStageFat>(max_nb);
    if (prec == 1) return smem_bytes<float, float, 4, 512, kStageFat>(max_nb);
    return smem_bytes<__nv_bfloat16, float, 4, 512, kStageFat>(max_nb);
  }
  if (prec == 0) return smem_bytes<double, double, 3, 256, kStageStd>(max_nb);
  if (prec == 1) return smem_bytes<float, float, 5, 256, kStageStd>(max_nb);
  return smem_bytes<__nv_bfloat16, float, 5, 256, kStageStd>(max_nb);
}

void launch_local_solve(int prec, int config, int N, int max_nb, const LocalArgs& a, cudaStream_t st) {
  if (config == 2) {
    if (prec == 0) launch_impl<double, double, 2, 512, kStageFat>(N, max_nb, a, st);
    else if (prec == 1) launch_impl<float, float, 4, 512, kStageFat>(N, max_nb, a, st);
    else launch_impl<__nv_bfloat16, float, 4, 512, kStageFat>(N, max_nb, a, st);
    return;
  }
  if (prec == 0) launch_impl<double, double, 3, 256, kStageStd>(N, max_nb, a, st);
  else if (prec == 1) launch_impl<float, float, 5, 256, kStageStd>(N, max_nb, a, st);
  else launch_impl<__nv_bfloat16, float, 5, 256, kStageStd>(N, max_nb, a, st);
}

void launch_to_solve_layout(int prec, int64_t nblocks, const int64_t* poff, const double* L, const double* dinv,
                            void* dst, float* tsc, cudaStream_t st) {
  if (nblocks <= 0) return;
  if (prec == 0) k_to_solve_layout<double><<<(unsigned)nblocks, kThreads, 0, st>>>(poff, L, dinv, (double*)dst, nullptr);
  else if (prec == 1) k_to_solve_layout<float><<<(unsigned)nblocks, kThreads, 0, st>>>(poff, L, dinv, (float*)dst, nullptr);
  else k_to_solve_layout<__nv_bfloat16><<<(unsigned)nblocks, kThreads, 0, st>>>(poff, L, dinv, (__nv_bfloat16*)dst, tsc);
}

}  // namespace lsq
