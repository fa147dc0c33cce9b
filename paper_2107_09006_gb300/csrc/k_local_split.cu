// Batched local solves with each subdomain split over a cluster of C CTAs (FP32 factors).
//
// Same solve storage and arithmetic as k_local_solve (forward v_b <- L_bb^{-1}(v_b -
// L_off v_window), backward x_b = L_bb^{-T} v_b; v_window -= L_off^T x_b), for
// subdomains that have an SM each to spare: C CTAs (one cluster) share one subdomain's
// factor stream.  Chunk k of a block row's segment (counted from its end, CC columns
// each) belongs to CTA k mod C, so CTA 0 holds every diagonal tile and takes every
// diagonal step; CTA r > 0 only ever touches tiles at least r T rows below the diagonal
// (T = CC / 32), which CTA 0 finished r T steps earlier.  The CTAs exchange 32-entry
// vectors through distributed shared memory (stores to the peer's shared memory, then
// one release-arrive per lane on the peer's mbarrier):
//   forward:  CTA r sends its partial sum of row b to CTA 0; CTA 0 sends every finished
//             v_b to the CTAs that will read it;
//   backward: CTA 0 sends x_b to every CTA; CTA r accumulates its updates of v in a
//             zeroed copy and sends block j's sum to CTA 0 after row j + r T, the last
//             row in which it touches block j.
// Each CTA sums what it receives in rank order, so the result is deterministic.
// Message slots form rings of D rows (D > (C - 1) T), indexed by the message's place in
// its sweep (row or block b in the forward sweep, nb - 1 - b in the backward sweep, so
// that slot o mod D sees its messages in order and the wait for message o expects phase
// parity (o / D) mod 2); the waits that every row makes keep a sender from reusing a
// slot its receiver has not read.  Every wait is bounded;
// a CTA whose wait gives up sets the error slot and stops, its peers' waits on it give
// up in turn, and all CTAs of the cluster meet at a final cluster barrier before any of
// them exits (no CTA leaves while a peer may still write into its shared memory).
#include "common.cuh"
#include "kernels.h"

namespace lsq {

namespace {

constexpr int kSplitThreads = 512;
constexpr int kSplitStage = 32768;  // bytes per ring stage (256 FP32 columns)
constexpr int kSplitStages = 4;
constexpr int kSplitRing = 16;      // message slots (rows)
constexpr long long kSplitWait = 4000000000ll;  // about two seconds at GB300 clocks

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ int cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return (int)r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// address of the same shared-memory object in CTA `rank` of this cluster
__device__ __forceinline__ uint32_t peer_addr(const void* p, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(su32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_peer(uint32_t addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void arrive_peer(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(bar))
               : "memory");
}
// stage barrier (completed by a bulk copy of this CTA)
__device__ __forceinline__ bool try_stage(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// message barrier (completed by peers' release-arrives at cluster scope)
__device__ __forceinline__ bool try_msg(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
template <bool kMsg>
__device__ __forceinline__ void bounded_wait(uint64_t* bar, uint32_t parity, int* abort_flag) {
  auto probe = [&]() { return kMsg ? try_msg(bar, parity) : try_stage(bar, parity); };
  if (probe()) return;
  const long long t0 = clock64();
  while (!probe())
    if (clock64() - t0 > kSplitWait) {
      *abort_flag = 1;
      return;
    }
}

// The chunks one CTA owns, in the order it consumes them: forward sweep, rows
// ascending, each row's owned chunks from the segment's start (k descending);
// backward sweep, rows descending, k ascending.  Rows without an owned chunk are
// skipped (the issuing thread's view; the consumer walks every row).
struct OwnIter {
  int sweep, b, k, nb, r, C, CC;
  const int32_t* tf;
  __device__ int nch(int bb) const { return ((bb - tf[bb] + 1) * kT + CC - 1) / CC; }
  __device__ void seek() {
    for (;;) {
      if (sweep == 0) {
        if (b >= nb) { sweep = 1; b = nb - 1; continue; }
        const int n = nch(b);
        if (n > r) { k = r + ((n - 1 - r) / C) * C; return; }
        ++b;
      } else {
        if (b < 0) return;
        if (nch(b) > r) { k = r; return; }
        --b;
      }
    }
  }
  __device__ void start(const int32_t* tf_, int nb_, int r_, int C_, int CC_) {
    tf = tf_; nb = nb_; r = r_; C = C_; CC = CC_; sweep = 0; b = 0; k = 0;
    seek();
  }
  __device__ bool done() const { return sweep == 1 && b < 0; }
  __device__ void next() {
    if (sweep == 0) {
      if (k - C >= r) { k -= C; return; }
      ++b;
    } else {
      if (k + C < nch(b)) { k += C; return; }
      --b;
    }
    seek();
  }
};

// Shared-memory layout: ring | red (NT) | tv (32) | xv (32) | stage barriers (S) |
// message barriers pf, df, vf, xf (D each) | abort flag | pbuf, dbuf (D C 32 each) |
// xbuf (D 32) | v (nb 32, 16-byte aligned) | poff (nb) | tf (nb).
template <int C>
__host__ __device__ constexpr size_t split_v_offset() {
  return ((size_t)kSplitStages * kSplitStage + (kSplitThreads + 64) * 4 + (kSplitStages + 4 * kSplitRing) * 8 + 16 +
          (2 * kSplitRing * C * 32 + kSplitRing * 32) * 4 + 15) /
         16 * 16;
}

template <int C>
__global__ void __launch_bounds__(kSplitThreads, 1) k_local_split(LocalArgs a) {
  constexpr int NT = kSplitThreads, NW = NT / 32, S = kSplitStages, D = kSplitRing;
  constexpr int CC = kSplitStage / (kT * 4);  // columns per stage
  constexpr int CHUNK = CC * kT;              // floats per stage
  constexpr int T = CC / kT;                  // tiles per chunk
  constexpr int CPW = CC / NW;                // forward: contiguous columns per warp
  static_assert(D > (C - 1) * T, "the message ring must exceed the largest lag between the CTAs");
  static_assert(CPW % 4 == 0 && CC <= NT, "stage geometry");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* ring = reinterpret_cast<float*>(smem_raw);
  float* red = reinterpret_cast<float*>(smem_raw + (size_t)S * kSplitStage);
  float* tv = red + NT;
  float* xv = tv + 32;
  uint64_t* bars = reinterpret_cast<uint64_t*>(xv + 32);
  uint64_t* pf = bars + S;  // CTA 0: partial sums of row b from every peer
  uint64_t* df = pf + D;    // CTA 0: updates of block j from every peer
  uint64_t* vf = df + D;    // CTA r > 0: v_b from CTA 0
  uint64_t* xf = vf + D;    // CTA r > 0: x_b from CTA 0
  int* abort_flag = reinterpret_cast<int*>(xf + D);
  float* pbuf = reinterpret_cast<float*>(abort_flag + 4);
  float* dbuf = pbuf + D * C * 32;
  float* xbuf = dbuf + D * C * 32;
  float* v = reinterpret_cast<float*>(smem_raw + split_v_offset<C>());

  const int rank = cluster_rank();
  const int i = blockIdx.x / C;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t o0 = a.om_off[i];
  const int ni = (int)(a.om_off[i + 1] - o0);
  const int64_t b0 = a.blk_off[i];
  const int nb = (int)(a.blk_off[i + 1] - b0);
  const float* fac = reinterpret_cast<const float*>(a.fac);
  if (nb == 0) return;  // the whole cluster (same subdomain) leaves; the host rejects empty subdomains
  int64_t* poff = reinterpret_cast<int64_t*>(v + (size_t)nb * kT);
  int32_t* tf = reinterpret_cast<int32_t*>(poff + nb);
  for (int k = tid; k < nb; k += NT) {
    poff[k] = a.blk_poff[b0 + k];
    tf[k] = a.blk_tf[b0 + k];
  }
  if (tid == 0) {
    for (int s = 0; s < S; ++s) bar_init(&bars[s], 1);
    for (int d = 0; d < D; ++d) {
      bar_init(&pf[d], 32 * (C - 1));
      bar_init(&df[d], 32 * (C - 1));
      bar_init(&vf[d], 32);
      bar_init(&xf[d], 32);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  cluster_sync();  // every CTA's barriers are initialised before any peer arrives on them

  auto nch = [&](int bb) { return ((bb - tf[bb] + 1) * kT + CC - 1) / CC; };
  OwnIter prod{};
  int issued = 0;
  const bool issuer = tid == NT - 32;
  auto issue = [&](int stage) {
    const int wd = (prod.b - tf[prod.b] + 1) * kT;
    const int hi = wd - prod.k * CC;
    const int lo = max(0, hi - CC);
    const uint32_t bytes = (uint32_t)((hi - lo) * kT * 4);
    if (!in_range(poff[prod.b] + (int64_t)hi * kT - 1, a.fac_elems, a.err) || !in_range(poff[prod.b], a.fac_elems, a.err)) {
      *abort_flag = 1;
    } else {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      expect_tx(&bars[stage], bytes);
      copy_g2s(ring + stage * CHUNK, fac + poff[prod.b] + (int64_t)lo * kT, bytes, &bars[stage]);
    }
    prod.next();
    ++issued;
  };
  if (issuer && !a.stall) {
    prod.start(tf, nb, rank, C, CC);
    for (int s = 0; s < S - 1 && !prod.done(); ++s) issue(s);
  }
  if (rank == 0) {
    // gather r(Omega_i), scaled by the equilibration, and the coarse restriction
    for (int k = tid; k < nb * kT; k += NT)
      v[k] = (k < ni && in_range(a.om_glob[o0 + k], a.n_cols, a.err)) ? (float)(a.r[a.om_glob[o0 + k]] * a.eqs[o0 + k])
                                                                       : 0.f;
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
  }
  __syncthreads();

  const int rot = tid & (kT / 4 - 1);  // skew of the backward column reads (16-byte groups)
  float xr[kT];
  int q = 0;  // owned chunks consumed
  for (int sweep = 0; sweep < 2 && !*abort_flag; ++sweep) {
    if (sweep == 1 && rank > 0) {
      // v becomes the sum of this CTA's backward updates; blocks it never updates
      // (j + rank T beyond the last row) are sent as zeros now
      for (int k = tid; k < nb * kT; k += NT) v[k] = 0.f;
      __syncthreads();
      if (w == 0)
        for (int j = nb - 1; j >= 0 && j + rank * T > nb - 1; --j) {
          const int o = nb - 1 - j;
          st_peer(peer_addr(&dbuf[((o % D) * C + rank) * 32 + lane], 0), 0.f);
          arrive_peer(peer_addr(&df[o % D], 0));
        }
    }
    for (int bi = 0; bi < nb; ++bi) {
      const int b = sweep == 0 ? bi : nb - 1 - bi;
      const int t0 = tf[b];
      const int wd = (b - t0 + 1) * kT;
      const int offw = wd - kT;
      const int n = nch(b);
      const bool has = n > rank;
      float acc = 0.f;
      // before the row: the values this CTA reads (v up to block b - rank T in the
      // forward sweep, x_b in the backward sweep); waiting at every row also keeps the
      // senders within the message ring
      // Every thread polls the message barrier itself (its own acquire), so no CTA
      // barrier follows; a wait that gives up is acted on at the next uniform check.
      if (rank > 0) {
        const int j = sweep == 0 ? b - rank * T : nb - 1 - b;  // message place in the sweep
        if (j >= 0)
          bounded_wait<true>(sweep == 0 ? &vf[j % D] : &xf[j % D], (uint32_t)((j / D) & 1), abort_flag);
        if (sweep == 1 && has) {
          const float* xb = xbuf + (j % D) * 32;
#pragma unroll
          for (int g = 0; g < kT / 4; ++g) {
            const float4 t4 = *reinterpret_cast<const float4*>(xb + ((g + rot) & (kT / 4 - 1)) * 4);
            xr[4 * g] = t4.x; xr[4 * g + 1] = t4.y; xr[4 * g + 2] = t4.z; xr[4 * g + 3] = t4.w;
          }
        }
      }
      if (has) {
        int k = sweep == 0 ? rank + ((n - 1 - rank) / C) * C : rank;
        for (;;) {
          const int stage = q % S;
          if (issuer && !a.stall && !prod.done()) issue((q + S - 1) % S);
          bounded_wait<false>(&bars[stage], (uint32_t)((q / S) & 1), abort_flag);
          const float* ch = ring + stage * CHUNK;
          const int hi = wd - k * CC;
          const int lo = max(0, hi - CC);
          const int phi = min(hi, offw);  // panel columns of this chunk: [lo, phi)
          float* vw = v + t0 * kT;
          if (sweep == 0) {
            const int c0 = lo + w * CPW;
            if (c0 < phi) {
              const float* colp = ch + (c0 - lo) * kT + lane;
              float s0 = 0.f, s1 = 0.f;
              if (c0 + CPW <= phi) {
#pragma unroll
                for (int jj = 0; jj < CPW; jj += 4) {
                  const float4 v4 = *reinterpret_cast<const float4*>(vw + c0 + jj);
                  s0 += colp[(jj + 0) * kT] * v4.x;
                  s1 += colp[(jj + 1) * kT] * v4.y;
                  s0 += colp[(jj + 2) * kT] * v4.z;
                  s1 += colp[(jj + 3) * kT] * v4.w;
                }
              } else {
                for (int c = c0; c < phi; ++c) s0 += colp[(c - c0) * kT] * vw[c];
              }
              acc += s0 + s1;
            }
            if (k == 0) {  // (rank 0 only) the diagonal step of row b
              red[w * 32 + lane] = acc;
              __syncthreads();
              if (w == 0) {
                float s = 0.f;
#pragma unroll
                for (int u = 0; u < NW; ++u) s += red[u * 32 + lane];
                if (C > 1) {
                  bounded_wait<true>(&pf[b % D], (uint32_t)((b / D) & 1), abort_flag);
                  for (int r = 1; r < C; ++r) s += pbuf[((b % D) * C + r) * 32 + lane];
                }
                tv[lane] = v[b * kT + lane] - s;
                __syncwarp();
                const float* Dt = ch + (offw - lo) * kT;  // inverse diagonal tile, column-major
                float x0 = 0.f, x1 = 0.f;
#pragma unroll 8
                for (int c = 0; c < kT; c += 2) {
                  x0 += Dt[c * kT + lane] * tv[c];
                  x1 += Dt[(c + 1) * kT + lane] * tv[c + 1];
                }
                const float x = x0 + x1;
                v[b * kT + lane] = x;
                for (int r = 1; r < C; ++r)
                  if (b <= nb - 1 - r * T) {
                    st_peer(peer_addr(&v[b * kT + lane], r), x);
                    arrive_peer(peer_addr(&vf[b % D], r));
                  }
              }
            }
          } else {
            if (k == 0) {  // (rank 0 only) x_b from the final v_b
              if (w == 0) {
                float y = v[b * kT + lane];
                const int o = nb - 1 - b;  // place of block b's messages in the backward sweep
                if (C > 1) {
                  bounded_wait<true>(&df[o % D], (uint32_t)((o / D) & 1), abort_flag);
                  for (int r = 1; r < C; ++r) y += dbuf[((o % D) * C + r) * 32 + lane];
                }
                tv[lane] = y;
                __syncwarp();
                const float* Dt = ch + (offw - lo) * kT;
                float x0 = 0.f, x1 = 0.f;
#pragma unroll 8
                for (int u = 0; u < kT; u += 2) {
                  const int r0 = (u + lane) & 31, r1 = (u + 1 + lane) & 31;  // skewed walk: no bank conflicts
                  x0 += Dt[lane * kT + r0] * tv[r0];
                  x1 += Dt[lane * kT + r1] * tv[r1];
                }
                const float x = x0 + x1;
                xv[lane] = x;
                v[b * kT + lane] = x;
                for (int r = 1; r < C; ++r) {
                  st_peer(peer_addr(&xbuf[(o % D) * 32 + lane], r), x);
                  arrive_peer(peer_addr(&xf[o % D], r));
                }
              }
              __syncthreads();
#pragma unroll
              for (int g = 0; g < kT / 4; ++g) {
                const float4 t4 = *reinterpret_cast<const float4*>(xv + ((g + rot) & (kT / 4 - 1)) * 4);
                xr[4 * g] = t4.x; xr[4 * g + 1] = t4.y; xr[4 * g + 2] = t4.z; xr[4 * g + 3] = t4.w;
              }
            }
            // v_window -= L_off^T x_b: one thread per column, 16-byte reads in a rotated order
            const int c = lo + tid;
            if (tid < CC && c < phi) {
              const float4* c4 = reinterpret_cast<const float4*>(ch + (c - lo) * kT);
              float s = 0.f;
#pragma unroll
              for (int kk = 0; kk < 8; ++kk) {
                const float4 u = c4[(kk + rot) & 7];
                s += u.x * xr[4 * kk] + u.y * xr[4 * kk + 1] + u.z * xr[4 * kk + 2] + u.w * xr[4 * kk + 3];
              }
              vw[c] -= s;
            }
          }
          __syncthreads();
          if (*abort_flag) break;
          ++q;
          if (sweep == 0) {
            if (k - C < rank) break;
            k -= C;
          } else {
            if (k + C >= n) break;
            k += C;
          }
        }
        if (*abort_flag) break;
      }
      // after the row: peers send their forward partial of row b, or their summed
      // updates of block b - rank T (final for this CTA after row b)
      if (rank > 0) {
        if (sweep == 0) {
          if (has) {
            red[w * 32 + lane] = acc;
            __syncthreads();
          }
          if (w == 0) {
            float s = 0.f;
            if (has) {
#pragma unroll
              for (int u = 0; u < NW; ++u) s += red[u * 32 + lane];
            }
            st_peer(peer_addr(&pbuf[((b % D) * C + rank) * 32 + lane], 0), s);
            arrive_peer(peer_addr(&pf[b % D], 0));
          }
        } else {
          const int j = b - rank * T;
          if (j >= 0 && w == 0) {
            const int o = nb - 1 - j;
            st_peer(peer_addr(&dbuf[((o % D) * C + rank) * 32 + lane], 0), v[j * kT + lane]);
            arrive_peer(peer_addr(&df[o % D], 0));
          }
        }
        // (no barrier here: red is written again only after a later chunk's barrier, which
        // warp 0 reaches after reading it, and this CTA never updates block b - rank T
        // again after row b)
      }
    }
    __syncthreads();  // a uniform view of the abort flag before the next sweep or the exit
  }
  if (*abort_flag) {
    if (issuer) {
      if (a.err[0] == 0.0) a.err[0] = kErrTimeout;
      // bounded drain of the copies still in flight before the CTA's shared memory is released
      for (int qq = q; qq < issued; ++qq) {
        const long long t0 = clock64();
        while (!try_stage(&bars[qq % S], (uint32_t)((qq / S) & 1)))
          if (clock64() - t0 > kSplitWait) break;
      }
    }
  }
  __syncthreads();
  cluster_sync();  // no CTA leaves while a peer may still write into its shared memory
  if (rank == 0 && !*abort_flag)
    for (int k = tid; k < ni; k += NT) a.y[o0 + k] = (double)v[k] * a.eqs[o0 + k];
}

template <int C>
size_t split_smem(int max_nb) {
  return split_v_offset<C>() + (size_t)max_nb * (kT * 4 + sizeof(int64_t) + sizeof(int32_t));
}

}  // namespace

size_t local_split_smem(int max_nb) { return split_smem<2>(max_nb); }

int local_split_cluster() { return 2; }

bool local_split_launch(int N, int max_nb, const LocalArgs& a, cudaStream_t st) {
  static size_t raised = 0;
  const size_t sm = split_smem<2>(max_nb);
  if (sm > raised) {
    if (cudaFuncSetAttribute(k_local_split<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
      return false;
    raised = sm;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)N * 2, 1, 1);
  cfg.blockDim = dim3(kSplitThreads, 1, 1);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_local_split<2>, a) == cudaSuccess;
}

}  // namespace lsq
