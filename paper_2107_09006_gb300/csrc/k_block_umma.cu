// Multi right-hand-side local solves on the 5th-generation tensor cores (tcgen05).
//
// y_i = C_ii^{-1} R_i r for R <= 32 right-hand sides and every subdomain, as in the
// block path's other local-solve kernels, but the triangular sweeps are right-looking
// so that each block step's update is one tall product the tensor cores can take:
//   forward,  for b = 0 .. nb-1:  Y_b = L_bb^{-1} V_b;   V_j -= L_jb Y_b   (j > b, L_jb stored)
//   backward, for b = nb-1 .. 0:  X_b = L_bb^{-T} V_b;   V_t -= L_bt^T X_b (tf_b <= t < b)
// The update of one step stacks its factor tiles (L_jb, or L_bt^T) into M = 128 row
// chunks (four 32 x 32 tiles) and runs D = A Y_b (N = 32 right-hand sides, K = 32) as
// tcgen05.mma kind::tf32 with the accumulator in tensor memory; the solution operand is
// split into a TF32 head and tail (two MMAs into the same accumulator), the factor is
// stored TF32-rounded.  The 32 x 32 diagonal products stay on the CUDA cores in FP32.
//
// Layout of an operand in shared memory: K-major core matrices of 8 rows x 16 bytes
// (no swizzle), the K-direction core matrices 128 bytes apart (leading byte offset) and
// the 8-row groups 1024 bytes apart (stride byte offset), so a 32 x 32 tile is 4 KB and
// four tiles one after another form an M = 128 operand.  The factor copies are stored
// in that layout so one bulk copy lands a whole chunk.
//
// Steps overlap: the MMA warp commits the products of a step's first chunk (the next
// block rows the diagonal products need) separately from the rest; the compute warps
// apply that chunk before the next diagonal product and the other chunks while the next
// step's products run (two halves of tensor memory, two operand buffers).  A step updates
// at most 32 tiles (8 chunks), i.e. factor block rows of at most 33 tiles.
//
// Roles (one CTA per SM, subdomains dealt round-robin over the CTAs in decreasing size):
// warps 0-7 gather the right-hand side, run the diagonal products and apply the
// accumulators to the window of pending tiles kept in shared memory; warp 8 issues the
// MMAs; warps 9 and 10 stream the factor chunks and the diagonal tiles by bulk
// asynchronous copies.
// They meet only on mbarriers; every wait is bounded and a give-up sets the error slot,
// after which every role drains what it has in flight and the CTA returns.
#include "common.cuh"
#include "kernels.h"

namespace lsq {

namespace {

constexpr int kTileBytes = 4096;         // one 32 x 32 FP32/TF32 tile in core-matrix layout
constexpr int kChunkTiles = 4;           // M = 128
constexpr int kChunkBytes = kTileBytes * kChunkTiles;
constexpr int kFSMax = 8;                // factor chunk stages (at most; the launch picks what fits)
constexpr int kDS = 3;                   // diagonal tile stages
constexpr int kDRow = 36;                 // floats per row of a diagonal tile (16-byte rows)
constexpr int kDiagFloats = 32 * kDRow;  // padded row-major L_bb^{-1} (forward) or L_bb^{-T} (backward)
constexpr int kVRow = 36;                // floats per row of a window tile (16-byte rows, no conflicts)
constexpr int kVTile = 32 * kVRow;
constexpr int kUThreads = 352;           // 8 compute warps, MMA warp, two copy warps
constexpr long long kUWait = 4000000000ll;  // about two seconds

__device__ __forceinline__ uint32_t s_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mb_init(uint64_t* b, uint32_t c) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(b)), "r"(c) : "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(b)) : "memory");
}
__device__ __forceinline__ void mb_expect(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mb_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(s_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   s_addr(dst)),
               "l"(src), "r"(bytes), "r"(s_addr(bar))
               : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void compute_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
// Barrier of the compute warps that also returns whether any of them passed pred != 0:
// the same answer in every compute thread, so they all leave their loops together.
__device__ __forceinline__ bool compute_sync_any(int pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 1, 256, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(pred)
      : "memory");
  return r != 0;
}

// Bounded wait: true on success; gives up (false) after about two seconds or as soon as
// another role has flagged an abort.
__device__ __forceinline__ bool mb_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
  if (mb_try(b, parity)) return true;
  const long long t0 = clock64();
  while (!mb_try(b, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > kUWait) return false;
  }
  return true;
}

// Shared-memory matrix descriptor of a K-major operand without swizzle: start address,
// leading byte offset 128 (next core matrix along K), stride byte offset 1024 (next
// 8-row group), descriptor version 1.
__device__ __forceinline__ uint64_t op_desc(uint32_t addr, uint32_t lbo = 128, uint32_t sbo = 1024) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         ((uint64_t)1 << 46);
}
// The solution operand uses K-direction core matrices 144 bytes apart (8-row groups
// 1152 bytes apart): element (n, k) then sits in bank ((n & 7) * 4 + k) mod 32, so the 32
// lanes of a warp, one row k each, store a column n without bank conflicts.
constexpr uint32_t kBLbo = 144, kBSbo = 8 * kBLbo;
__device__ __forceinline__ uint32_t b_offset(int n, int k) {
  return (uint32_t)((n >> 3) * kBSbo + (k >> 2) * kBLbo + (n & 7) * 16 + (k & 3) * 4);
}
// Instruction descriptors: D FP32, A and B TF32, both K-major, M = 128.  N = 64: the 64
// columns of B are the 32 right-hand sides' TF32 heads (0-31) and tails (32-63), so one
// MMA per K step gives both partial products, which the epilogue adds (steps of up to 4
// chunks).  N = 32 (wide steps, up to 8 chunks): the heads and the tails are two MMAs
// into the same 32 accumulator columns.
constexpr uint32_t kIdesc64 = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint32_t kIdesc32 = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_addr(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
}

// Rows of 32 accumulator columns at taddr and taddr + 32 (heads' and tails' partial
// products), added: both loads are in flight before the single wait.
__device__ __forceinline__ void tmem_ld_sum(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32], t[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(t[0]), "=r"(t[1]), "=r"(t[2]), "=r"(t[3]), "=r"(t[4]), "=r"(t[5]), "=r"(t[6]), "=r"(t[7]),
        "=r"(t[8]), "=r"(t[9]), "=r"(t[10]), "=r"(t[11]), "=r"(t[12]), "=r"(t[13]), "=r"(t[14]), "=r"(t[15]),
        "=r"(t[16]), "=r"(t[17]), "=r"(t[18]), "=r"(t[19]), "=r"(t[20]), "=r"(t[21]), "=r"(t[22]), "=r"(t[23]),
        "=r"(t[24]), "=r"(t[25]), "=r"(t[26]), "=r"(t[27]), "=r"(t[28]), "=r"(t[29]), "=r"(t[30]), "=r"(t[31])
      : "r"(taddr + 32));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]) + __uint_as_float(t[c]);
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t y;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
  return __uint_as_float(y);
}

// byte offset of element (row, k) in a K-major core-matrix operand of 32-wide K
__host__ __device__ __forceinline__ uint32_t cm_offset(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

struct USmem {
  unsigned char* fring;  // fs chunks of kChunkBytes
  float* bop;            // solution operand, two buffers: 64 x 32 (b_offset layout), heads then tails
  float* dring;          // kDS padded diagonal tiles
  float* win;            // ring of window tiles, kVTile floats each
  uint64_t* full;        // [fs]
  uint64_t* empty;       // [fs]
  uint64_t* dfull;       // [kDS]
  uint64_t* dempty;      // [kDS]
  uint64_t* bready;
  uint64_t* d0ready;     // chunk 0 of a step's products done
  uint64_t* drest;       // [2] all of a step's products done, one barrier per tensor-memory half
                         // (its waits come a step late, so one barrier could complete twice
                         // before the wait and the parity would then name the wrong phase)
  uint64_t* fin;
  uint32_t* tslot;
  int* abort_flag;
};

__host__ __device__ inline size_t umma_smem_bytes(int ring, int fs) {
  return 1024 + (size_t)fs * kChunkBytes + 2 * 8 * kBSbo + (size_t)kDS * kDiagFloats * 4 +
         (size_t)ring * kVTile * 4 + (2 * kFSMax + 2 * kDS + 5) * 8 + 16;
}

__device__ inline USmem carve(unsigned char* base, int ring, int fs) {
  USmem s;
  unsigned char* p = reinterpret_cast<unsigned char*>(((uintptr_t)base + 1023) & ~(uintptr_t)1023);
  s.fring = p; p += (size_t)fs * kChunkBytes;
  s.bop = reinterpret_cast<float*>(p); p += 2 * 8 * kBSbo;
  s.dring = reinterpret_cast<float*>(p); p += (size_t)kDS * kDiagFloats * 4;
  s.win = reinterpret_cast<float*>(p); p += (size_t)ring * kVTile * 4;
  uint64_t* bars = reinterpret_cast<uint64_t*>(p);
  s.full = bars; s.empty = bars + kFSMax; s.dfull = bars + 2 * kFSMax; s.dempty = bars + 2 * kFSMax + kDS;
  s.bready = bars + 2 * kFSMax + 2 * kDS; s.d0ready = s.bready + 1; s.drest = s.bready + 2; s.fin = s.bready + 4;
  s.tslot = reinterpret_cast<uint32_t*>(s.bready + 5);
  s.abort_flag = reinterpret_cast<int*>(s.tslot + 1);
  return s;
}

// Tiles of the update of step (sweep, global block row g): [off[g], off[g + 1]) in the
// sweep's copy; target local block row of tile e: row[e].
struct StepTiles {
  const int64_t* off;
  const int32_t* row;
};

__global__ void __launch_bounds__(kUThreads, 1) k_b_local_umma(BUmmaArgs a) {
  extern __shared__ unsigned char smem_raw[];
  const int FS = a.fs;
  const USmem s = carve(smem_raw, a.ring, FS);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  volatile int* abort_flag = s.abort_flag;
  if (tid == 0) {
    for (int k = 0; k < FS; ++k) { mb_init(&s.full[k], 1); mb_init(&s.empty[k], 1); }
    for (int k = 0; k < kDS; ++k) { mb_init(&s.dfull[k], 1); mb_init(&s.dempty[k], 1); }
    mb_init(s.bready, 1);
    mb_init(s.d0ready, 1);
    mb_init(&s.drest[0], 1);
    mb_init(&s.drest[1], 1);
    mb_init(s.fin, 1);
    *s.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(s.tslot)),
                 "r"((uint32_t)a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *s.tslot;
  const StepTiles fw{a.f_off, a.f_row}, bw{a.b_off, a.b_row};
  const int RING = a.ring, R = a.R;

  if (w >= 9) {
    // ---------------- copy warps: warp 9 streams the factor chunks, warp 10 the diagonal
    // tiles (one thread each, separate warps so that neither waits behind the other), in
    // consumption order and as far ahead as its ring allows
    if (lane == 0 && !a.stall) {
      const bool diag = w == 10;
      const int NSTG = diag ? kDS : FS;
      uint64_t* fullb = diag ? s.dfull : s.full;
      uint64_t* emptyb = diag ? s.dempty : s.empty;
      uint32_t q = 0;  // copies issued so far
      bool ok = true;
      for (int k = blockIdx.x; k < a.N && ok; k += gridDim.x) {
        const int i = a.order[k];
        const int64_t b0 = a.blk_off[i];
        const int nb = (int)(a.blk_off[i + 1] - b0);
        for (int sw = 0; sw < 2 && ok; ++sw) {
          const StepTiles& T = sw == 0 ? fw : bw;
          const float* src = sw == 0 ? a.ffac : a.bfac;
          for (int st = 0; st < nb && ok; ++st) {
            const int64_t g = b0 + (sw == 0 ? st : nb - 1 - st);
            if (diag) {
              const int ds = (int)(q % kDS);
              if (!mb_wait(&emptyb[ds], ((q / kDS) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
              mb_expect(&fullb[ds], kDiagFloats * 4);
              bulk_copy(s.dring + (size_t)ds * kDiagFloats, a.dinv + (2 * g + sw) * kDiagFloats, kDiagFloats * 4,
                        &fullb[ds]);
              ++q;
              continue;
            }
            const int64_t e0 = T.off[g], e1 = T.off[g + 1];
            const int64_t ntl = sw == 0 ? a.f_tiles : a.b_tiles;
            if (e1 > e0 && (!in_range(e0, ntl, a.err) || !in_range(e1 - 1, ntl, a.err))) {
              ok = false;  // (bounds-checked build: a tile range outside the copy is not read)
              break;
            }
            for (int64_t e = e0; e < e1 && ok; e += kChunkTiles) {
              const int fs = (int)(q % FS);
              if (!mb_wait(&emptyb[fs], ((q / FS) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
              const int nt = (int)(e1 - e < kChunkTiles ? e1 - e : kChunkTiles);
              mb_expect(&fullb[fs], (uint32_t)nt * kTileBytes);
              bulk_copy(s.fring + (size_t)fs * kChunkBytes, src + e * 1024, (uint32_t)nt * kTileBytes, &fullb[fs]);
              ++q;
            }
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        if (a.err[0] == 0.0) a.err[0] = kErrTimeout;
      }
      // drain: every issued copy has landed before the CTA's shared memory goes away (a
      // landed copy's phase stays complete until its stage is refilled, which no longer
      // happens)
      for (uint32_t qq = q > (uint32_t)NSTG ? q - NSTG : 0; qq < q; ++qq) {
        const long long t0 = clock64();
        while (!mb_try(&fullb[qq % NSTG], (qq / NSTG) & 1u))
          if (clock64() - t0 > kUWait) break;
      }
    }
  } else if (w == 8) {
    // ---------------- MMA warp: one thread issues every step's update products
    if (lane == 0) {
      uint32_t fq = 0, sq = 0;  // chunks consumed, update steps run
      bool ok = true;
      // descriptors: the operand buffers' four K steps, and the first factor stage (a stage
      // and K step offset is added to the start-address field, which it cannot overflow)
      uint64_t bdesc[2][4];
#pragma unroll
      for (int bf = 0; bf < 2; ++bf)
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
          bdesc[bf][ks] = op_desc(s_addr(s.bop) + bf * 8 * kBSbo + ks * 2 * kBLbo, kBLbo, kBSbo);
      const uint64_t adesc0 = op_desc(s_addr(s.fring));
      for (int k = blockIdx.x; k < a.N && ok; k += gridDim.x) {
        const int i = a.order[k];
        const int64_t b0 = a.blk_off[i];
        const int nb = (int)(a.blk_off[i + 1] - b0);
        for (int sw = 0; sw < 2 && ok; ++sw) {
          const StepTiles& T = sw == 0 ? fw : bw;
          for (int st = 0; st < nb && ok; ++st) {
            const int64_t g = b0 + (sw == 0 ? st : nb - 1 - st);
            const int64_t e0 = T.off[g], e1 = T.off[g + 1];
            if (e1 == e0) continue;
            if (!mb_wait(s.bready, sq & 1u, abort_flag)) { ok = false; break; }
            tc_after();
            // step sq's accumulators: half (sq & 1) of tensor memory, ncol columns per chunk
            const uint32_t tb = tmem + (uint32_t)(256 * (sq & 1u));
            const uint64_t* bd = bdesc[sq & 1u];
            int c = 0;
            for (int64_t e = e0; e < e1; e += kChunkTiles, ++c) {
              const int fs = (int)(fq % FS);
              if (!mb_wait(&s.full[fs], (fq / FS) & 1u, abort_flag)) { ok = false; break; }
              tc_after();
              const uint64_t ad = adesc0 + (uint64_t)((fs * kChunkBytes) >> 4);
              const uint32_t dt = tb + (uint32_t)(a.ncol * c);
              if (a.ncol == 64) {
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)
                  mma_tf32(dt, ad + (uint64_t)(ks * 16), bd[ks], kIdesc64, ks > 0 ? 1u : 0u);
              } else {
                // the tails' rows of B start 4 groups of 8 rows further
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                  mma_tf32(dt, ad + (uint64_t)(ks * 16), bd[ks], kIdesc32, ks > 0 ? 1u : 0u);
                  mma_tf32(dt, ad + (uint64_t)(ks * 16), bd[ks] + (uint64_t)((4 * kBSbo) >> 4), kIdesc32, 1u);
                }
              }
              mma_commit(&s.empty[fs]);  // the stage is free once these products are done
              if (c == 0) mma_commit(s.d0ready);  // the next step may apply chunk 0
              ++fq;
            }
            if (!ok) break;
            mma_commit(&s.drest[sq & 1u]);
            ++sq;
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        if (a.err[0] == 0.0) a.err[0] = kErrTimeout;
      }
      // every product issued has finished before tensor memory is released
      mma_commit(s.fin);
      const long long t0 = clock64();
      while (!mb_try(s.fin, 0))
        if (clock64() - t0 > kUWait) break;
    }
  } else {
    // ---------------- compute warps (256 threads)
    // Everything a step reads from global memory is fetched one step ahead, so that the
    // chain of block steps never waits on a global load: the step's tile range, the rows
    // its tiles update, the gathered right-hand side (indices two steps ahead, values one
    // step ahead), the forward results re-entering the backward window and the
    // equilibration scales of the outputs.
    // diagonal product: row dr (one per lane), right-hand sides dn .. dn+3 (per warp)
    const int dr = tid & 31, dn = (tid >> 5) * 4;
    uint32_t dq = 0, sq = 0;
    bool ok = true;
    float* spill = a.spill;
    for (int k = blockIdx.x; k < a.N && ok; k += gridDim.x) {
      const int i = a.order[k];
      const int64_t o0 = a.om_off[i];
      const int ni = (int)(a.om_off[i + 1] - o0);
      const int64_t b0 = a.blk_off[i];
      const int nb = (int)(a.blk_off[i + 1] - b0);
      // this thread's 4 entries (row e >> 5, right-hand side e & 31, e = tid + 256 u) of a
      // local block row j of the gathered right-hand side (zero past n_i and R): first
      // the gather indices and scales, then the values
      // (the loaded words are kept as they are until used, so the loads stay in flight)
      struct RhsIdx { int32_t gi[4]; double sc[4]; };
      auto fetch_idx = [&](int j, RhsIdx& x) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = tid + 256 * u, r = e >> 5, n = e & 31, l = j * 32 + r;
          x.gi[u] = -1;
          x.sc[u] = 0.0;
          if (j < nb && l < ni && n < R && in_range(a.om_glob[o0 + l], a.n_cols, a.err)) {
            x.gi[u] = a.om_glob[o0 + l];
            x.sc[u] = a.eqs[o0 + l];
          }
        }
      };
      auto fetch_val = [&](const RhsIdx& x, double (&f)[4]) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          f[u] = 0.0;
          if (x.gi[u] >= 0) f[u] = a.Rv[(int64_t)x.gi[u] * R + ((tid + 256 * u) & 31)];
        }
      };
      auto store_rhs = [&](int j, const RhsIdx& x, const double (&f)[4]) {
        float* V = s.win + (size_t)(j % RING) * kVTile;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = tid + 256 * u;
          V[(e >> 5) * kVRow + (e & 31)] = (float)(f[u] * x.sc[u]);
        }
      };
      RhsIdx ia, ib;  // indices of rows RING (values in flight) and RING + 1
      double pre[4];
      for (int j = 0; j < RING && j < nb; ++j) {
        fetch_idx(j, ia);
        fetch_val(ia, pre);
        store_rhs(j, ia, pre);
      }
      fetch_idx(RING, ia);
      fetch_val(ia, pre);
      fetch_idx(RING + 1, ib);
      compute_sync();
      for (int sw = 0; sw < 2 && ok; ++sw) {
        const StepTiles& T = sw == 0 ? fw : bw;
        float4 sp = make_float4(0.f, 0.f, 0.f, 0.f);  // backward: prefetched spill tile
        bool sp_valid = false;
        int64_t ne0 = T.off[b0 + (sw == 0 ? 0 : nb - 1)], ne1 = T.off[b0 + (sw == 0 ? 0 : nb - 1) + 1];
        double osc = 0.0;  // backward: equilibration scale of this thread's output row
        auto fetch_osc = [&](int bb) {
          const int l = bb * 32 + dr;
          osc = 0.0;
          if (l < ni) osc = a.eqs[o0 + l];
        };
        if (sw == 1) fetch_osc(nb - 1);
        // The previous step's products (if it had any): chunk 0 holds the rows the next
        // diagonal products need and is applied first (warps 0-3, tile w); chunks 1-3 are
        // applied after this step's diagonal product, while this step's products run
        // (chunk c by warp 4 ((c - 1) & 1) + tile).  Rows of those tiles: fetched a step
        // ahead.
        bool pv = false;
        uint32_t psq = 0;
        int64_t pe0 = 0, pe1 = 0;
        // chunk-0 tile w; this warp's deferred tiles: tile (w & 3) of chunks 1 + (w >> 2) + 2k
        int prow0 = 0, prow[4] = {0, 0, 0, 0};
        const int q4 = w & 3, cd0 = 1 + (w >> 2);
        const int ncol = a.ncol;
        auto apply = [&](uint32_t col, int64_t e, int64_t e_end, int row) {
          // (warp-uniform: tcgen05.ld runs on all lanes of a warp or none)
          if (e >= e_end) return;
          float d[32];
          if (ncol == 64) tmem_ld_sum(col + ((uint32_t)(32 * q4) << 16), d);
          else tmem_ld32(col + ((uint32_t)(32 * q4) << 16), d);
          float* Vj = s.win + (size_t)(row % RING) * kVTile + lane * kVRow;
#pragma unroll
          for (int n4 = 0; n4 < 8; ++n4) {
            float4 v = *reinterpret_cast<float4*>(Vj + 4 * n4);
            v.x -= d[4 * n4]; v.y -= d[4 * n4 + 1]; v.z -= d[4 * n4 + 2]; v.w -= d[4 * n4 + 3];
            *reinterpret_cast<float4*>(Vj + 4 * n4) = v;
          }
        };
        for (int st = 0; st < nb; ++st) {
          const int b = sw == 0 ? st : nb - 1 - st;
          const int64_t g = b0 + b;
          const int64_t e0 = ne0, e1 = ne1;
          if (st + 1 < nb) {
            const int64_t gn = b0 + (sw == 0 ? b + 1 : b - 1);
            ne0 = T.off[gn];
            ne1 = T.off[gn + 1];
          }
          if (sw == 1) {
            // tile b - RING + 1 enters the backward window (into the slot row b + 1 has
            // left; fetched from the forward spill one step ahead)
            const int t = b - RING + 1;
            if (sp_valid) *reinterpret_cast<float4*>(s.win + (size_t)(t % RING) * kVTile + (tid >> 3) * kVRow +
                                                     4 * (tid & 7)) = sp;
            // the tile that enters at the next step, b - RING (rows >= nb - RING stayed
            // resident from the forward sweep and are never fetched)
            sp_valid = b - RING >= 0;
            if (sp_valid) sp = reinterpret_cast<const float4*>(spill + (b0 + b - RING) * 1024)[tid];
          }
          // (the abort flag is read by lane 0 and shared, so that a warp takes a tcgen05.ld
          // with all of its lanes or none)
          if (pv) {  // chunk 0 of the previous step's products
            if (!mb_wait(s.d0ready, psq & 1u, abort_flag)) *abort_flag = 1;
            tc_after();
            const bool go = __shfl_sync(0xffffffffu, *abort_flag == 0 ? 1 : 0, 0);
            if (w < 4 && go) apply(tmem + 256 * (psq & 1u), pe0 + q4, pe1, prow0);
            tc_before();
          }
          compute_sync();  // V_b is complete
          // diagonal product on the CUDA cores (FP32): lane = output row, warp = group of
          // four right-hand sides (the window rows are read as broadcasts)
          const int ds = (int)(dq % kDS);
          if (!mb_wait(&s.dfull[ds], (dq / kDS) & 1u, abort_flag)) *abort_flag = 1;
          const float* D = s.dring + (size_t)ds * kDiagFloats;
          const float* V = s.win + (size_t)(b % RING) * kVTile;
          float4 y0 = make_float4(0.f, 0.f, 0.f, 0.f), y1 = y0;
          if (!*abort_flag) {
            const float4* Dr = reinterpret_cast<const float4*>(D + dr * kDRow);
#pragma unroll
            for (int c4 = 0; c4 < 8; ++c4) {
              const float4 d = Dr[c4];
              const float4 v0 = *reinterpret_cast<const float4*>(V + (4 * c4) * kVRow + dn);
              const float4 v1 = *reinterpret_cast<const float4*>(V + (4 * c4 + 1) * kVRow + dn);
              const float4 v2 = *reinterpret_cast<const float4*>(V + (4 * c4 + 2) * kVRow + dn);
              const float4 v3 = *reinterpret_cast<const float4*>(V + (4 * c4 + 3) * kVRow + dn);
              y0.x += d.x * v0.x; y0.y += d.x * v0.y; y0.z += d.x * v0.z; y0.w += d.x * v0.w;
              y1.x += d.y * v1.x; y1.y += d.y * v1.y; y1.z += d.y * v1.z; y1.w += d.y * v1.w;
              y0.x += d.z * v2.x; y0.y += d.z * v2.y; y0.z += d.z * v2.z; y0.w += d.z * v2.w;
              y1.x += d.w * v3.x; y1.y += d.w * v3.y; y1.z += d.w * v3.z; y1.w += d.w * v3.w;
            }
          }
          const float y[4] = {y0.x + y1.x, y0.y + y1.y, y0.z + y1.z, y0.w + y1.w};
          if (e1 > e0) {
            // the solution operand of this step, head and tail (K-major: k = row dr), into
            // buffer (sq & 1); its last reader, the products of step sq - 2, is done
            float* bo = s.bop + (size_t)(sq & 1u) * (8 * kBSbo / 4);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float hi = tf32_round(y[q]);
              bo[b_offset(dn + q, dr) >> 2] = hi;
              bo[b_offset(32 + dn + q, dr) >> 2] = tf32_round(y[q] - hi);
            }
            fence_async_smem();
          }
          tc_before();
          compute_sync();  // V_b and the diagonal tile read, the operand written
          if (tid == 0) {
            mb_arrive(&s.dempty[ds]);
            if (e1 > e0) mb_arrive(s.bready);
          }
          ++dq;
          // rows of this step's tiles, for its products' application at the next step
          int nrow0 = 0, nrow[4] = {0, 0, 0, 0};
          if (e1 > e0) {
            if (w < 4 && e0 + q4 < e1) nrow0 = T.row[e0 + q4];
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) {
              const int64_t e = e0 + 4 * (cd0 + 2 * k2) + q4;
              if (e < e1) nrow[k2] = T.row[e];
            }
          }
          if (sw == 0) {
            if (b < nb - RING) {
              *reinterpret_cast<float4*>(spill + g * 1024 + dr * 32 + dn) = make_float4(y[0], y[1], y[2], y[3]);
              // the right-hand side of row b + RING takes the slot row b has left
              store_rhs(b + RING, ia, pre);
              ia = ib;
              fetch_val(ia, pre);
              fetch_idx(b + RING + 2, ib);
            } else {
              *reinterpret_cast<float4*>(s.win + (size_t)(b % RING) * kVTile + dr * kVRow + dn) =
                  make_float4(y[0], y[1], y[2], y[3]);
            }
          } else {
            const int l = b * 32 + dr;
            if (l < ni) {
#pragma unroll
              for (int q = 0; q < 4; ++q)
                if (dn + q < R) a.Y[(o0 + l) * R + dn + q] = (double)y[q] * osc;
            }
            if (b > 0) fetch_osc(b - 1);
          }
          if (pv) {  // the other chunks of the previous step's products
            if (!mb_wait(&s.drest[psq & 1u], (psq >> 1) & 1u, abort_flag)) *abort_flag = 1;
            tc_after();
            const uint32_t pt = tmem + 256 * (psq & 1u);
            if (__shfl_sync(0xffffffffu, *abort_flag == 0 ? 1 : 0, 0)) {
#pragma unroll
              for (int k2 = 0; k2 < 4; ++k2) {
                const int c = cd0 + 2 * k2;
                apply(pt + ncol * c, pe0 + 4 * c + q4, pe1, prow[k2]);
              }
            }
            tc_before();
          }
          pv = e1 > e0;
          if (pv) {
            psq = sq++;
            pe0 = e0;
            pe1 = e1;
            prow0 = nrow0;
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) prow[k2] = nrow[k2];
          }
          if (compute_sync_any(*abort_flag)) { ok = false; break; }
        }
        if (ok && pv) {
          // (the last step of a sweep has no products; kept for any factor where it does)
          if (!mb_wait(s.d0ready, psq & 1u, abort_flag) || !mb_wait(&s.drest[psq & 1u], (psq >> 1) & 1u, abort_flag))
            *abort_flag = 1;
          tc_after();
          const uint32_t pt = tmem + 256 * (psq & 1u);
          if (!__shfl_sync(0xffffffffu, *abort_flag != 0 ? 1 : 0, 0)) {
            if (w < 4) apply(pt, pe0 + q4, pe1, prow0);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) {
              const int c = cd0 + 2 * k2;
              apply(pt + ncol * c, pe0 + 4 * c + q4, pe1, prow[k2]);
            }
          }
          tc_before();
          if (compute_sync_any(*abort_flag)) ok = false;
        }
      }
    }
    if (!ok && tid == 0 && a.err[0] == 0.0) a.err[0] = kErrTimeout;
  }
  tc_before();
  __syncthreads();
  tc_after();
  if (w == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)a.tmem_cols)
                 : "memory");
}

// Setup: the forward copy (tile e = L_jb, rows of L along M, its columns along K), the
// backward copy (tile e = L_bt^T: columns of L along M, its rows along K), both TF32
// rounded in core-matrix layout, from the FP32 solve storage (column-major tiles).
__global__ void k_bu_copy(int64_t ntiles, const int64_t* __restrict__ src_off, const float* __restrict__ L32,
                          float* __restrict__ dst, int transpose) {
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const float* src = L32 + src_off[t];
    float* d = dst + t * 1024;
    for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
      const int c = e >> 5, r = e & 31;  // source element (r, c) at c * 32 + r
      const uint32_t o = transpose ? cm_offset(c, r) : cm_offset(r, c);
      d[o >> 2] = tf32_round(src[e]);
    }
  }
}

// Setup: the inverse diagonal tile of every block row, twice (L_bb^{-1} for the forward
// sweep, L_bb^{-T} for the backward sweep), row-major with rows of kDRow floats.
__global__ void k_bu_diag(int64_t nblocks, const int64_t* __restrict__ poff, const float* __restrict__ L32,
                          float* __restrict__ dst) {
  for (int64_t g = blockIdx.x; g < nblocks; g += gridDim.x) {
    const int64_t po = poff[g];
    const int width = (int)((poff[g + 1] - po) / 32);
    const float* D = L32 + po + (int64_t)(width - 32) * 32;  // column-major inverse tile
    for (int e = threadIdx.x; e < 32 * kDRow; e += blockDim.x) {
      const int r = e / kDRow, c = e % kDRow;
      dst[(2 * g) * kDiagFloats + e] = c < 32 ? D[c * 32 + r] : 0.f;
      dst[(2 * g + 1) * kDiagFloats + e] = c < 32 ? D[r * 32 + c] : 0.f;
    }
  }
}

}  // namespace

size_t block_local_umma_smem(int ring, int fs) { return umma_smem_bytes(ring, fs); }

int block_local_umma_stages(int ring, size_t smem_limit) {
  int fs = kFSMax;
  while (fs > 2 && umma_smem_bytes(ring, fs) > smem_limit) --fs;
  return fs;
}

int block_local_umma_tmem_cols(int max_step_tiles) {
  // two halves (consecutive steps' accumulators) of 4 chunks x 64 or 8 chunks x 32 columns
  return max_step_tiles <= 8 * kChunkTiles ? 512 : 0;
}

int block_local_umma_ncol(int max_step_tiles) { return max_step_tiles <= 4 * kChunkTiles ? 64 : 32; }

bool block_local_umma_prepare(size_t smem) {
  return cudaFuncSetAttribute(k_b_local_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess;
}

void launch_b_local_umma(const BUmmaArgs& a, int grid, cudaStream_t st) {
  k_b_local_umma<<<grid, kUThreads, umma_smem_bytes(a.ring, a.fs), st>>>(a);
}

void launch_bu_copy(int64_t ntiles, const int64_t* src_off, const float* L32, float* dst, int transpose,
                    cudaStream_t st) {
  if (ntiles <= 0) return;
  k_bu_copy<<<(unsigned)(ntiles > 65536 ? 65536 : ntiles), kThreads, 0, st>>>(ntiles, src_off, L32, dst, transpose);
}

void launch_bu_diag(int64_t nblocks, const int64_t* poff, const float* L32, float* dst, cudaStream_t st) {
  if (nblocks <= 0) return;
  k_bu_diag<<<(unsigned)(nblocks > 65536 ? 65536 : nblocks), kThreads, 0, st>>>(nblocks, poff, L32, dst);
}

}  // namespace lsq
