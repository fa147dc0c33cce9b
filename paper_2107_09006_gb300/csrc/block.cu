// Multi right-hand-side PCG on the normal equations: R <= 32 right-hand sides of every
// problem of the handle advance together, each (problem, right-hand side) pair with its
// own CG scalars (the same recurrences as the single-vector path: plain PCG for FP64
// local factors, the flexible form for FP32/BF16 factors), its own stopping test and
// its own true-residual check.  A pair that meets its test is frozen (alpha = 0) while
// the others continue; the iteration is one CUDA graph replayed until every pair has
// passed.  Every kernel serves all pairs: the factor tiles, A and the coarse basis are
// read once per iteration for all R right-hand sides.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "handle.h"

using namespace lsi;

namespace {

constexpr int kChunkCols = 256;

lsq::BChunks chunks(const ls_handle* h) {
  return lsq::BChunks{h->blk.nchunks, h->blk.chunk_start.p, h->blk.chunk_prob.p};
}

lsq::BScal scal(ls_handle* h) {
  const int64_t P = (int64_t)h->nprob * 32;
  double* s = h->blk.sc.p;
  return lsq::BScal{s, s + P, s + 2 * P, s + 3 * P, s + 4 * P, s + 5 * P, s + 6 * P, s + 7 * P,
                    h->blk.act.p, h->blk.its.p, h->blk.stat.p};
}

int arith_bytes(int prec) { return prec == LS_PREC_F64 ? 8 : 4; }
int fac_bytes(int prec) { return prec == LS_PREC_F64 ? 8 : prec == LS_PREC_F32 ? 4 : 2; }

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void ensure_buffers(ls_handle* h, int R) {
  BlockState& B = h->blk;
  if (B.R >= R) return;
  if (B.gexec) {
    cudaGraphExecDestroy(B.gexec);
    B.gexec = nullptr;
  }
  const size_t n = (size_t)h->n * R, m = (size_t)h->m * R;
  B.X.alloc(n); B.Rv.alloc(n); B.Rold.alloc(n); B.Z.alloc(n); B.P.alloc(n); B.W.alloc(n);
  B.Q.alloc(m); B.B.alloc(m); B.Bu.alloc(m);
  B.Y.alloc((size_t)h->total_local * R);
  B.R0.alloc(std::max<size_t>((size_t)h->n0 * R, 1));
  B.Y0.alloc(std::max<size_t>((size_t)h->n0 * R, 1));
  if (B.ZT.p) B.Y0f.alloc(std::max<size_t>((size_t)h->n0 * R, 1));
  B.R = R;
}

// The update tiles of every block step of the right-looking sweeps (tcgen05 kernel) and
// the copies they are read from, built from the solve storage at the first use.
void umma_prepare(ls_handle* h) {
  BlockState& B = h->blk;
  if (B.Uf.p) return;
  cudaStream_t st = h->st;
  const int64_t NB = h->total_blocks;
  std::vector<int64_t> boff((size_t)h->N + 1), poff((size_t)NB + 1);
  std::vector<int32_t> tf((size_t)NB);
  CK(cudaMemcpyAsync(boff.data(), h->blk_off.p, sizeof(int64_t) * boff.size(), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(poff.data(), h->blk_poff.p, sizeof(int64_t) * poff.size(), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(tf.data(), h->blk_tf.p, sizeof(int32_t) * tf.size(), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  std::vector<int64_t> foff((size_t)NB + 1, 0), boff2((size_t)NB + 1, 0), fsrc, bsrc;
  std::vector<int32_t> frow, brow;
  for (int i = 0; i < h->N; ++i) {
    const int64_t b0 = boff[i];
    const int nb = (int)(boff[i + 1] - b0);
    for (int b = 0; b < nb; ++b) {
      // forward step b: L_jb for the rows j > b whose envelope reaches column tile b
      foff[b0 + b] = (int64_t)frow.size();
      for (int j = b + 1; j < nb && j < b + h->wmax; ++j)
        if (tf[b0 + j] <= b) {
          fsrc.push_back(poff[b0 + j] + (int64_t)(b - tf[b0 + j]) * 1024);
          frow.push_back(j);
        }
      // backward step b: L_bt for the tile columns b > t >= tf_b of block row b
      boff2[b0 + b] = (int64_t)brow.size();
      for (int t = b - 1; t >= tf[b0 + b]; --t) {  // nearest row first: it is needed first
        bsrc.push_back(poff[b0 + b] + (int64_t)(t - tf[b0 + b]) * 1024);
        brow.push_back(t);
      }
    }
  }
  foff[NB] = (int64_t)frow.size();
  boff2[NB] = (int64_t)brow.size();
  B.uf_off.upload(foff, st);
  B.ub_off.upload(boff2, st);
  B.uf_row.upload(frow, st);
  B.ub_row.upload(brow, st);
  DevBuf<int64_t> fs, bs;
  fs.upload(fsrc, st);
  bs.upload(bsrc, st);
  B.Uf.alloc(std::max<size_t>(frow.size(), 1) * 1024);
  B.Ub.alloc(std::max<size_t>(brow.size(), 1) * 1024);
  B.Ud.alloc((size_t)NB * 2 * 32 * 36);
  lsq::launch_bu_copy((int64_t)frow.size(), fs.p, h->L32.p, B.Uf.p, 0, st);
  lsq::launch_bu_copy((int64_t)brow.size(), bs.p, h->L32.p, B.Ub.p, 1, st);
  lsq::launch_bu_diag(NB, h->blk_poff.p, h->L32.p, B.Ud.p, st);
  CK(cudaStreamSynchronize(st));
  check_launch("tcgen05 factor copies");
}

void swizzle_prepare(ls_handle* h) {
  BlockState& B = h->blk;
  if (B.Lsw.p) return;
  B.Lsw.alloc(h->fac_elems);
  lsq::launch_b_swizzle(h->fac_elems, h->L32.p, B.Lsw.p, h->st);
  CK(cudaStreamSynchronize(h->st));
  check_launch("swizzled factor copy");
}

void launch_local_kernel(ls_handle* h, int kernel, int R, const double* Rin) {
  BlockState& B = h->blk;
  cudaStream_t st = h->st;
  if (kernel == 2) {
    lsq::BUmmaArgs u{};
    u.N = h->N; u.order = B.order.p;
    u.om_off = h->om_off.p; u.om_glob = h->om_glob.p; u.eqs = h->eqs.p; u.blk_off = h->blk_off.p;
    u.ffac = B.Uf.p; u.f_off = B.uf_off.p; u.f_row = B.uf_row.p;
    u.bfac = B.Ub.p; u.b_off = B.ub_off.p; u.b_row = B.ub_row.p;
    u.dinv = B.Ud.p;
    u.Rv = Rin; u.Y = B.Y.p; u.R = R;
    u.spill = reinterpret_cast<float*>(B.Vg.p);
    u.ring = B.u_ring; u.tmem_cols = B.u_tmem; u.fs = B.u_fs;
    u.ncol = lsq::block_local_umma_ncol(std::max(h->wmax - 1, 1));
    u.err = h->scal.p + lsq::S_ERR;
    u.stall = h->opt.test_stall;
    u.n_cols = h->n; u.f_tiles = (int64_t)(B.Uf.n / 1024); u.b_tiles = (int64_t)(B.Ub.n / 1024);
    lsq::launch_b_local_umma(u, B.u_grid, st);
    return;
  }
  lsq::BLocalArgs a{};
  a.N = h->N; a.order = B.order.p; a.qctr = B.qctr.p;
  a.om_off = h->om_off.p; a.om_glob = h->om_glob.p; a.eqs = h->eqs.p;
  a.blk_off = h->blk_off.p; a.blk_tf = h->blk_tf.p; a.blk_poff = h->blk_poff.p;
  a.fac = h->prec == LS_PREC_F64 ? (const void*)h->L64.p
        : h->prec == LS_PREC_F32 ? (const void*)h->L32.p : (const void*)h->L16.p;
  a.tsc = h->prec == LS_PREC_BF16 ? h->tsc.p : nullptr;
  a.Rv = Rin; a.Y = B.Y.p; a.R = R; a.Vg = B.Vg.p; a.ring = B.ring;
  a.err = h->scal.p + lsq::S_ERR;
  a.stall = h->opt.test_stall;
  a.n_cols = h->n;
  if (kernel == 1) {
    a.fac = B.Lsw.p;
    a.tsc = nullptr;
    lsq::launch_b_local_tc(a, B.local_grid, st);
  } else {
    lsq::launch_b_local(h->prec, a, B.local_grid, st);
  }
}

// FP32 factors: which tensor-core local solve this handle uses (option block_kernel, or
// the faster of the two, timed once here, outside any stream capture, on the first
// block apply's right-hand side).
void choose_local_kernel(ls_handle* h, int R, const double* Rin) {
  BlockState& B = h->blk;
  if (B.kernel != 0 || !B.use_tc) return;
  const int opt = h->opt.block_kernel;
  if (opt == 2 && !B.u_ok)
    throw LsError(LS_ERR_UNSUPPORTED, "the tcgen05 local solve does not fit this factor's widest block row");
  if (opt == 1 || (!B.u_ok && opt == 0)) {
    swizzle_prepare(h);
    B.kernel = 1;
    return;
  }
  umma_prepare(h);
  if (opt == 2 || h->opt.test_stall) {
    B.kernel = 2;
    return;
  }
  swizzle_prepare(h);
  cudaStream_t st = h->st;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float ms[3] = {0.f, 0.f, 0.f};
  for (int k = 1; k <= 2; ++k) {
    launch_local_kernel(h, k, R, Rin);  // warm-up
    CK(cudaEventRecord(e0, st));
    launch_local_kernel(h, k, R, Rin);
    CK(cudaEventRecord(e1, st));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms[k], e0, e1));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  check_launch("block local-solve timing");
  B.kernel = ms[2] <= ms[1] ? 2 : 1;
  // the other kernel's factor copy is not needed any more
  CK(cudaStreamSynchronize(st));
  if (B.kernel == 2) {
    B.Lsw.release();
  } else {
    B.Uf.release(); B.Ub.release(); B.Ud.release();
    B.uf_off.release(); B.ub_off.release(); B.uf_row.release(); B.ub_row.release();
  }
}

// z = M^{-1} r for all pairs, with the partials of r.z (and rold.z when flexible).
void precond_block(ls_handle* h, int R, const double* Rin, double* Zout, bool flex, bool timed) {
  BlockState& B = h->blk;
  cudaStream_t st = h->st;
  choose_local_kernel(h, R, Rin);
  if (timed) record_event(h->ev[2], st);
  launch_local_kernel(h, B.use_tc ? B.kernel : 0, R, Rin);
  if (timed) record_event(h->ev[3], st);
  const bool coarse = h->coarse && h->n0 > 0;
  const bool zt = coarse && B.ZT.p != nullptr;
  if (coarse) {
    if (zt)
      lsq::launch_b_restrict32(h->N, R, h->int_off.p, h->int_glob.p, h->coff.p, B.zt_off.p, B.ZT.p, Rin, B.R0.p, st);
    else
      lsq::launch_b_restrict(h->N, R, h->int_off.p, h->int_glob.p, h->zoff.p, h->coff.p, h->Z.p, Rin, B.R0.p, st);
    const lsq::CoarseBlocks cb{h->cb_prob_of_sub.p, h->cb_base.p, h->cb_ld.p, h->cb_c0.p};
    lsq::launch_b_coarse(B.nct, R, B.ct_prob.p, B.ct_row.p, cb, B.n0q.p, h->Xinv.p, B.R0.p, B.Y0.p,
                         zt ? B.Y0f.p : nullptr, st);
  }
  if (timed) record_event(h->ev[4], st);
  lsq::BScatterArgs s{};
  s.R = R;
  s.Rp = 1;
  while (s.Rp < R) s.Rp <<= 1;
  s.map_ptr = h->map_ptr.p; s.map_idx = h->map_idx.p; s.Y = B.Y.p;
  s.coarse = coarse ? 1 : 0; s.part = h->part.p; s.jj_of = h->jj_of.p; s.zoff = h->zoff.p; s.coff = h->coff.p;
  s.nI = h->nI.p; s.Z = h->Z.p; s.Y0 = B.Y0.p;
  if (zt) { s.ZT = B.ZT.p; s.zt_off = B.zt_off.p; s.Y0f = B.Y0f.p; }
  s.Rv = Rin; s.Rold = flex ? B.Rold.p : nullptr; s.Zout = Zout;
  s.part1 = B.parts.p; s.part2 = B.parts.p + (size_t)B.nchunks * 32;
  lsq::launch_b_scatter(chunks(h), s, st);
}

int precond_launches(const ls_handle* h) { return 2 + ((h->coarse && h->n0 > 0) ? 2 : 0); }

void iteration_block(ls_handle* h, int R, bool flex) {
  BlockState& B = h->blk;
  cudaStream_t st = h->st;
  const bool timed = h->opt.time_kernels != 0;
  const lsq::BScal sc = scal(h);
  const lsq::BChunks ch = chunks(h);
  double* part2 = B.parts.p + (size_t)B.nchunks * 32;
  if (timed) record_event(h->ev[0], st);
  lsq::launch_b_spmm_csr(csr(h), B.P.p, B.Q.p, R, st);
  lsq::launch_b_spmm_csc(ch, csc(h), B.Q.p, B.W.p, R, B.P.p, B.parts.p, st);
  if (timed) record_event(h->ev[1], st);
  lsq::launch_b_finish(h->nprob, B.pc_off.p, B.parts.p, nullptr, R, sc, lsq::kFinAlpha, 0, st);
  lsq::launch_b_update(ch, R, sc.alpha, B.P.p, B.W.p, B.X.p, B.Rv.p, flex ? B.Rold.p : nullptr, B.parts.p, st);
  CK(cudaMemsetAsync(B.stat.p, 0, sizeof(int), st));
  lsq::launch_b_finish(h->nprob, B.pc_off.p, B.parts.p, nullptr, R, sc, lsq::kFinRR, 0, st);
  precond_block(h, R, B.Rv.p, B.Z.p, flex, timed);
  lsq::launch_b_finish(h->nprob, B.pc_off.p, B.parts.p, flex ? part2 : nullptr, R, sc, lsq::kFinBeta, flex ? 1 : 0,
                       st);
  lsq::launch_b_pupdate(ch, R, sc.beta, B.Z.p, B.P.p, 0, st);
  if (timed) record_event(h->ev[5], st);
  CK(cudaMemcpyAsync(B.pin, B.stat.p, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(B.pin + 2, h->scal.p + lsq::S_ERR, sizeof(double), cudaMemcpyDeviceToHost, st));
}

int iteration_launches(const ls_handle* h) { return 8 + precond_launches(h); }

template <class T>
std::vector<T> fetch(const T* p, size_t n, cudaStream_t st) {
  std::vector<T> v(n);
  if (n) CK(cudaMemcpyAsync(v.data(), p, sizeof(T) * n, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return v;
}

// tt per pair, W receiving the residual vectors: mode 0 ||A^T (B - A X)||^2 (b given),
// mode 1 ||G - A^T (A X)||^2 (the normal-equations right-hand side G given).
std::vector<double> true_residual_block(ls_handle* h, int R, int mode, int* launches) {
  BlockState& B = h->blk;
  cudaStream_t st = h->st;
  const lsq::BScal sc = scal(h);
  lsq::launch_b_spmm_csr(csr(h), B.X.p, B.Q.p, R, st);
  if (mode == 0) {
    lsq::launch_b_sub((int64_t)h->m * R, B.B.p, B.Q.p, st);
    lsq::launch_b_spmm_csc(chunks(h), csc(h), B.Q.p, B.W.p, R, nullptr, B.parts.p, st);
  } else {
    lsq::launch_b_spmm_csc(chunks(h), csc(h), B.Q.p, B.W.p, R, nullptr, nullptr, st);
    lsq::launch_b_resid(chunks(h), R, B.G.p, B.W.p, B.parts.p, st);
  }
  lsq::launch_b_finish(h->nprob, B.pc_off.p, B.parts.p, nullptr, R, sc, lsq::kFinTT, 0, st);
  *launches += 4;
  return fetch(sc.tt, (size_t)h->nprob * R, st);
}

}  // namespace

namespace lsi {

void block_plan(ls_handle* h) {
  BlockState& B = h->blk;
  cudaStream_t st = h->st;
  // chunks
  std::vector<int64_t> start;
  std::vector<int32_t> prob;
  B.h_pc_off.assign(h->nprob + 1, 0);
  for (int q = 0; q < h->nprob; ++q) {
    B.h_pc_off[q] = (int64_t)start.size();
    for (int64_t j = h->h_n_off[q]; j < h->h_n_off[q + 1]; j += kChunkCols) {
      start.push_back(j);
      prob.push_back(q);
    }
  }
  B.h_pc_off[h->nprob] = (int64_t)start.size();
  B.nchunks = (int64_t)start.size();
  start.push_back(h->n);
  B.chunk_start.upload(start, st);
  B.chunk_prob.upload(prob, st);
  B.pc_off.upload(B.h_pc_off, st);
  B.parts.alloc((size_t)B.nchunks * 32 * 2);
  B.sc.alloc((size_t)h->nprob * 32 * 8);
  B.sc.zero(st);
  B.act.alloc((size_t)h->nprob * 32);
  B.its.alloc((size_t)h->nprob * 32);
  B.stat.alloc(2);
  B.qctr.alloc(1);
  if (!B.pin) CK(cudaMallocHost(&B.pin, 4 * sizeof(int)));
  // work order of the persistent local solve: subdomains by decreasing size
  std::vector<int32_t> order(h->N);
  for (int i = 0; i < h->N; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return h->h_om_off[a + 1] - h->h_om_off[a] > h->h_om_off[b + 1] - h->h_om_off[b];
  });
  B.order.upload(order, st);
  B.ring = h->wmax;
  int optin = 0, sms = 0;
  CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->dev));
  const size_t need = lsq::block_local_smem(fac_bytes(h->prec), arith_bytes(h->prec), B.ring);
  B.local_ok = need <= (size_t)optin;
  B.use_tc = h->prec == LS_PREC_F32;
  if (B.local_ok) {
    const int occ = B.use_tc ? lsq::block_local_tc_occupancy(B.ring) : lsq::block_local_occupancy(h->prec, B.ring);
    B.local_grid = std::max(1, std::min(h->N, sms * std::max(occ, 1)));
    B.Vg.alloc((size_t)h->total_blocks * 1024 * arith_bytes(h->prec));
  }
  if (B.use_tc) {
    // tcgen05 kernel: a window of (widest block row + 1) tiles, one CTA per SM, tensor
    // memory for the M = 128 chunks of the largest step (at most widest - 1 tiles)
    B.u_ring = h->wmax + 1;
    B.u_tmem = lsq::block_local_umma_tmem_cols(std::max(h->wmax - 1, 1));
    B.u_fs = lsq::block_local_umma_stages(B.u_ring, (size_t)optin);
    B.u_smem = lsq::block_local_umma_smem(B.u_ring, B.u_fs);
    B.u_ok = B.local_ok && B.u_tmem > 0 && B.u_smem <= (size_t)optin && lsq::block_local_umma_prepare(B.u_smem);
    B.u_grid = std::max(1, std::min(h->N, sms));
    cudaGetLastError();
  }
  B.kernel = 0;
  // coarse tiles (problem, 32-row tile)
  std::vector<int32_t> cp, cr, n0q(h->nprob, 0);
  for (int q = 0; q < h->nprob; ++q) {
    n0q[q] = h->h_n0q.empty() ? 0 : h->h_n0q[q];
    for (int t = 0; t < (n0q[q] + 31) / 32; ++t) {
      cp.push_back(q);
      cr.push_back(t);
    }
  }
  B.nct = (int)cp.size();
  // mixed forms: the coarse restriction and prolongation run in FP32 from a transposed
  // copy of the basis (the coarse solve itself stays FP64)
  if (h->prec != LS_PREC_F64 && h->coarse && h->n0 > 0) {
    std::vector<int64_t> zo(h->N + 1, 0);
    for (int i = 0; i < h->N; ++i) zo[i + 1] = zo[i] + (int64_t)h->h_nI[i] * ((h->h_k[i] + 3) & ~3);
    B.zt_off.upload(zo, st);
    B.ZT.alloc(std::max<int64_t>(zo[h->N], 1));
    lsq::launch_b_ztrans(h->N, h->int_off.p, h->zoff.p, h->coff.p, B.zt_off.p, h->Z.p, B.ZT.p, st);
  }
  B.ct_prob.upload(cp, st);
  B.ct_row.upload(cr, st);
  B.n0q.upload(n0q, st);
  CK(cudaStreamSynchronize(st));
  check_launch("block plan");
}

namespace {

void check_block(const ls_handle* h, int R) {
  if (R < 1 || R > 32) throw LsError(LS_ERR_UNSUPPORTED, "the multi right-hand-side path takes 1 to 32 right-hand sides");
  if (h->opt.variant != 0)
    throw LsError(LS_ERR_UNSUPPORTED, "the multi right-hand-side path applies the additive two-level operator");
  if (!h->blk.local_ok)
    throw LsError(LS_ERR_UNSUPPORTED, "the widest local factor block row (" + std::to_string(h->blk.ring) +
                                          " tiles) does not fit the multi right-hand-side local solve");
}

// the caller's column-major array (host or device, rows x R) as a device pointer
// (host data goes through the staging buffer Bu)
const double* device_view(ls_handle* h, const double* p, int64_t rows, int R) {
  if (is_device_ptr(p)) return p;
  CK(cudaMemcpyAsync(h->blk.Bu.p, p, sizeof(double) * rows * R, cudaMemcpyHostToDevice, h->st));
  return h->blk.Bu.p;
}

// Block PCG from x = 0 once Rv holds the normal-equations right-hand side of every pair
// and gg its squared norms; mode 0: b in B (true residual A^T (b - A x)), mode 1: G
// given (true residual G - A^T A x).  Result in X.  Returns whether all pairs passed.
bool block_core(ls_handle* h, int R, double rtol, int mode, const std::vector<double>& gg, ls_info& inf,
                int& launches) {
  BlockState& B = h->blk;
  cudaStream_t st = h->st;
  const bool flex = h->prec != LS_PREC_F64;
  const int NP = h->nprob * R;
  const lsq::BScal sc = scal(h);
  const lsq::BChunks ch = chunks(h);
  const int fixed = h->opt.fixed_iters;
  std::vector<double> thr2(NP);
  std::vector<int> act(NP);
  int nact = 0;
  for (int i = 0; i < NP; ++i) {
    if (!std::isfinite(gg[i])) throw LsError(LS_ERR_NONFINITE, "right-hand side is not finite");
    act[i] = gg[i] > 0.0 ? 1 : 0;
    thr2[i] = fixed > 0 ? -1.0 : rtol * rtol * gg[i];
    nact += act[i];
  }
  CK(cudaMemcpyAsync(sc.thr2, thr2.data(), sizeof(double) * NP, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(sc.act, act.data(), sizeof(int) * NP, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(sc.its, 0, sizeof(int) * NP, st));
  CK(cudaMemsetAsync(B.X.p, 0, sizeof(double) * h->n * R, st));
  CK(cudaMemsetAsync(B.stat.p, 0, sizeof(int) * 2, st));
  CK(cudaMemsetAsync(h->scal.p + lsq::S_ERR, 0, sizeof(double), st));
  auto restart = [&]() {
    precond_block(h, R, B.Rv.p, B.Z.p, false, false);
    lsq::launch_b_finish(h->nprob, B.pc_off.p, B.parts.p, nullptr, R, sc, lsq::kFinBeta0, 0, st);
    lsq::launch_b_pupdate(ch, R, sc.beta, B.Z.p, B.P.p, 1, st);
    launches += precond_launches(h) + 2;
    inf.local_launches += 1;
  };
  const int maxit = fixed > 0 ? fixed : h->opt.maxit;
  bool converged = nact == 0;
  int it = 0, restarts = 0;
  std::vector<double> tt;
  if (!converged) {
    restart();
    check_launch("initial block preconditioner apply");
  }
  const bool timed = h->opt.time_kernels != 0;
  bool graph_this = h->opt.use_graph != 0;
  while (!converged && it < maxit) {
    if (graph_this) {
      if (!B.gexec || B.gR != R) {
        if (B.gexec) cudaGraphExecDestroy(B.gexec);
        B.gexec = nullptr;
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        iteration_block(h, R, flex);
        CK(cudaStreamEndCapture(st, &g));
        cudaError_t e = cudaGraphInstantiate(&B.gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
          B.gexec = nullptr;
          cudaGetLastError();
          graph_this = false;
          continue;
        }
        B.gR = R;
      }
      CK(cudaGraphLaunch(B.gexec, st));
    } else {
      iteration_block(h, R, flex);
    }
    CK(cudaStreamSynchronize(st));
    check_launch("block CG iteration");
    ++it;
    launches += iteration_launches(h);
    inf.local_launches += 1;
    if (timed) {
      float ta = 0.f, tb = 0.f, tc = 0.f, td = 0.f;
      CK(cudaEventElapsedTime(&ta, h->ev[0], h->ev[1]));
      CK(cudaEventElapsedTime(&tb, h->ev[2], h->ev[3]));
      CK(cudaEventElapsedTime(&tc, h->ev[3], h->ev[4]));
      CK(cudaEventElapsedTime(&td, h->ev[0], h->ev[5]));
      inf.ms_spmv += ta; inf.ms_local += tb; inf.ms_coarse += tc; inf.ms_iter += td;
    }
    const double* perr = reinterpret_cast<const double*>(B.pin + 2);
    if (*perr == lsq::kErrBounds)
      throw LsError(LS_ERR_INVALID, "an index out of range was met (bounds-checked build) at iteration " +
                                        std::to_string(it));
    if (*perr != 0.0)
      throw LsError(LS_ERR_DEVICE_TIMEOUT, "a bounded wait in the block local-solve kernel gave up at iteration " +
                                               std::to_string(it));
    if (B.pin[1] != 0)
      throw LsError(LS_ERR_NONFINITE, "block CG breakdown (non-finite scalar or non-positive p.Cp) at iteration " +
                                          std::to_string(it));
    if (fixed > 0) continue;
    if (B.pin[0] == 0) {
      tt = true_residual_block(h, R, mode, &launches);
      int fail = 0;
      for (int i = 0; i < NP; ++i) {
        act[i] = (gg[i] > 0.0 && tt[i] > thr2[i]) ? 1 : 0;
        fail += act[i];
      }
      if (fail == 0) {
        converged = true;
        break;
      }
      CK(cudaMemcpyAsync(sc.act, act.data(), sizeof(int) * NP, cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(B.Rv.p, B.W.p, sizeof(double) * h->n * R, cudaMemcpyDeviceToDevice, st));
      ++restarts;
      restart();
    }
  }
  if (tt.empty() || !converged) tt = true_residual_block(h, R, mode, &launches);
  std::vector<int> its = fetch(sc.its, NP, st);
  std::vector<double> rr = fetch(sc.rr, NP, st);
  check_launch("block solve");
  B.h_its.assign(its.begin(), its.end());
  B.h_rel.assign(NP, 0.0);
  double worst = 0.0, worst_rec = 0.0;
  for (int i = 0; i < NP; ++i) {
    const double g = gg[i] > 0.0 ? std::sqrt(gg[i]) : 1.0;
    B.h_rel[i] = gg[i] > 0.0 ? std::sqrt(std::max(tt[i], 0.0)) / g : 0.0;
    worst = std::max(worst, B.h_rel[i]);
    if (gg[i] > 0.0) worst_rec = std::max(worst_rec, std::sqrt(std::max(rr[i], 0.0)) / g);
    inf.iters = std::max(inf.iters, its[i]);
  }
  if (fixed > 0) inf.iters = it;
  inf.restarts = restarts;
  inf.relres_true = worst;
  inf.relres_recursive = worst_rec;
  inf.n0 = h->sinfo.n0; inf.kmin = h->sinfo.kmin; inf.kmax = h->sinfo.kmax; inf.tau_used = h->sinfo.tau_used;
  inf.delta = h->sinfo.delta; inf.t_setup = h->sinfo.t_setup; inf.t_eig = h->sinfo.t_eig;
  inf.eig_steps_max = h->sinfo.eig_steps_max;
  inf.lanes_csr = h->lanes_csr; inf.lanes_csc = h->lanes_csc; inf.normal_product = h->normal_kind; inf.local_config = h->local_cfg;
  inf.local_kernel = h->blk.use_tc ? h->blk.kernel : 0;
  return converged || fixed > 0;
}

}  // namespace

ls_status block_solve(ls_handle* h, const double* b, int R, double rtol, double* x, ls_info* info) {
  BlockState& B = h->blk;
  cudaStream_t st = h->st;
  check_block(h, R);
  const double t0 = now_s();
  ensure_buffers(h, R);
  ls_info inf{};
  inf.bad_subdomain = -1;
  int launches = 0;
  const lsq::BScal sc = scal(h);
  // B = P b (interleaved), R = A^T B, gg = ||A^T B||^2
  lsq::launch_b_load_rows(h->m, R, h->perm.p, device_view(h, b, h->m, R), B.B.p, st);
  lsq::launch_b_spmm_csc(chunks(h), csc(h), B.B.p, B.Rv.p, R, nullptr, B.parts.p, st);
  CK(cudaMemsetAsync(B.act.p, 0, sizeof(int) * h->nprob * R, st));
  lsq::launch_b_finish(h->nprob, B.pc_off.p, B.parts.p, nullptr, R, sc, lsq::kFinGG, 0, st);
  launches += 3;
  const std::vector<double> gg = fetch(sc.gg, (size_t)h->nprob * R, st);
  const bool ok = block_core(h, R, rtol, 0, gg, inf, launches);
  // x (caller's column-major layout)
  if (is_device_ptr(x)) {
    lsq::launch_b_store_cols(h->n, R, B.X.p, x, st);
  } else {
    lsq::launch_b_store_cols(h->n, R, B.X.p, B.Bu.p, st);
    CK(cudaMemcpyAsync(x, B.Bu.p, sizeof(double) * h->n * R, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  launches += 1;
  inf.launches = launches;
  inf.t_solve = now_s() - t0;
  if (info) *info = inf;
  if (!ok)
    throw LsError(LS_ERR_NOT_CONVERGED, "maximum number of iterations reached, worst true relative residual " +
                                            std::to_string(inf.relres_true));
  return LS_OK;
}

ls_status block_backward(ls_handle* h, const double* b, const double* x, const double* grad_x, int R, double rtol,
                         double* grad_b, double* grad_vals, ls_info* info) {
  BlockState& B = h->blk;
  cudaStream_t st = h->st;
  check_block(h, R);
  const double t0 = now_s();
  ensure_buffers(h, R);
  B.G.alloc((size_t)h->n * R);
  ls_info inf{};
  inf.bad_subdomain = -1;
  int launches = 0;
  const lsq::BScal sc = scal(h);
  // lambda = C^{-1} grad_x for every pair: G = grad_x (interleaved), R = G, gg = ||G||^2
  lsq::launch_b_load_cols(h->n, R, device_view(h, grad_x, h->n, R), B.G.p, st);
  CK(cudaMemsetAsync(B.Rv.p, 0, sizeof(double) * h->n * R, st));
  lsq::launch_b_resid(chunks(h), R, B.G.p, B.Rv.p, B.parts.p, st);
  CK(cudaMemsetAsync(B.act.p, 0, sizeof(int) * h->nprob * R, st));
  lsq::launch_b_finish(h->nprob, B.pc_off.p, B.parts.p, nullptr, R, sc, lsq::kFinGG, 0, st);
  launches += 3;
  const std::vector<double> gg = fetch(sc.gg, (size_t)h->nprob * R, st);
  const bool ok = block_core(h, R, rtol, 1, gg, inf, launches);  // lambda in X
  // A lambda (rows of the reordered matrix); grad_b = P^T A lambda
  lsq::launch_b_spmm_csr(csr(h), B.X.p, B.Q.p, R, st);
  if (grad_b) {
    if (is_device_ptr(grad_b)) {
      lsq::launch_b_store_rows(h->m, R, h->perm.p, B.Q.p, grad_b, st);
    } else {
      lsq::launch_b_store_rows(h->m, R, h->perm.p, B.Q.p, B.Bu.p, st);
      CK(cudaMemcpyAsync(grad_b, B.Bu.p, sizeof(double) * h->m * R, cudaMemcpyDeviceToHost, st));
    }
    launches += 1;
  }
  if (grad_vals) {
    // x interleaved into Z, b into B, rho = b - A x into Bu
    lsq::launch_b_load_cols(h->n, R, device_view(h, x, h->n, R), B.Z.p, st);
    lsq::launch_b_load_rows(h->m, R, h->perm.p, device_view(h, b, h->m, R), B.B.p, st);
    lsq::launch_b_spmm_csr(csr(h), B.Z.p, B.Bu.p, R, st);
    lsq::launch_b_sub((int64_t)h->m * R, B.B.p, B.Bu.p, st);
    DevBuf<double> gout;
    gout.alloc(h->nnz);
    lsq::launch_b_grad_vals(csr(h), h->entmap.p, R, B.Bu.p, B.X.p, B.Q.p, B.Z.p, gout.p, st);
    CK(cudaMemcpyAsync(grad_vals, gout.p, sizeof(double) * h->nnz, cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
    launches += 5;
  }
  CK(cudaStreamSynchronize(st));
  check_launch("block adjoint");
  inf.launches = launches;
  inf.t_solve = now_s() - t0;
  if (info) *info = inf;
  if (!ok)
    throw LsError(LS_ERR_NOT_CONVERGED, "adjoint solve: maximum number of iterations reached, worst true relative "
                                        "residual " + std::to_string(inf.relres_true));
  return LS_OK;
}

}  // namespace lsi
