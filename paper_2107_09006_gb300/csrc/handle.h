// Internal: the handle behind the C ABI and the helpers shared by the translation units
// of the library (setup and single right-hand-side solve in api.cu, the batched
// multi right-hand-side solve in block.cu).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <chrono>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/ls_schwarz.h"
#include "kernels.h"

namespace lsi {

struct LsError : std::runtime_error {
  ls_status st;
  LsError(ls_status s, const std::string& m) : std::runtime_error(m), st(s) {}
};

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      throw LsError(e_ == cudaErrorMemoryAllocation ? LS_ERR_OOM : LS_ERR_CUDA,               \
                    std::string(#call) + ": " + cudaGetErrorString(e_));                      \
  } while (0)

template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  void alloc(size_t count) {
    release();
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      throw LsError(LS_ERR_OOM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
    }
    n = count;
  }
  void zero(cudaStream_t st) { CK(cudaMemsetAsync(p, 0, n * sizeof(T), st)); }
  void upload(const std::vector<T>& v, cudaStream_t st) {
    alloc(v.size());
    if (!v.empty()) CK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  }
  template <class U>
  void upload_from(const U* src, size_t count, cudaStream_t st) {
    alloc(count);
    if (count) CK(cudaMemcpyAsync(p, src, count * sizeof(T), cudaMemcpyDefault, st));
  }
};

// NVTX ranges for the phases of setup and solve (seen by Nsight tools; a few
// nanoseconds each when no tool is attached).  next() closes the current range and
// opens the following one; the destructor closes the last, also on an error path.
struct Phase {
  bool open = false;
  explicit Phase(const char* name) { next(name); }
  Phase(const Phase&) = delete;
  Phase& operator=(const Phase&) = delete;
  void next(const char* name) {
    if (open) nvtxRangePop();
    nvtxRangePushA(name);
    open = true;
  }
  ~Phase() {
    if (open) nvtxRangePop();
  }
};

inline double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Records a timing event on st: as an external node while st is being captured into a
// graph (so the replay records it), as a plain record otherwise.
inline void record_event(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(st, &cs));
  if (cs == cudaStreamCaptureStatusActive) CK(cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal));
  else CK(cudaEventRecord(ev, st));
}

inline void check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw LsError(LS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Buffers and captured graph of the multi right-hand-side solve (block.cu); R is the
// number of right-hand sides they are sized for, vectors are interleaved [index][R].
struct BlockState {
  int R = 0;
  DevBuf<double> X, Rv, Rold, Z, P, W, Q, B, Y, R0, Y0, Bu, G;
  DevBuf<unsigned char> Vg;          // forward-sweep spill of the local solves
  DevBuf<double> parts, sc;          // chunk partials; per (problem, rhs) scalars
  DevBuf<int> act, its, stat;        // active mask, iterations, {nact, flag, err}
  DevBuf<unsigned> qctr;             // work counter of the persistent local solve
  int* pin = nullptr;                // pinned copy of stat
  cudaGraphExec_t gexec = nullptr;
  int gR = 0;
  // reduction chunks: column ranges inside one problem
  int64_t nchunks = 0;
  DevBuf<int64_t> chunk_start;
  DevBuf<int32_t> chunk_prob;
  std::vector<int64_t> h_pc_off;
  DevBuf<int64_t> pc_off;
  // persistent local solve: subdomains by decreasing size, grid size
  DevBuf<int32_t> order;
  int local_grid = 0;
  int ring = 0;           // solution tiles kept in shared memory (widest block row)
  bool local_ok = false;  // the ring fits the shared memory of one CTA
  bool use_tc = false;    // FP32 factors: tensor-core local solves from the swizzled copy
  DevBuf<float> Lsw;      // TF32-rounded swizzled factor tiles (made at the first block solve)
  // tcgen05 local solve (FP32 factors): per-step update tiles, the two TF32 copies in
  // core-matrix layout and the padded inverse diagonal tiles (made at the first block
  // solve that uses it); kernel: 1 the mma.sync kernel, 2 the tcgen05 kernel, 0 not yet
  // chosen (option block_kernel, or timed once at the first block solve)
  int kernel = 0;
  bool u_ok = false;
  int u_ring = 0, u_tmem = 0, u_grid = 0, u_fs = 0;
  size_t u_smem = 0;
  DevBuf<float> Uf, Ub, Ud;
  DevBuf<int64_t> uf_off, ub_off;
  DevBuf<int32_t> uf_row, ub_row;
  // coarse solve tiles: (problem, 32-row tile) pairs
  DevBuf<int32_t> ct_prob, ct_row, n0q;
  // mixed forms: FP32 transposed coarse basis and FP32 copy of the coarse solution
  DevBuf<float> ZT, Y0f;
  DevBuf<int64_t> zt_off;
  int nct = 0;
  std::vector<int> h_its;
  std::vector<double> h_rel;
  ~BlockState() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (pin) cudaFreeHost(pin);
  }
};

}  // namespace lsi

struct ls_handle {
  template <class T> using DevBuf = lsi::DevBuf<T>;
  int dev = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  cudaEvent_t ev_join = nullptr;  // orders a call against the caller's stream (ls_solve, ls_backward)
  ls_options opt{};
  double tau = 0.0;  // threshold given to ls_setup (<= 0: automatic)
  int64_t m = 0, n = 0, nnz = 0;
  int N = 0, lanes_csr = 8, lanes_csc = 32, grid_csr = 0, grid_csc = 0, prec = 0;

  DevBuf<int64_t> row_ptr, col_ptr;
  DevBuf<int32_t> col, crow, part;
  DevBuf<double> val, cval;
  // The device matrix is A' = P A (rows by first column): perm[new] = original row,
  // entmap[e'] = original CSR slot of entry e' of A'.
  DevBuf<int32_t> perm;
  DevBuf<int64_t> entmap;
  std::vector<int32_t> h_perm;
  lsq::SellDev sellA{}, sellB{};  // sliced-ELL copies of A and A^T (pointers below)
  DevBuf<int64_t> sellA_off, sellB_off;
  DevBuf<int32_t> sellA_perm, sellA_col, sellB_perm, sellB_col;
  DevBuf<double> sellA_val, sellB_val;
  DevBuf<int64_t> cperm, sellA_src, sellB_src;  // source A' CSR slot of the CSC / ELL copies
  // Row tiles of the one-pass normal product (normal_tiles.h); normal_kind: 1 two
  // products, 2 row tiles (option normal_product, or timed at setup).
  int normal_kind = 1;
  int nt_tiles = 0, nt_smem = 0, nt_cfg = 2;
  float nt_ms[5] = {0.f, 0.f, 0.f, 0.f, 0.f};  // setup timings: the pair, then configurations 1-4
  int64_t nt_stats[6] = {0, 0, 0, 0, 0, 0};  // LS_Q_NORMAL
  DevBuf<int64_t> nt_lo, nt_aoff, nt_boff, nt_poff, nt_asrc, nt_bsrc;
  DevBuf<int32_t> nt_wid, nt_as0, nt_bs0, nt_cb0, nt_cb1;
  DevBuf<uint16_t> nt_acol, nt_brow, nt_bcid;
  DevBuf<double> nt_aval, nt_bval, nt_part;

  DevBuf<int64_t> om_off, blk_off, blk_poff, map_ptr, map_idx, int_off;
  DevBuf<int32_t> om_glob, blk_tf, int_glob, int_loc, jj_of, nI;
  DevBuf<uint8_t> om_int;
  DevBuf<double> eqs, L64;
  DevBuf<float> L32, tsc;
  DevBuf<__nv_bfloat16> L16;
  int max_nb = 0;
  int local_cfg = 1;  // configuration of the single-vector local solve (option local_config)
  int64_t total_local = 0, total_blocks = 0, fac_elems = 0;

  bool coarse = false;
  int64_t n0 = 0, n0p = 0;
  DevBuf<int32_t> coff;
  DevBuf<int64_t> zoff;
  DevBuf<double> Z, Xinv;

  DevBuf<double> x, r, r_old, z, p, q, w, ybuf, r0, y0, tv, bv;
  DevBuf<double> bal_y, bal_t, bal_u, bal_v;  // work vectors of the balanced variant
  DevBuf<double> lq_u, lq_v, lq_q, lq_s, lq_t, lq_w;  // LSQR: u (m), v, M v, s, M^{-1} s, w
  DevBuf<int64_t> own;                                // RAS: local entry of column j in its own subdomain
  DevBuf<double> gm_V, gm_Z, gm_g, gm_h, gm_part;     // GMRES: Arnoldi basis, M^{-1} basis, A^T b, coefs
  DevBuf<double> parts, scal, ahist, bhist;
  DevBuf<unsigned> counters;  // ticket counters of the fused reductions
  DevBuf<int> ctr;
  double* pin = nullptr;  // pinned copy of the scalar slots
  int hist_cap = 0;

  cudaGraphExec_t gexec = nullptr;
  cudaEvent_t ev[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // kernel timing
  // The PCG loop as one graph: a conditional while node whose body is one iteration and
  // the loop test, then the copy of the scalar slots to the host.  Timing inside it uses
  // global-timer stamps (event records are not allowed in a conditional body).
  cudaGraphExec_t gloop = nullptr;
  int loop_kernels = 0;   // kernels of one loop-body pass
  bool stamping = false;  // timing marks become stamp kernels (while the loop body is captured)
  DevBuf<unsigned long long> stamps;  // [iteration][8] global-timer stamps of the loop

  // independent problems of one batched handle (block-diagonal A): problem q owns rows
  // [m_off[q], m_off[q+1]), columns [n_off[q], n_off[q+1]) and the subdomain ids
  // [N_off[q], N_off[q+1]); each has its own shift delta_q, threshold and coarse block.
  int nprob = 1;
  std::vector<int64_t> h_m_off, h_n_off;
  std::vector<int32_t> h_N_off, prob_of_sub;
  std::vector<double> h_delta, h_thr;
  DevBuf<double> dsub;                                 // delta of each subdomain's problem
  std::vector<int64_t> h_cb_base, h_cb_ld;             // coarse blocks (see lsq::CoarseBlocks)
  std::vector<int32_t> h_cb_c0, h_n0q;
  DevBuf<int32_t> cb_prob_of_sub, cb_c0;
  DevBuf<int64_t> cb_base, cb_ld;
  int64_t xinv_elems = 0;
  int wmax = 0;  // widest block row of any local factor, in 32 x 32 tiles
  lsi::BlockState blk;

  // host copies for queries
  std::vector<int64_t> h_om_off, h_xi_off;
  std::vector<int32_t> h_om_paper, h_xi, h_nI, h_k, h_steps;
  std::vector<double> h_lam;
  int kwant_cap = 0;
  ls_info sinfo{};

  ~ls_handle() {
    if (dev >= 0) cudaSetDevice(dev);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (gloop) cudaGraphExecDestroy(gloop);
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    if (ev_join) cudaEventDestroy(ev_join);
    if (pin) cudaFreeHost(pin);
    if (own_stream && st) cudaStreamDestroy(st);
  }
};

namespace lsi {

inline lsq::CsrDev csr(const ls_handle* h) {
  return lsq::CsrDev{h->m, h->n, h->row_ptr.p, h->col.p, h->val.p,
                     lsq::SellDev{h->sellA.nslices, h->sellA_off.p, h->sellA_perm.p, h->sellA_col.p, h->sellA_val.p}};
}
inline lsq::CscDev csc(const ls_handle* h) {
  return lsq::CscDev{h->m, h->n, h->col_ptr.p, h->crow.p, h->cval.p,
                     lsq::SellDev{h->sellB.nslices, h->sellB_off.p, h->sellB_perm.p, h->sellB_col.p, h->sellB_val.p}};
}

inline lsq::NormalTilesDev ntiles(ls_handle* h) {
  return lsq::NormalTilesDev{h->nt_tiles, h->nt_cfg, h->n, h->nt_smem, h->nt_lo.p, h->nt_wid.p, h->nt_as0.p, h->nt_bs0.p,
                             h->nt_aoff.p, h->nt_acol.p, h->nt_aval.p, h->nt_boff.p, h->nt_brow.p, h->nt_bval.p,
                             h->nt_bcid.p, h->nt_poff.p, h->nt_part.p, h->nt_cb0.p, h->nt_cb1.p,
                             h->scal.p ? h->scal.p + lsq::S_ERR : nullptr};
}

// The multi right-hand-side PCG (block.cu): b [R][m] and x [R][n], host or device.
ls_status block_solve(ls_handle* h, const double* b, int R, double rtol, double* x, ls_info* info);
// The adjoint of the block path (block.cu): lambda = C^{-1} grad_x for every pair, then
// grad_b = A lambda ([R][m]) and grad_vals summed over the pairs.
ls_status block_backward(ls_handle* h, const double* b, const double* x, const double* grad_x, int R, double rtol,
                         double* grad_b, double* grad_vals, ls_info* info);
// Chunk tables, work order and coarse tiles of the block solve (block.cu), built by setup.
void block_plan(ls_handle* h);

}  // namespace lsi
