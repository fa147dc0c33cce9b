// Launchers of the device kernels (host-callable; all asynchronous on `st`).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace lsq {

// ---- sparse products and CG vector kernels (k_krylov.cu) ----------------------------
// Sliced-ELL copy of a CSR matrix (slices of 32 rows; inside a window of 256 rows the
// rows are ordered by decreasing length; slice s holds width W_s = max length entries per
// row, column-major: entry k of slice row l at off[s] + 32 k + l; padding has value 0
// and column 0; perm[32 s + l] = original row, -1 for padding rows).
struct SellDev { int64_t nslices; const int64_t* off; const int32_t* perm; const int32_t* col; const double* val; };
struct CsrDev {
  int64_t m, n; const int64_t* row_ptr; const int32_t* col; const double* val;
  SellDev sell;  // used when the product runs with kernel code -2
};
struct CscDev {
  int64_t m, n; const int64_t* col_ptr; const int32_t* row; const double* val;
  SellDev sell;
};
// Kernel codes of the two sparse products (ls_info.lanes_csr / lanes_csc and the spmv
// option): 1, 2, 4, 8, 16, 32 lanes per row; -1 / -3 warp-stream with 16 / 32 rows per
// warp; -2 sliced ELL.
inline bool valid_spmv_code(int c) { return (c >= -3 && c <= -1) || c == 1 || c == 2 || c == 4 || c == 8 || c == 16 || c == 32; }

// Values a kernel writes into the error slot it is given: a bounded wait gave up, or
// (bounds-checked build) an index out of range was met and not used.
constexpr double kErrTimeout = 1.0, kErrBounds = 3.0;

// Scalar slots of the CG state kept on the device (copied to the host when the host
// needs them).  S_THR: squared residual threshold (rtol ||g||)^2 of the device loop (0: no
// test); S_ITS: iterations completed, written by the beta update.
enum {
  S_RZOLD = 0, S_ALPHA = 1, S_BETA = 2, S_RR = 3, S_FLAG = 4, S_GG = 5, S_ERR = 6,
  S_PW = 7, S_RZ = 8, S_RZO = 9, S_TMP = 10, S_THR = 11, S_ITS = 12, S_NSLOT = 14
};
constexpr int kMaxGrid = 65536;  // largest grid of a kernel that produces a dot product
constexpr int kVecGrid = 1216;   // grid cap of the n-vector kernels (8 blocks of 256 per SM)

// Where a fused dot product goes: per-block partials (parts[block], second sum at
// parts[stride + block]), a ticket counter (zero between uses) and the output slot(s)
// out[0] and out[out2].
struct DotSite { double* parts; int stride; unsigned* counter; double* out; int out2; };

void launch_spmv_csr(const CsrDev& A, const double* x, double* y, int lanes, int grid, cudaStream_t st);
// w = A^T q; with ds.parts != nullptr also (d . w) -> *ds.out (d = w if d == nullptr).
void launch_spmv_csc(const CscDev& At, const double* q, double* w, const double* d, const DotSite& ds, int lanes,
                     int grid, cudaStream_t st);
// Row tiles of A for the one-pass normal product w = A^T (A p) (layout: normal_tiles.h).
struct NormalTilesDev {
  int ntiles;
  int config;  // kernel configuration: 1, 2, 3 (512 threads, slices a warp takes at a time), 4 (1,024 threads)
  int64_t n;
  int smem_doubles;
  const int64_t* lo; const int32_t* wid; const int32_t* as0; const int32_t* bs0;
  const int64_t* aoff; const uint16_t* acol; const double* aval;
  const int64_t* boff; const uint16_t* brow; const double* bval; const uint16_t* bcid;
  const int64_t* poff; double* part;
  const int32_t* cb_t0; const int32_t* cb_t1;
  double* err;  // error slot (bounds-checked build)
};
// w = A^T (A v) over the row tiles (two launches: the tiles, then the per-column sum of
// their partial windows in tile order, with the fused d . w as in launch_spmv_csc).
void launch_normal_tiles(const NormalTilesDev& T, const double* v, double* w, const double* d, const DotSite& ds,
                         cudaStream_t st);
// Shared memory of the tile kernel for T (sets the kernel's limit; false if above the device's).
bool normal_tiles_prepare(const NormalTilesDev& T);

// alpha = scal[S_RZ] / scal[S_PW]; x += alpha p; r_old = r (if given); r -= alpha w; r.r -> rr.
void launch_cg_update(int64_t n, double* scal, const double* p, const double* w, double* x, double* r,
                      double* r_old, const DotSite& rr, int* ctr, double* alpha_hist, int hist_cap,
                      cudaStream_t st);
// beta from the scalar slots (plain or flexible form), p = z + beta p (init: p = z).
void launch_p_update(int64_t n, double* scal, int* ctr, double* beta_hist, int hist_cap, const double* z, double* p,
                     int init, int flex, cudaStream_t st);
// The loop test of the device-side PCG loop (a conditional while node of a CUDA graph):
// continue while no breakdown or device timeout is flagged, the recursive residual
// ||r||^2 = scal[S_RR] is above scal[S_THR] (when that is positive) and fewer than
// `limit` iterations have run.
void launch_cg_continue(const double* scal, const int* ctr, int limit, cudaGraphConditionalHandle hnd,
                        cudaStream_t st);
// Writes the global nanosecond timer into stamps[slot * 8 + k], slot = *ctr - after, when
// 0 <= slot < cap (kernel timing inside graphs, where event records are not allowed).
void launch_stamp(unsigned long long* stamps, const int* ctr, int cap, int k, int after, cudaStream_t st);
void launch_dot(int64_t n, const double* a, const double* b, const DotSite& ds, cudaStream_t st);
void launch_axpby(int64_t n, double alpha, const double* a, double beta, const double* b, double* out,
                  cudaStream_t st);
void launch_fill(int64_t n, double v, double* out, cudaStream_t st);
// dst[i] = src[idx[i]] for i < n
void launch_gather(int64_t n, const int32_t* idx, const double* src, double* dst, cudaStream_t st);
// dst[i] = src[idx[i]], or 0 where idx[i] < 0 (int64 indices)
void launch_gather64(int64_t n, const int64_t* idx, const double* src, double* dst, cudaStream_t st);
// dst[idx[i]] = src[i] (int32 or int64 indices; accumulate: dst[idx[i]] += src[i])
void launch_scatter_idx(int64_t n, const int32_t* idx32, const int64_t* idx64, const double* src, double* dst,
                        int accumulate, cudaStream_t st);

struct ScatterArgs {
  int64_t n;
  const int64_t* map_ptr; const int64_t* map_idx; const double* y;  // local solutions
  // coarse prolongation (coarse == 0: skipped)
  int coarse; const int32_t* part; const int32_t* jj_of; const int64_t* zoff; const int32_t* coff;
  const int32_t* nI; const double* Z; const double* y0;
  const double* r; const double* r_old;  // for the fused dots (r_old may be null)
  double* z;
  DotSite dots;  // r.z -> out[0], r_old.z -> out[out2]; parts == nullptr: no dots
  int add_coarse_only;  // 1: z = coarse term only; 2: z = local sum only
  int64_t total_local;  // entries of y (bounds-checked build)
  double* err;          // error slot (bounds-checked build)
};
void launch_scatter(const ScatterArgs& a, cudaStream_t st);
// One preconditioned LSQR step's vector updates: v = t / alpha, q = s / alpha, x += c1 w,
// w = v - c2 w.
void launch_lsqr_step(int64_t n, double inv_alpha, double c1, double c2, const double* t, const double* s, double* v,
                      double* q, double* x, double* w, cudaStream_t st);
// RAS prolongation z_j = a_j + y[own[j]] (a may be null)
void launch_ras_combine(int64_t n, const int64_t* own, const double* y, const double* a, double* z, cudaStream_t st);
// out[c] = V(:, c) . w for the k columns of V (column-major, ld); part holds
// multi_dot_grid(n) * k partial sums (deterministic order)
int multi_dot_grid(int64_t n);
void launch_multi_dot(int64_t n, const double* V, int64_t ld, int k, const double* w, double* part, double* out,
                      cudaStream_t st);
// out += sign * V coef (V column-major, ld; coef on the device)
void launch_multi_axpy(int64_t n, const double* V, int64_t ld, int k, const double* coef, double sign, double* out,
                       cudaStream_t st);
// r0 = R_0 v (coarse restriction alone, FP64)
void launch_restrict(int N, const int64_t* int_off, const int32_t* int_glob, const int64_t* zoff, const int32_t* coff,
                     const double* Z, const double* v, double* r0, cudaStream_t st);
// z = a + b - c with r.z -> ds.out[0] and (r_old != nullptr) r_old.z -> ds.out[ds.out2]
void launch_combine3(int64_t n, const double* a, const double* b, const double* c, double* z, const double* r,
                     const double* r_old, const DotSite& ds, cudaStream_t st);
void launch_gemv(int64_t n0, const double* X, const double* r0, double* y0, cudaStream_t st);
void launch_grad_vals(const CsrDev& A, const double* rho, const double* lam, const double* mu,
                      const double* x, double* g, int accumulate, cudaStream_t st);

// ---- block-envelope matrices (k_band.cu) -------------------------------------------
struct BandPlan {
  int N;
  const int64_t* om_off; const int32_t* om_glob; const uint8_t* om_int;
  const int64_t* blk_off; const int32_t* blk_tf; const int64_t* blk_poff;
  const int32_t* row_sub;  // subdomain of each local position (sum n_i entries)
};
// Assemble C_ii (all rows of A touching Omega_i) and C~_ii (rows Xi_i) into two
// zeroed storages (lower triangles).
void launch_assemble(const BandPlan& P, const CsrDev& A, const CscDev& At, const int32_t* part,
                     int64_t total_local, double* Cst, double* Ctst, cudaStream_t st);
// Per subdomain: cn2[i] = sum over interior rows of C of squared row norms (so that
// sum_i cn2[i] = ||C||_F^2); ctn2[i] = ||C~_ii||_F^2.
void launch_norms(const BandPlan& P, const double* Cst, const double* Ctst, double* cn2,
                  double* ctn2, cudaStream_t st);
// C_ii += delta_i I (dsub: one shift per subdomain, the shift of its problem),
// equilibrate C_ii with eqs = diag(C_ii)^{-1/2}; B_i = C~_ii + s_i I.
void launch_prep(const BandPlan& P, const double* dsub, const double* s, double* Cst, double* eqs,
                 const double* Ctst, double* Bst, cudaStream_t st);
// In-place Cholesky of every subdomain's matrix; idiag = 1 / diag(L);
// status[i] = 0 or 1 + the local row of the first nonpositive pivot.
// dinv: scratch of 1024 doubles per block row (inverse diagonal tiles).
void launch_band_cholesky(const BandPlan& P, double* st_fac, double* idiag, double* dinv, int* status,
                          cudaStream_t st);

// ---- batched local solves (k_local.cu) -----------------------------------------------
struct LocalArgs {
  const int64_t* om_off; const int32_t* om_glob; const double* eqs;
  const int64_t* blk_off; const int32_t* blk_tf; const int64_t* blk_poff;
  const void* fac; const float* tsc;  // solve storage (see k_local.cu); tsc: BF16 tile scales
  const double* r; double* y;
  int coarse; const int64_t* int_off; const int32_t* int_glob; const int64_t* zoff;
  const int32_t* coff; const double* Z; double* r0;
  double* err;  // set to 1 when a bounded wait on a copy gives up
  int stall;    // test hook: 1 issues no copies, so the bounded waits run out
  int64_t n_cols, fac_elems;  // bounds of the gather indices and the factor (bounds-checked build)
};
// config 1: 256 threads, 16 KB stages (two CTAs per SM); 2: 512 threads, 32 KB stages
// (one CTA per SM).
size_t local_solve_smem(int prec, int max_nb, int config);
void launch_local_solve(int prec, int config, int N, int max_nb, const LocalArgs& a, cudaStream_t st);
// Configuration 3 (FP32 factors, k_local_split.cu): each subdomain split over a cluster of
// local_split_cluster() CTAs of 512 threads.  The launcher returns false if the launch
// was refused (the caller keeps another configuration).
size_t local_split_smem(int max_nb);
int local_split_cluster();
bool local_split_launch(int N, int max_nb, const LocalArgs& a, cudaStream_t st);
// Block-envelope factor + inverse diagonal tiles (FP64) -> solve storage (prec 0/1/2);
// tsc receives one scale per 32x32 tile for BF16.
void launch_to_solve_layout(int prec, int64_t nblocks, const int64_t* poff, const double* L, const double* dinv,
                            void* dst, float* tsc, cudaStream_t st);

// ---- eigen setup (k_lanczos.cu) ----------------------------------------------------
struct EigArgs {
  BandPlan P;
  const double* Bfac; const double* Bidiag;  // chol(C~_ii + s I)
  const double* Ct;                          // C~_ii (lower), for D C_ii D products
  const double* delta;                       // per subdomain: D C_ii D = D C~_ii D + delta_i D
  int kwant_cap;                             // nev_max + 1
  int Kmax; int keep;                        // basis size and restart size
  int maxit; double tol;
  double* V; double* V2; int64_t vstride;    // per subdomain: Kmax vectors of vstride
  double* H; double* S;                      // per subdomain Kmax*Kmax
  double* vec;                               // per subdomain 3 * vstride work vectors
  double* lam;                               // per subdomain kwant_cap eigenvalues (out)
  int* nconv; int* steps; int* status;
};
size_t lanczos_smem(int max_nb);
void launch_lanczos(const EigArgs& a, cudaStream_t st);
// Z_i = interior rows of L_B^{-T} U_i for the first k_i Ritz vectors U_i (V holds them).
void launch_eigvec(const EigArgs& a, const int32_t* coff, const int64_t* zoff,
                   const int64_t* int_off, const int32_t* int_loc, double* Z, cudaStream_t st);

// ---- coarse operator (k_coarse.cu) -------------------------------------------------
// C_00 is block diagonal over independent problems: problem q's block (coarse indices
// [c0[q], c0[q] + n0_q)) is dense row-major with leading dimension ld[q] (n0_q rounded
// up to 32) at C00 + base[q].  One problem: base 0, ld n0p, c0 0.
struct CoarseBlocks { const int32_t* prob_of_sub; const int64_t* base; const int64_t* ld; const int32_t* c0; };
void launch_coarse_w(int N, const int64_t* xi_off, const int32_t* xi, const int32_t* coff,
                     const int64_t* woff, const int64_t* zoff, const int32_t* nI, const CsrDev& A,
                     const int32_t* part, const int32_t* jj_of, const double* Z, double* W,
                     int64_t total_xi, const int32_t* xi_sub, cudaStream_t st);
void launch_coarse_pairs(int npairs, const int32_t* pi, const int32_t* pj, const int64_t* poff,
                         const int32_t* ppi, const int32_t* ppj, const int32_t* coff,
                         const int64_t* woff, const int64_t* zoff, const int32_t* nI,
                         const double* W, const double* Z, const double* dsub, const CoarseBlocks& cb,
                         double* C00, cudaStream_t st);
// Dense SPD inverse through its Cholesky factor (tiles of 32; n a multiple of 32,
// row-major, full storage): A is replaced by A^{-1}; Y (n x n) and dinv (n/32 * 1024)
// are scratch; *status (device) receives 0 or 1 + the first failing row.
void dense_spd_inverse(int64_t n, double* A, double* Y, double* dinv, int* status, cudaStream_t st);

// ---- multi right-hand-side kernels (k_block.cu) ----------------------------------------
// Block vectors are interleaved: entry (j, k) of an n x R block at j * R + k (R <= 32).
// Chunks: ranges of at most 256 columns inside one problem; chunk c covers
// [start[c], start[c+1]) of problem prob[c]; partial sums live at part[c * 32 + k].
struct BChunks { int64_t n; const int64_t* start; const int32_t* prob; };
// Per (problem, right-hand side) CG scalars, index q * R + k; stat[0] counts the
// still-active pairs after a residual update, stat[1] flags a breakdown.
struct BScal {
  double* gg; double* thr2; double* rzold; double* pw; double* alpha; double* beta; double* rr; double* tt;
  int* act; int* its; int* stat;
};
enum { kFinGG = 0, kFinAlpha = 1, kFinRR = 2, kFinBeta0 = 3, kFinBeta = 4, kFinTT = 5 };
struct BScatterArgs {
  int R, Rp;
  const int64_t* map_ptr; const int64_t* map_idx; const double* Y;  // local solutions [sum n_i][R]
  int coarse; const int32_t* part; const int32_t* jj_of; const int64_t* zoff; const int32_t* coff;
  const int32_t* nI; const double* Z; const double* Y0;
  const float* ZT; const int64_t* zt_off; const float* Y0f;  // FP32 prolongation when ZT != nullptr
  const double* Rv; const double* Rold; double* Zout; double* part1; double* part2;
};
constexpr int kBlockRingBytes = 32768;  // shared-memory ring of factor tiles per CTA
struct BLocalArgs {
  int N; const int32_t* order; unsigned* qctr;  // work queue: subdomains by decreasing size
  const int64_t* om_off; const int32_t* om_glob; const double* eqs;
  const int64_t* blk_off; const int32_t* blk_tf; const int64_t* blk_poff;
  const void* fac; const float* tsc;
  const double* Rv; double* Y; int R;
  void* Vg;  // forward-sweep spill: 32 x 32 arithmetic-precision tile per block row
  int ring;  // tiles of the solution window kept in shared memory (>= widest block row)
  double* err;
  int stall;  // test hook: 1 issues no copies, so the bounded waits run out
  int64_t n_cols;  // rows of Rv (bounds-checked build)
};
size_t block_local_smem(int fac_bytes, int arith_bytes, int ring);
int block_local_occupancy(int prec, int ring);
void launch_b_local(int prec, const BLocalArgs& a, int grid, cudaStream_t st);
// FP32 factors on the tensor cores (TF32 MMA): a.fac is the swizzled TF32 copy that
// launch_b_swizzle makes from the FP32 solve storage.
int block_local_tc_occupancy(int ring);
void launch_b_local_tc(const BLocalArgs& a, int grid, cudaStream_t st);
void launch_b_swizzle(int64_t nelem, const float* src, float* dst, cudaStream_t st);

// FP32 factors on the 5th-generation tensor cores (tcgen05, k_block_umma.cu): right-
// looking sweeps whose block-step updates run as M = 128 MMAs with the accumulator in
// tensor memory.  f_* / b_*: the update tiles of the forward / backward step of global
// block row g are [off[g], off[g + 1]) of the forward / backward copy (TF32, core-matrix
// layout, 1024 floats per tile), row[e] the local block row tile e updates; dinv: the
// inverse diagonal tile of every block row, row-major with rows of 33 floats.
struct BUmmaArgs {
  int N; const int32_t* order;                  // subdomains by decreasing size (dealt round-robin)
  const int64_t* om_off; const int32_t* om_glob; const double* eqs;
  const int64_t* blk_off;
  const float* ffac; const int64_t* f_off; const int32_t* f_row;
  const float* bfac; const int64_t* b_off; const int32_t* b_row;
  const float* dinv;
  const double* Rv; double* Y; int R;
  float* spill;   // forward results of block rows that leave the window (1024 floats per block row)
  int ring;       // window tiles kept in shared memory (>= widest block row + 1)
  int tmem_cols;  // tensor-memory columns (512: two steps x 256)
  int ncol;       // accumulator columns per chunk: 64 (steps of <= 4 chunks) or 32 (<= 8)
  int fs;         // factor chunk stages (block_local_umma_stages)
  double* err;
  int stall;      // test hook: 1 issues no copies, so the bounded waits run out
  int64_t n_cols, f_tiles, b_tiles;  // bounds of Rv and of the two copies (bounds-checked build)
};
size_t block_local_umma_smem(int ring, int fs);
// the most factor chunk stages (2 .. 8) whose shared memory fits smem_limit
int block_local_umma_stages(int ring, size_t smem_limit);
// tensor-memory columns for steps of at most max_step_tiles update tiles (0: unsupported)
int block_local_umma_tmem_cols(int max_step_tiles);
// accumulator columns per chunk for such steps (64, or 32 for more than 4 chunks)
int block_local_umma_ncol(int max_step_tiles);
bool block_local_umma_prepare(size_t smem);
void launch_b_local_umma(const BUmmaArgs& a, int grid, cudaStream_t st);
// tile t of dst <- the 32 x 32 column-major tile at L32 + src_off[t], TF32-rounded, in
// core-matrix layout (transpose: the tile's columns along M)
void launch_bu_copy(int64_t ntiles, const int64_t* src_off, const float* L32, float* dst, int transpose,
                    cudaStream_t st);
void launch_bu_diag(int64_t nblocks, const int64_t* poff, const float* L32, float* dst, cudaStream_t st);
void launch_b_spmm_csr(const CsrDev& A, const double* X, double* Y, int R, cudaStream_t st);
void launch_b_spmm_csc(const BChunks& ch, const CscDev& At, const double* Q, double* W, int R, const double* D,
                       double* part, cudaStream_t st);
void launch_b_update(const BChunks& ch, int R, const double* alpha, const double* P, const double* W, double* X,
                     double* Rv, double* Rold, double* part, cudaStream_t st);
void launch_b_pupdate(const BChunks& ch, int R, const double* beta, const double* Z, double* P, int init,
                      cudaStream_t st);
void launch_b_finish(int nprob, const int64_t* pc_off, const double* part, const double* part2, int R,
                     const BScal& s, int mode, int flex, cudaStream_t st);
void launch_b_scatter(const BChunks& ch, const BScatterArgs& a, cudaStream_t st);
void launch_b_restrict(int N, int R, const int64_t* int_off, const int32_t* int_glob, const int64_t* zoff,
                       const int32_t* coff, const double* Z, const double* Rv, double* R0, cudaStream_t st);
void launch_b_coarse(int ntiles, int R, const int32_t* ct_prob, const int32_t* ct_row, const CoarseBlocks& cb,
                     const int32_t* n0q, const double* Xinv, const double* R0, double* Y0, float* Y0f,
                     cudaStream_t st);
// FP32 transposed coarse basis (mixed forms): ZT[zt_off[i] + jj * kp_i + t] = Zbar_i[t, jj],
// kp_i = k_i rounded up to 4; restriction with it.
void launch_b_ztrans(int N, const int64_t* int_off, const int64_t* zoff, const int32_t* coff, const int64_t* zt_off,
                     const double* Z, float* ZT, cudaStream_t st);
void launch_b_restrict32(int N, int R, const int64_t* int_off, const int32_t* int_glob, const int32_t* coff,
                         const int64_t* zt_off, const float* ZT, const double* Rv, double* R0, cudaStream_t st);
void launch_b_load_rows(int64_t m, int R, const int32_t* perm, const double* Bu, double* Bb, cudaStream_t st);
void launch_b_store_cols(int64_t n, int R, const double* Xb, double* Xu, cudaStream_t st);
// b = a - b over len entries
void launch_b_sub(int64_t len, const double* a, double* b, cudaStream_t st);
// Xb = interleaved copy of the caller's column-major n-vectors Xu ([R][n])
void launch_b_load_cols(int64_t n, int R, const double* Xu, double* Xb, cudaStream_t st);
// Yu[k * m + perm[r]] = Yb[r * R + k]
void launch_b_store_rows(int64_t m, int R, const int32_t* perm, const double* Yb, double* Yu, cudaStream_t st);
// W = G - W and the chunk partials of W . W
void launch_b_resid(const BChunks& ch, int R, const double* G, double* W, double* part, cudaStream_t st);
// gradient on the stored entries of A (caller's CSR order through entmap), summed over
// the R right-hand sides: rho lam^T - (A lam) x^T sampled on the pattern
void launch_b_grad_vals(const CsrDev& A, const int64_t* entmap, int R, const double* rho, const double* lam,
                        const double* Al, const double* X, double* out, cudaStream_t st);

}  // namespace lsq
