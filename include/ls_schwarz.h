/*
 * ls_schwarz.h -- C ABI of a GB300 (sm_103a) solver for sparse linear least squares
 *
 *     min_x || A x - b ||_2,   A in R^{m x n}, m >= n,
 *
 * by conjugate gradients on the normal equations C x = A^T b, C = A^T A (eq. (1.2)
 * of Al Daas, Jolivet & Scott, arXiv 2107.09006), preconditioned by the two-level
 * additive Schwarz preconditioner of eq. (2.3):
 *
 *     M^{-1} = R_0^T C_00^{-1} R_0 + sum_i R_i^T C_ii^{-1} R_i,
 *
 * with overlapping subdomains Omega_i = [Omega_I,i, Omega_Gamma,i] built from the
 * rows Xi_i of A that touch the interior columns (Section 3), local matrices
 * C_ii = A(:,Omega_i)^T A(:,Omega_i) (Section 3.1), the local SPSD splittings
 * C~_ii = A(Xi_i,Omega_i)^T A(Xi_i,Omega_i) (eq. (3.2)), and a coarse space from the
 * shifted generalized eigenproblems D_i C_ii D_i v = lambda (C~_ii + s I) v with
 * threshold tau (eqs. (3.4)-(3.6), Algorithm 1).  C is never formed in the solve:
 * it is applied as A^T (A p) (Section 4.1.3).
 *
 * Conventions shared by every call:
 *  - Pointers may be host or device memory (the library inspects each one); the
 *    caller owns every pointer it passes and may free it after the call returns.
 *  - Index arrays are 0-based.  CSR column indices must be strictly increasing
 *    within each row (no duplicates); "nonzero" means "stored", as in Section 3.
 *  - Every call returns an ls_status; on failure ls_last_error() gives a message
 *    (thread-local, valid until the next call from the same thread) and no output
 *    is to be trusted, but the handle stays valid for ls_free.
 *  - Calls are synchronous with respect to their outputs: when a call returns,
 *    its outputs are written (device outputs are complete on the handle's stream).
 *  - All device work of a handle runs on one CUDA stream on the device that was
 *    current at ls_setup; calls on one handle must not overlap.
 */
#ifndef LS_SCHWARZ_H
#define LS_SCHWARZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LS_OK = 0,
    LS_ERR_INVALID = 1,        /* bad argument: sizes, CSR structure, partition ids     */
    LS_ERR_OOM = 2,            /* device or host allocation failed                      */
    LS_ERR_CUDA = 3,           /* a CUDA runtime call failed                            */
    LS_ERR_FACTOR = 4,         /* a local or coarse Cholesky met a pivot <= 0           */
    LS_ERR_EIGEN = 5,          /* a local eigensolve did not converge                   */
    LS_ERR_NOT_CONVERGED = 6,  /* maxit reached before the residual test passed         */
    LS_ERR_NONFINITE = 7,      /* NaN or Inf met in the input or in a CG scalar         */
    LS_ERR_DEVICE_TIMEOUT = 8, /* a bounded device-side wait gave up                    */
    LS_ERR_UNSUPPORTED = 9     /* valid request outside what this build implements     */
} ls_status;

typedef enum {
    LS_PREC_F64 = 0,  /* local factors and triangular solves in FP64 (plain CG)             */
    LS_PREC_F32 = 1,  /* local factors in FP32, FP64 outer flexible CG                      */
    LS_PREC_BF16 = 2  /* local factors in BF16 with one FP32 scale per 32x32 tile, FP32
                         accumulation, FP64 outer flexible CG                               */
} ls_precision;

typedef struct {
    int nev_max;       /* most coarse vectors per subdomain (Section 4 uses 300)       */
    double delta_rel;  /* construction shift delta = delta_rel ||C||_F (Section 4.1.2) */
    double s_rel;      /* GEVP shift s_i = s_rel ||C~_ii||_F (Section 4.1.2)           */
    int factor_prec;   /* ls_precision                                                  */
    int maxit;         /* CG iteration limit                                            */
    int coarse;        /* 1: two-level additive (eq. (2.3)); 0: one-level ASM (eq. (2.1)) */
    int fixed_iters;   /* > 0: run exactly this many CG iterations, no residual test    */
    int eig_maxit;     /* limit on Lanczos steps per subdomain eigensolve               */
    double eig_tol;    /* relative Ritz residual tolerance of the eigensolve           */
    int use_graph;     /* 1: replay each CG iteration as a captured CUDA graph          */
    int time_kernels;  /* 1: time the local-solve and sparse-product launches of each
                          iteration with CUDA events (reported in ls_info)           */
    int equilibrate;   /* 1: build the preconditioner for the column-equilibrated problem
                          A S (S = diag(1/||A(:,j)||)) and apply S M_S^{-1} S.  Without
                          shifts the method is invariant under column scaling; with the
                          shifts delta and s of Section 4.1.2 it is not, and badly scaled
                          columns then see a shift far above their diagonal.  0 (the
                          default) follows the paper as written.                      */
    int variant;       /* second level: 0 additive (eq. (2.3), the default); 1 balanced,
                          Q + (I - CQ)^T M_1 (I - CQ) with Q = R_0^T C_00^{-1} R_0 and the
                          one-level M_1 (Section 2): two more products with C and one
                          more coarse correction per apply; 2 deflated with the
                          restricted first level (RAS, each column takes the solution
                          of its own subdomain only), Q + M_RAS (I - CQ): not symmetric,
                          so it needs solver = 2 (GMRES).  1 and 2: single-problem
                          handles, one right-hand side (else LS_ERR_UNSUPPORTED).      */
    int solver;        /* outer Krylov method of ls_solve: 0 PCG on the normal equations
                          (the default); 1 LSQR preconditioned with M^{-1} (the paper's
                          solver, Section 4.1.3): Golub-Kahan bidiagonalization in the
                          inner product of M, one preconditioner apply per iteration,
                          the same stopping test on the true residual; 2 restarted
                          GMRES on C x = A^T b, right-preconditioned (flexible form),
                          restart length `restart`.  1 and 2: single problem, one
                          right-hand side; ls_backward always uses PCG.               */
    int restart;       /* GMRES restart length (default 100, as in Section 4)          */
    int spmv;          /* kernel of the products with A and A^T: 0 (the default) times
                          every candidate at setup and keeps the fastest for each;
                          otherwise one code for both: 1, 2, 4, 8, 16, 32 lanes per
                          row; -1 / -3 warp-stream (16 / 32 rows per warp); -2 sliced
                          ELL (LS_ERR_INVALID else).  ls_info.lanes_csr / lanes_csc
                          report the codes in use.                                    */
    int test_stall;    /* test hook, 0 (the default) in normal use: 1 makes the
                          local-solve kernels (single-vector and block) issue none of
                          their bulk copies, so every bounded wait for one gives up
                          (after about two seconds), the kernel sets the error slot and
                          returns with nothing in flight, and the solve returns
                          LS_ERR_DEVICE_TIMEOUT.  The CUDA context stays usable.      */
    int block_kernel;  /* local solve of the multi right-hand-side path with FP32 factors:
                          0 (the default) times both at the first block solve and keeps
                          the faster; 1 TF32 mma.sync tiles, left-looking sweeps; 2
                          tcgen05 MMAs (M = 128, accumulator in tensor memory),
                          right-looking sweeps (LS_ERR_UNSUPPORTED if the widest factor
                          block row does not fit its shared-memory window).  Both round
                          the factor to TF32.  ls_info.local_kernel reports the choice. */
    int normal_product;/* form of the product C v = A^T (A v): 0 (the default) times both
                          at setup and keeps the faster (the two products alone when
                          spmv forces a kernel, and on batched handles, whose solves
                          run the multi right-hand-side products); 1 two products,
                          q = A v then A^T q; 2
                          row tiles: A is cut into tiles of consecutive rows whose
                          entries fall in a narrow column window, each tile forms A v
                          for its rows and A^T of that for its window in shared memory
                          from one tile-local copy, and the windows are summed per
                          column in tile order (LS_ERR_UNSUPPORTED if one row's column
                          span does not fit the shared memory of a block).  Both are
                          bitwise repeatable.  ls_info.normal_product reports the form. */
    int normal_kernel; /* row tiles: kernel configuration, 1, 2 or 3: blocks of 512
                          threads whose warps take that many slices (of 32 rows or 32
                          columns) at a time (more loads in flight, more registers); 4:
                          blocks of 1,024 threads, one slice per warp; 0 (the default)
                          times the four at setup.  Same results for all.            */
    int local_config;  /* single-vector local solve: 1 blocks of 256 threads with 16 KB
                          stages, two per SM (many subdomains); 2 blocks of 512 threads
                          with 32 KB stages, one per SM (subdomains that each get an SM:
                          twice the warps, twice the columns per stage); 3 (FP32 factors)
                          each subdomain split over a cluster of 2 such blocks on two
                          SMs, which share its factor stream and exchange partial sums
                          and solution blocks through distributed shared memory (when
                          twice the subdomain count does not exceed the SM count); 0 (the
                          default) times those that fit at the end of setup and keeps
                          the fastest (1 without timing on batched handles, whose solves
                          run the multi right-hand-side path, and with test_stall);
                          LS_ERR_UNSUPPORTED when a forced one does not fit.
                          ls_info.local_config reports it.                             */
} ls_options;

typedef struct {
    int iters;               /* CG iterations of the last solve                            */
    int restarts;            /* restarts from the true residual                            */
    double relres_recursive; /* ||r_k|| / ||A^T b|| of the recursion at exit               */
    double relres_true;      /* ||A^T (b - A x)|| / ||A^T b|| recomputed at exit           */
    double kappa_lanczos;    /* condition estimate of M^{-1} C from the CG coefficients     */
    int n0;                  /* coarse dimension sum_i k_i                                  */
    int kmin, kmax;          /* fewest / most coarse vectors of one subdomain              */
    double tau_used;         /* the threshold tau actually applied                          */
    double delta;            /* the construction shift delta                                */
    double t_setup;          /* seconds: whole ls_setup                                     */
    double t_eig;            /* seconds: the local eigensolves                              */
    double t_solve;          /* seconds: the last ls_solve / ls_backward                    */
    int bad_subdomain;       /* subdomain of a factor / eigen failure, else -1              */
    int eig_steps_max;       /* most Lanczos steps one subdomain needed                     */
    double ms_local;         /* with time_kernels: total ms of the local-solve launches     */
    double ms_spmv;          /* with time_kernels: total ms of the A and A^T launches       */
    double ms_coarse;        /* with time_kernels: total ms of the coarse GEMV launches      */
    int local_launches;      /* local-solve launches of the last solve                      */
    int launches;            /* kernels launched by the last solve (all of this library's)  */
    double ms_iter;          /* with time_kernels: total ms of whole CG iterations (kernels) */
    int lanes_csr, lanes_csc;/* kernel codes of the products with A / A^T (option spmv)    */
    int local_kernel;        /* local-solve kernel of the last solve: 0 the single-vector or
                                CUDA-core block kernel, 1 TF32 mma.sync block kernel, 2
                                tcgen05 block kernel                                       */
    int normal_product;      /* form of the A^T (A v) products: 1 two products, 2 row tiles */
    int local_config;        /* configuration of the single-vector local solve (option)      */
} ls_info;

typedef struct ls_handle ls_handle;

/* Fill *opt with the defaults: nev_max = 16, delta_rel = 1e-10,
 * s_rel = 1e-8, factor_prec = LS_PREC_F64, maxit = 1000, coarse = 1,
 * fixed_iters = 0, eig_maxit = 3000, eig_tol = 1e-11, use_graph = 1, time_kernels = 0,
 * equilibrate = 0, variant = 0, solver = 0, restart = 100, spmv = 0, test_stall = 0,
 * block_kernel = 0, normal_product = 0, normal_kernel = 0, local_config = 0. */
void ls_default_options(ls_options* opt);

/* Build the preconditioner (Algorithm 1, whose inputs are A, the subdomain count N and
 * the threshold tau) for A given as CSR and a nonoverlapping column partition.
 *   m, n            rows and columns of A (m >= 1, n >= 1)
 *   row_ptr[m+1]    int64 CSR row offsets; col[nnz] int32; val[nnz] float64
 *   nparts          number N of subdomains (1 <= N <= n)
 *   part[n]         int32 subdomain id of every column (the sets Omega_I,i)
 *   overlap         must be 1 (Omega_Gamma,i = distance one in G(C), Section 2);
 *                   any other value returns LS_ERR_UNSUPPORTED
 *   tau             eigenvalue threshold of the coarse space: keep lambda > 1/tau
 *                   (Lemma 2.4, eq. (3.6)), at most opt->nev_max vectors per subdomain,
 *                   largest first.  tau <= 0 selects it automatically:
 *                   1/tau = max_i lambda_{i, nev_max+1}, so no subdomain keeps more than
 *                   nev_max vectors and the cap never truncates.  tau >= 1 returns
 *                   LS_ERR_UNSUPPORTED (it would keep the eigenvalue-1 cluster).
 *   opt             options (NULL: defaults)
 *   stream          cudaStream_t the handle runs its work on (NULL: the handle creates
 *                   its own non-blocking stream); setup is ordered after the work
 *                   already queued on it and has finished when the call returns
 *   out             receives the handle
 * The index sets are built on the host; local matrices, their Cholesky factors,
 * the eigensolves and the coarse operator are built on the device.  A and the
 * partition are copied: the caller may free them afterwards.
 * Errors: LS_ERR_INVALID (sizes, unsorted or out-of-range indices, part out of
 * range, non-finite values), LS_ERR_FACTOR (info via ls_handle_info), LS_ERR_EIGEN,
 * LS_ERR_OOM, LS_ERR_CUDA, LS_ERR_UNSUPPORTED. */
ls_status ls_setup(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col,
                   const double* val, int32_t nparts, const int32_t* part, int overlap,
                   double tau, const ls_options* opt, void* stream, ls_handle** out);

/* Batched setup: nprob independent least-squares problems in one handle, given as one
 * block-diagonal matrix (the "many problems share a launch" pattern).
 *   m_off[nprob+1], n_off[nprob+1]  host int64 offsets: problem q owns the rows
 *                   [m_off[q], m_off[q+1]) and the columns [n_off[q], n_off[q+1]);
 *                   a row may only touch the columns of its own problem
 *   row_ptr, col, val  the whole matrix in CSR (m = m_off[nprob], n = n_off[nprob])
 *   part[n]         subdomain ids; the ids of problem q form one range, in problem
 *                   order (problem 0 owns ids 0 .. N_1-1, problem 1 the next ones, ...)
 * Every problem is set up as if alone: its own delta = delta_rel ||C_q||_F, its own
 * automatic threshold (tau <= 0; tau > 0 applies to every problem) and its own dense
 * coarse block.  Other arguments and errors as ls_setup (LS_ERR_INVALID also for a row
 * or subdomain crossing problems). */
ls_status ls_setup_batched(int32_t nprob, const int64_t* m_off, const int64_t* n_off,
                           const int64_t* row_ptr, const int32_t* col, const double* val,
                           int32_t nparts, const int32_t* part, int overlap, double tau,
                           const ls_options* opt, void* stream, ls_handle** out);

/* Solve min ||A x - b|| for nrhs right-hand sides by PCG on C x = A^T b with x_0 = 0.
 *   b[m * nrhs]     column-major right-hand sides (host or device)
 *   rtol            stop when ||A^T (b - A x)|| <= rtol ||A^T b|| (true residual,
 *                   recomputed whenever the recursive residual passes the test; if
 *                   the true one fails, CG restarts from it)
 *   x[n * nrhs]     output, column-major (host or device)
 *   info            statistics (may be NULL)
 *   stream          the caller's cudaStream_t (NULL: the legacy default stream, as in
 *                   every CUDA API).  The call's device work starts after the work
 *                   already queued on `stream`, and work queued on `stream` after the
 *                   call is ordered after it.  The work itself runs on the handle's
 *                   stream (fixed at ls_setup: its CUDA graphs are captured there);
 *                   passing that stream adds nothing, another one adds an event
 *                   record and wait at entry and at exit.
 * One right-hand side on a single-problem handle runs the single-vector path.
 * Otherwise (nrhs in 1..32, or a batched handle) all right-hand sides and problems
 * advance together: every kernel of an iteration serves all of them, each (problem,
 * right-hand side) pair keeps its own CG scalars and stops on its own test (its
 * ||A_q^T b_q|| in the denominator), and info carries the largest iteration count and
 * true residual; the per-pair values are in ls_query(LS_Q_BATCH).
 * Errors: LS_ERR_NOT_CONVERGED (x holds the last iterate), LS_ERR_NONFINITE,
 * LS_ERR_UNSUPPORTED (nrhs > 32 on the multi right-hand-side path). */
ls_status ls_solve(ls_handle* h, const double* b, int nrhs, double rtol, double* x,
                   ls_info* info, void* stream);

/* Reverse mode of x(A, b) = C^{-1} A^T b.  With lambda = C^{-1} grad_x solved by the
 * same preconditioned CG to rtol:
 *   grad_b = A lambda                                   (m entries per right-hand side)
 *   grad_vals[k] = rho_r lambda_c - (A lambda)_r x_c    for CSR entry k = (r, c),
 *                  rho = b - A x                        (summed over right-hand sides)
 * b, x, grad_x are the forward inputs/outputs (column-major, host or device);
 * grad_b or grad_vals may be NULL to skip them.  On a batched handle the adjoint solves of
 * all (problem, right-hand side) pairs run together on the block path (nrhs <= 32), each
 * to its own test relative to its ||grad_x||; grad_vals is summed over the pairs.
 * stream: the caller's stream, ordered against as in ls_solve. */
ls_status ls_backward(ls_handle* h, const double* b, const double* x, const double* grad_x,
                      int nrhs, double rtol, double* grad_b, double* grad_vals, ls_info* info,
                      void* stream);

/* Replace the values of A (same pattern; val[nnz] in the caller's CSR order, host or
 * device) in the operator the solves apply; the preconditioner built by ls_setup is
 * kept as it is (it stays a valid SPD preconditioner; rebuild with ls_setup when the
 * values move far).  Used by finite-difference checks and optimization loops. */
ls_status ls_update_values(ls_handle* h, const double* val);

/* Release everything the handle owns.  NULL is ignored. */
void ls_free(ls_handle* h);

/* Message of the last failing call on this thread ("" if none). */
const char* ls_last_error(void);

/* Setup statistics (n0, k range, tau, delta, times, failing subdomain). */
ls_status ls_handle_info(const ls_handle* h, ls_info* info);

/* ---- inspection calls used by tests and benchmarks ------------------------------ */

/* z = M^{-1} r for one vector (host or device pointers, n entries each); which = 0:
 * the full two-level operator (additive or balanced, as ls_options.variant selects),
 * 1: the local sum only, 2: the coarse term Q r only.
 * Batched handles: LS_ERR_UNSUPPORTED. */
ls_status ls_apply_preconditioner(ls_handle* h, const double* r, double* z, int which);

/* w = A^T (A p) for one vector (host or device pointers, n entries each). */
ls_status ls_apply_normal(ls_handle* h, const double* p, double* w);

typedef enum {
    LS_Q_SIZES = 0,    /* int64[N*4]: n_i, n_I,i, |Xi_i|, k_i per subdomain          */
    LS_Q_OMEGA = 1,    /* int32[n_i]: Omega_i of subdomain i in [Omega_I, Omega_Gamma] order */
    LS_Q_XI = 2,       /* int32[|Xi_i|]: Xi_i of subdomain i, ascending             */
    LS_Q_EIGVALS = 3,  /* float64[k_want]: the computed top eigenvalues of subdomain i,
                          descending (k_want = min(nev_max + 1, n_i))               */
    LS_Q_ZBAR = 4,     /* float64[k_i * n_I,i]: coarse basis of subdomain i, one
                          vector after another, over Omega_I,i ascending            */
    LS_Q_EIGSTEPS = 5, /* int32[N]: Lanczos steps per subdomain                     */
    LS_Q_STORAGE = 6,  /* int64[8]: factor elements (all subdomains), sum n_i, block
                          rows, coarse-basis elements, n0, padded n0, nnz(A), factor
                          precision (ls_precision)                                  */
    LS_Q_BATCH = 7,    /* float64[2 * nprob * nrhs] of the last multi right-hand-side
                          solve: iterations, then true relative residuals, each
                          indexed [problem * nrhs + rhs]                              */
    LS_Q_NORMAL = 8    /* int64[12]: the row tiles of the normal product (the first seven
                          0 when the two-product form runs): tiles, stored entries of
                          the row copy and of the column copy (padding included), row
                          slices, column slices, sum of the window widths, kernel
                          configuration (option normal_kernel); then the setup timings
                          behind the choice in ns per product (0: not timed): the two
                          products, then configurations 1 to 4                       */
} ls_query_kind;

/* Copy one inspected array to the host buffer out (capacity cap elements of the
 * kind's type).  Returns LS_ERR_INVALID if i is out of range or cap is too small. */
ls_status ls_query(const ls_handle* h, int kind, int i, void* out, int64_t cap);

/* Host-only construction of the index sets of Section 3 (no GPU needed).
 *   Outputs (caller-allocated, sizes from a first call with NULL outputs):
 *   omega_off[N+1], omega[sum n_i]   Omega_i in [Omega_I, Omega_Gamma] order
 *   n_interior[N]                    n_I,i
 *   xi_off[N+1], xi[sum |Xi_i|]      Xi_i ascending
 * Call with omega == NULL to receive the totals in *omega_total and *xi_total. */
ls_status ls_build_index_sets(int64_t m, int64_t n, const int64_t* row_ptr,
                              const int32_t* col, int32_t nparts, const int32_t* part,
                              int64_t* omega_total, int64_t* xi_total, int64_t* omega_off,
                              int32_t* omega, int32_t* n_interior, int64_t* xi_off,
                              int32_t* xi);

/* ---- allocation-free entry point ------------------------------------------------ */

/* w = A^T (A p) without any allocation by the library.  The paper has no counterpart:
 * this is for callers that cannot call cudaMalloc -- code whose device memory must all
 * come from a framework's own pool or from a fixed budget set aside at start-up, and
 * real-time loops that must stay out of the CUDA memory allocator (cudaMalloc and
 * cudaFree can synchronise the device and take an unbounded time).
 *   m, n, nnz        sizes of A (1 <= m <= 8,388,608; n >= 1)
 *   row_ptr, col, val        A in CSR (device memory: int64[m+1], int32[nnz], f64[nnz])
 *   col_ptr, row, cval       A in CSC (device memory: int64[n+1], int32[nnz], f64[nnz]),
 *                            rows ascending within each column
 *   p (f64[n], device)       input;  w (f64[n], device) output
 *   stream                   cudaStream_t to launch on (NULL: the legacy default stream)
 * The intermediate q = A p lives in one fixed file-scope device array of 8,388,608
 * doubles (64 MB) per GPU; larger m returns LS_ERR_INVALID.  The array belongs to this
 * library's module for that source file and is reserved when the module loads into a
 * CUDA context: at the first call on that device under lazy module loading (the CUDA
 * default), at context creation under CUDA_MODULE_LOADING=EAGER, for every process
 * that loads the library; it is held until the context is destroyed or the process
 * exits.  The first call in a context looks up the array's device address (once per
 * device and context, with that device current; a context made after cudaDeviceReset
 * gets its own lookup): make that first call before any stream capture.  All calls
 * share the array and it keeps the last call's contents: calls whose work can overlap
 * on the GPU (other streams, other threads) race and must be ordered by the caller.
 * The call is asynchronous on `stream`; the library checks only sizes and NULL
 * pointers (the Python binding also checks dtypes, lengths and devices); a pointer of
 * the wrong kind or length is read or written out of bounds on the device.  Errors:
 * LS_ERR_INVALID, LS_ERR_CUDA (also when an error from earlier work is already pending
 * on this thread: it is reported, not cleared).  Messages: ls_noalloc_last_error(). */
ls_status ls_normal_product_noalloc(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col,
                                    const double* val, const int64_t* col_ptr, const int32_t* row,
                                    const double* cval, int64_t nnz, const double* p, double* w,
                                    void* stream);

/* Message of the last failing ls_normal_product_noalloc on this thread ("" if none). */
const char* ls_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LS_SCHWARZ_H */
