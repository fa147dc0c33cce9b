// The C ABI (include/ls_schwarz.h): handle, setup orchestration (Algorithm 1 of
// arXiv 2107.09006 on the device), the PCG solve loop with optional CUDA-graph
// replay of each iteration, the adjoint solve and the inspection calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ls_schwarz.h"
#include "host_sets.h"
#include "normal_tiles.h"
#include "kernels.h"

namespace {

thread_local std::string g_err;



// data[e] *= scale[idx[e]]
__global__ void k_scale_by_gather(int64_t n, const int32_t* idx, const double* scale, double* data) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    data[e] *= scale[idx[e]];
}

// Zbar_i[t, jj] *= scale[interior column jj of subdomain i]  (one block per subdomain)
__global__ void k_scale_zbar(const int32_t* coff, const int64_t* zoff, const int64_t* int_off,
                             const int32_t* int_glob, const double* scale, double* Z) {
  const int i = blockIdx.x;
  const int k = coff[i + 1] - coff[i];
  const int64_t io = int_off[i], nI = int_off[i + 1] - io;
  for (int64_t e = threadIdx.x; e < (int64_t)k * nI; e += blockDim.x) Z[zoff[i] + e] *= scale[int_glob[io + e % nI]];
}

__global__ void k_set_diag(double* A, int64_t ld, int64_t from, int64_t to, double v) {
  for (int64_t k = from + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < to; k += (int64_t)gridDim.x * blockDim.x)
    A[k * ld + k] = v;
}

int pow2_lanes(double avg) {
  int v = 1;
  while (v < 32 && v < avg) v <<= 1;
  return v;
}

// Extreme eigenvalues of a symmetric tridiagonal matrix by Sturm bisection.
double tridiag_extreme(const std::vector<double>& d, const std::vector<double>& e, bool largest) {
  const int k = (int)d.size();
  double lo = 1e300, hi = -1e300;
  for (int j = 0; j < k; ++j) {
    const double r = (j > 0 ? std::fabs(e[j - 1]) : 0.0) + (j + 1 < k ? std::fabs(e[j]) : 0.0);
    lo = std::min(lo, d[j] - r);
    hi = std::max(hi, d[j] + r);
  }
  auto count_below = [&](double x) {
    int c = 0;
    double q = 1.0;
    for (int j = 0; j < k; ++j) {
      const double ee = j > 0 ? e[j - 1] : 0.0;
      q = d[j] - x - (j > 0 ? ee * ee / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0) ++c;
    }
    return c;
  };
  const int target = largest ? k - 1 : 0;  // index of the wanted eigenvalue
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count_below(mid) > target) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace


#include "handle.h"

using namespace lsi;

namespace {

lsq::DotSite site(ls_handle* h, int slot, int counter, int out2 = 0) {
  return lsq::DotSite{h->parts.p, lsq::kMaxGrid, h->counters.p + counter, h->scal.p + slot, out2};
}


bool balanced(const ls_handle* h) { return h->opt.variant == 1 && h->coarse && h->n0 > 0; }

// Timing mark k of an iteration: an event record, or a global-timer stamp while the
// device-side loop's body is being captured.
void mark(ls_handle* h, int k) {
  if (h->stamping) lsq::launch_stamp(h->stamps.p, h->ctr.p, h->hist_cap, k, k == 5 ? 1 : 0, h->st);
  else record_event(h->ev[k], h->st);
}

// y = local solves of rin (and, with_coarse, the fused coarse restriction r0 = R_0 rin)
void launch_local(ls_handle* h, const double* rin, bool with_coarse) {
  lsq::LocalArgs a{};
  a.om_off = h->om_off.p; a.om_glob = h->om_glob.p; a.eqs = h->eqs.p;
  a.blk_off = h->blk_off.p; a.blk_tf = h->blk_tf.p; a.blk_poff = h->blk_poff.p;
  a.fac = h->prec == LS_PREC_F64 ? (const void*)h->L64.p
        : h->prec == LS_PREC_F32 ? (const void*)h->L32.p : (const void*)h->L16.p;
  a.tsc = h->prec == LS_PREC_BF16 ? h->tsc.p : nullptr;
  a.err = h->scal.p + lsq::S_ERR;
  a.r = rin; a.y = h->ybuf.p;
  a.coarse = with_coarse ? 1 : 0;
  a.int_off = h->int_off.p; a.int_glob = h->int_glob.p; a.zoff = h->zoff.p; a.coff = h->coff.p;
  a.Z = h->Z.p; a.r0 = h->r0.p;
  a.stall = h->opt.test_stall;
  a.n_cols = h->n; a.fac_elems = h->fac_elems;
  if (h->local_cfg == 3) {
    if (!lsq::local_split_launch(h->N, h->max_nb, a, h->st))
      throw LsError(LS_ERR_CUDA, std::string("local solve (cluster launch): ") + cudaGetErrorString(cudaGetLastError()));
    return;
  }
  lsq::launch_local_solve(h->prec, h->local_cfg, h->N, h->max_nb, a, h->st);
}

// The local-solve configuration: forced by the option, else the candidates that fit
// timed on the factors (two launches each after a warm one).  Configuration 3 (FP32
// factors only) splits each subdomain over a cluster of CTAs; it is a candidate when
// every CTA of every cluster can have an SM of its own.
void choose_local_config(ls_handle* h, int optin) {
  h->local_cfg = 1;
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->dev));
  const bool fits[4] = {false, true, lsq::local_solve_smem(h->prec, h->max_nb, 2) <= (size_t)optin,
                        h->prec == LS_PREC_F32 && lsq::local_split_smem(h->max_nb) <= (size_t)optin &&
                            (int64_t)h->N * lsq::local_split_cluster() <= sms};
  if (h->opt.local_config != 0) {
    if (!fits[h->opt.local_config])
      throw LsError(LS_ERR_UNSUPPORTED, "local_config = " + std::to_string(h->opt.local_config) +
                                            ": not available for this factor precision, subdomain count or size");
    h->local_cfg = h->opt.local_config;
    return;
  }
  if (h->opt.test_stall || h->nprob > 1) return;  // (batched handles solve through the block path)
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int pick = 1;
  for (int cfg = 1; cfg <= 3; ++cfg) {
    if (!fits[cfg]) continue;
    h->local_cfg = cfg;
    try {
      launch_local(h, h->r.p, false);
    } catch (const LsError&) {
      cudaGetLastError();  // a refused cluster launch: the configuration is not a candidate
      continue;
    }
    CK(cudaEventRecord(e0, h->st));
    for (int k = 0; k < 2; ++k) launch_local(h, h->r.p, false);
    CK(cudaEventRecord(e1, h->st));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) { best = ms; pick = cfg; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  check_launch("local-solve configuration timing");
  h->local_cfg = pick;
}

// out = Q v = R_0^T C_00^{-1} R_0 v (restriction, dense coarse solve, prolongation)
void coarse_term(ls_handle* h, const double* v, double* out) {
  cudaStream_t st = h->st;
  lsq::launch_restrict(h->N, h->int_off.p, h->int_glob.p, h->zoff.p, h->coff.p, h->Z.p, v, h->r0.p, st);
  lsq::launch_gemv(h->n0p, h->Xinv.p, h->r0.p, h->y0.p, st);
  lsq::ScatterArgs s{};
  s.n = h->n; s.map_ptr = h->map_ptr.p; s.map_idx = h->map_idx.p; s.y = h->ybuf.p;
  s.total_local = h->total_local; s.err = h->scal.p + lsq::S_ERR;
  s.coarse = 1; s.part = h->part.p; s.jj_of = h->jj_of.p; s.zoff = h->zoff.p;
  s.coff = h->coff.p; s.nI = h->nI.p; s.Z = h->Z.p; s.y0 = h->y0.p;
  s.z = out;
  s.add_coarse_only = 1;
  lsq::launch_scatter(s, st);
}

// out = A^T (A v) in the form chosen at setup (two products, or the row tiles), with the
// fused d . out into ds when ds.parts is set.
void normal_product(ls_handle* h, const double* v, double* out, const double* d, const lsq::DotSite& ds,
                    cudaStream_t st) {
  if (h->normal_kind == 2) {
    lsq::launch_normal_tiles(ntiles(h), v, out, d, ds, st);
    return;
  }
  lsq::launch_spmv_csr(csr(h), v, h->q.p, h->lanes_csr, h->grid_csr, st);
  lsq::launch_spmv_csc(csc(h), h->q.p, out, d, ds, h->lanes_csc, h->grid_csc, st);
}

// out = C v = A^T (A v)
void apply_C(ls_handle* h, const double* v, double* out) {
  normal_product(h, v, out, nullptr, lsq::DotSite{}, h->st);
}

// Kernels of one apply of the balanced operator (see precond_balanced).
constexpr int kBalancedLaunches = 14;

// z = Q r + (I - Q C) M_1 (I - C Q) r (the balanced two-level operator of Section 2)
// with the fused dots r.z (and r_old.z).
void precond_balanced(ls_handle* h, const double* rin, double* zout, bool dots, bool flex, bool timed) {
  cudaStream_t st = h->st;
  coarse_term(h, rin, h->bal_y.p);                                     // Q r
  apply_C(h, h->bal_y.p, h->bal_t.p);                                  // C Q r
  lsq::launch_axpby(h->n, 1.0, rin, -1.0, h->bal_t.p, h->bal_t.p, st);  // t = (I - CQ) r
  if (timed) mark(h, 2);
  launch_local(h, h->bal_t.p, false);
  if (timed) mark(h, 3);
  lsq::ScatterArgs s{};
  s.n = h->n; s.map_ptr = h->map_ptr.p; s.map_idx = h->map_idx.p; s.y = h->ybuf.p;
  s.total_local = h->total_local; s.err = h->scal.p + lsq::S_ERR;
  s.z = h->bal_u.p;
  s.add_coarse_only = 2;
  lsq::launch_scatter(s, st);                                          // u = M_1 t
  apply_C(h, h->bal_u.p, h->bal_t.p);                                  // C u
  coarse_term(h, h->bal_t.p, h->bal_v.p);                              // Q C u
  if (timed) mark(h, 4);
  lsq::launch_combine3(h->n, h->bal_y.p, h->bal_u.p, h->bal_v.p, zout, rin, flex ? h->r_old.p : nullptr,
                       dots ? site(h, lsq::S_RZ, 2, lsq::S_RZO - lsq::S_RZ) : lsq::DotSite{}, st);
}

// z = Q r + M_RAS (I - C Q) r (the deflated second level of Section 2 with the RAS first
// level; without a coarse space, z = M_RAS r).  No fused dots: only GMRES uses it.
void precond_deflated(ls_handle* h, const double* rin, double* zout, bool timed) {
  cudaStream_t st = h->st;
  const bool coarse = h->coarse && h->n0 > 0;
  const double* t = rin;
  if (coarse) {
    coarse_term(h, rin, h->bal_y.p);                                     // Q r
    apply_C(h, h->bal_y.p, h->bal_t.p);                                  // C Q r
    lsq::launch_axpby(h->n, 1.0, rin, -1.0, h->bal_t.p, h->bal_t.p, st);  // (I - CQ) r
    t = h->bal_t.p;
  }
  if (timed) mark(h, 2);
  launch_local(h, t, false);
  if (timed) mark(h, 3);
  lsq::launch_ras_combine(h->n, h->own.p, h->ybuf.p, coarse ? h->bal_y.p : nullptr, zout, st);
  if (timed) mark(h, 4);
}

int deflated_launches(const ls_handle* h) { return 2 + ((h->coarse && h->n0 > 0) ? 6 : 0); }

// z = M^{-1} r (which: 0 both terms, 1 local only, 2 coarse only) with the fused dots
// r.z (and r_old.z for the flexible recurrence) into the partial arrays.
void precond(ls_handle* h, const double* rin, double* zout, int which, bool dots, bool flex, bool timed = false) {
  cudaStream_t st = h->st;
  if (which == 0 && h->opt.variant == 2) {
    precond_deflated(h, rin, zout, timed);
    return;
  }
  if (which == 0 && balanced(h)) {
    precond_balanced(h, rin, zout, dots, flex, timed);
    return;
  }
  if (which != 0 && which != 1) throw LsError(LS_ERR_INVALID, "precond: which must be 0 or 1");
  if (timed) mark(h, 2);
  const bool use_coarse = h->coarse && h->n0 > 0 && which != 1;
  if (which != 2) launch_local(h, rin, use_coarse);
  if (timed) mark(h, 3);
  if (use_coarse) lsq::launch_gemv(h->n0p, h->Xinv.p, h->r0.p, h->y0.p, st);
  if (timed) mark(h, 4);
  lsq::ScatterArgs s{};
  s.n = h->n; s.map_ptr = h->map_ptr.p; s.map_idx = h->map_idx.p; s.y = h->ybuf.p;
  s.total_local = h->total_local; s.err = h->scal.p + lsq::S_ERR;
  s.coarse = use_coarse ? 1 : 0; s.part = h->part.p; s.jj_of = h->jj_of.p; s.zoff = h->zoff.p;
  s.coff = h->coff.p; s.nI = h->nI.p; s.Z = h->Z.p; s.y0 = h->y0.p;
  s.r = rin; s.r_old = flex ? h->r_old.p : nullptr; s.z = zout;
  s.dots = dots ? site(h, lsq::S_RZ, 2, lsq::S_RZO - lsq::S_RZ) : lsq::DotSite{};
  s.add_coarse_only = which == 2 ? 1 : 0;
  lsq::launch_scatter(s, st);
}

// One PCG iteration: w = A^T (A p), alpha, x, r, z = M^{-1} r, beta, p.
// Kernels one iteration launches (for the launch count reported in ls_info).
int iteration_launches(const ls_handle* h) {
  if (balanced(h)) return 4 + kBalancedLaunches;
  return 6 + ((h->coarse && h->n0 > 0) ? 1 : 0);
}

void iteration(ls_handle* h, bool flex, bool copy_scalars = true) {
  cudaStream_t st = h->st;
  const bool timed = h->opt.time_kernels != 0;
  if (timed) mark(h, 0);
  normal_product(h, h->p.p, h->w.p, h->p.p, site(h, lsq::S_PW, 0), st);
  if (timed) mark(h, 1);
  lsq::launch_cg_update(h->n, h->scal.p, h->p.p, h->w.p, h->x.p, h->r.p, flex ? h->r_old.p : nullptr,
                        site(h, lsq::S_RR, 1), h->ctr.p, h->ahist.p, h->hist_cap, st);
  precond(h, h->r.p, h->z.p, 0, true, flex, timed);
  lsq::launch_p_update(h->n, h->scal.p, h->ctr.p, h->bhist.p, h->hist_cap, h->z.p, h->p.p, 0, flex ? 1 : 0, st);
  if (timed) mark(h, 5);
  if (copy_scalars) CK(cudaMemcpyAsync(h->pin, h->scal.p, sizeof(double) * lsq::S_NSLOT, cudaMemcpyDeviceToHost, st));
}

// Builds h->gloop: while (loop test) { one PCG iteration }, then the scalar slots to the
// host.  The body is captured from the same launch sequence as iteration(); the loop test
// kernel sets the while condition from the device scalars, so the host waits once per
// pass of the loop instead of once per iteration.  Returns false (and leaves gloop null)
// when the graph cannot be built, e.g. on a driver without conditional nodes.
bool build_loop_graph(ls_handle* h, bool flex, int limit) {
  cudaStream_t st = h->st;
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return false;
  bool ok = false;
  do {
    cudaGraphConditionalHandle hnd;
    if (cudaGraphConditionalHandleCreate(&hnd, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) break;
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hnd;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t wnode;
    if (cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &np) != cudaSuccess) break;
    cudaGraph_t body = np.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      break;
    h->stamping = h->opt.time_kernels != 0;
    iteration(h, flex, false);
    lsq::launch_cg_continue(h->scal.p, h->ctr.p, limit, hnd, st);
    h->stamping = false;
    cudaGraph_t captured = nullptr;
    if (cudaStreamEndCapture(st, &captured) != cudaSuccess) break;
    size_t nnodes = 0;
    if (cudaGraphGetNodes(body, nullptr, &nnodes) != cudaSuccess) break;
    cudaGraphNode_t cnode;
    if (cudaGraphAddMemcpyNode1D(&cnode, g, &wnode, 1, h->pin, h->scal.p, sizeof(double) * lsq::S_NSLOT,
                                 cudaMemcpyDeviceToHost) != cudaSuccess)
      break;
    if (cudaGraphInstantiate(&h->gloop, g, 0) != cudaSuccess) {
      h->gloop = nullptr;
      break;
    }
    h->loop_kernels = (int)nnodes;
    ok = true;
  } while (false);
  h->stamping = false;
  cudaGraphDestroy(g);
  if (!ok) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(st, &junk);
      if (junk) cudaGraphDestroy(junk);
    }
    cudaGetLastError();
  }
  return ok;
}

// Reads one scalar slot of the device CG state (synchronising the stream).
double dev_sum(ls_handle* h, int slot = lsq::S_TMP) {
  double v = 0;
  CK(cudaMemcpyAsync(&v, h->scal.p + slot, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return v;
}

// ||g - C x||^2 into the host: mode 0 as ||A^T (b - A x)||^2, mode 1 as ||g - A^T (A x)||^2.
// Leaves the residual vector in h->w; adds the kernels it launched to *launches.
double true_residual(ls_handle* h, int mode, int* launches) {
  Phase phase("true residual");
  cudaStream_t st = h->st;
  lsq::launch_spmv_csr(csr(h), h->x.p, h->q.p, h->lanes_csr, h->grid_csr, st);
  if (mode == 0) {
    lsq::launch_axpby(h->m, 1.0, h->bv.p, -1.0, h->q.p, h->q.p, st);
    lsq::launch_spmv_csc(csc(h), h->q.p, h->w.p, nullptr, site(h, lsq::S_TMP, 0), h->lanes_csc, h->grid_csc, st);
    *launches += 3;
  } else {
    lsq::launch_spmv_csc(csc(h), h->q.p, h->w.p, nullptr, lsq::DotSite{}, h->lanes_csc, h->grid_csc, st);
    lsq::launch_axpby(h->n, 1.0, h->tv.p, -1.0, h->w.p, h->w.p, st);
    lsq::launch_dot(h->n, h->w.p, h->w.p, site(h, lsq::S_TMP, 3), st);
    *launches += 4;
  }
  return dev_sum(h);
}

// PCG on C x = g.  mode 0: g = A^T b with b in h->bv (true residual A^T (b - A x));
// mode 1: g given in h->tv (true residual g - A^T A x).  Result in h->x.
ls_status solve_core(ls_handle* h, int mode, double rtol, ls_info* info) {
  cudaStream_t st = h->st;
  const int64_t n = h->n;
  const bool flex = h->prec != LS_PREC_F64;
  const double t0 = now_s();
  ls_info inf{};
  inf.bad_subdomain = -1;
  int launches = 0;
  // r = g, gg = ||g||^2
  if (mode == 0) {
    lsq::launch_spmv_csc(csc(h), h->bv.p, h->r.p, nullptr, site(h, lsq::S_TMP, 0), h->lanes_csc, h->grid_csc, st);
  } else {
    CK(cudaMemcpyAsync(h->r.p, h->tv.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    lsq::launch_dot(n, h->r.p, h->r.p, site(h, lsq::S_TMP, 3), st);
  }
  const double gg = dev_sum(h);
  launches += 1;
  if (!std::isfinite(gg)) throw LsError(LS_ERR_NONFINITE, "right-hand side is not finite");
  const double gn = std::sqrt(gg);
  lsq::launch_fill(n, 0.0, h->x.p, st);
  launches += 1;
  CK(cudaMemsetAsync(h->ctr.p, 0, sizeof(int), st));
  CK(cudaMemsetAsync(h->scal.p, 0, sizeof(double) * lsq::S_NSLOT, st));
  if (gn == 0.0) {
    CK(cudaStreamSynchronize(st));
    inf.t_solve = now_s() - t0;
    inf.launches = launches;
    if (info) *info = inf;
    return LS_OK;
  }
  auto restart = [&]() {
    precond(h, h->r.p, h->z.p, 0, true, false);
    lsq::launch_p_update(n, h->scal.p, h->ctr.p, h->bhist.p, h->hist_cap, h->z.p, h->p.p, 1, 0, st);
    launches += iteration_launches(h) - 3;
    inf.local_launches += 1;
  };
  restart();
  check_launch("initial preconditioner apply");
  const int fixed = h->opt.fixed_iters;
  const int maxit = fixed > 0 ? fixed : h->opt.maxit;
  const bool timed = h->opt.time_kernels != 0;
  bool converged = false;
  int it = 0, restarts = 0;
  double rr = gg;
  bool graph_this = h->opt.use_graph != 0;
  bool loop_this = graph_this;
  // the device-side loop's test: (rtol ||g||)^2 on the recursive residual (none with
  // fixed_iters); the host applies the same test to the same double
  const double thr2 = (rtol * gn) * (rtol * gn);
  lsq::launch_fill(1, fixed > 0 ? 0.0 : thr2, h->scal.p + lsq::S_THR, st);
  launches += 1;
  while (it < maxit) {
    int done_now = 1;  // iterations this pass ran
    if (loop_this) {
      if (!h->gloop) {  // built once per handle: the loop only touches fixed buffers
        if (timed && !h->stamps.p) h->stamps.alloc((size_t)h->hist_cap * 8);
        if (!build_loop_graph(h, flex, maxit)) {
          loop_this = false;
          continue;
        }
      }
      {
        Phase phase("PCG loop pass (device-side while graph)");
        CK(cudaGraphLaunch(h->gloop, st));
        CK(cudaStreamSynchronize(st));
      }
      check_launch("CG loop");
      done_now = (int)h->pin[lsq::S_ITS] - it;
      if (done_now < 1) throw LsError(LS_ERR_CUDA, "the device-side CG loop ran no iteration");
      launches += done_now * h->loop_kernels;
      if (timed) {
        std::vector<unsigned long long> tsm((size_t)done_now * 8);
        const int first = std::min(it, h->hist_cap);
        const int cnt = std::max(0, std::min(it + done_now, h->hist_cap) - first);
        if (cnt > 0) {
          CK(cudaMemcpy(tsm.data(), h->stamps.p + (size_t)first * 8, sizeof(unsigned long long) * 8 * cnt,
                        cudaMemcpyDeviceToHost));
          for (int j = 0; j < cnt; ++j) {
            const unsigned long long* t = tsm.data() + (size_t)j * 8;
            inf.ms_spmv += (t[1] - t[0]) * 1e-6;
            inf.ms_local += (t[3] - t[2]) * 1e-6;
            inf.ms_coarse += (t[4] - t[3]) * 1e-6;
            inf.ms_iter += (t[5] - t[0]) * 1e-6;
          }
        }
      }
    } else {
      if (graph_this) {
        if (!h->gexec) {  // built once per handle: the iteration only touches fixed buffers
          cudaGraph_t g;
          CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
          iteration(h, flex);
          CK(cudaStreamEndCapture(st, &g));
          cudaError_t e = cudaGraphInstantiate(&h->gexec, g, 0);
          cudaGraphDestroy(g);
          if (e != cudaSuccess) {
            h->gexec = nullptr;
            cudaGetLastError();
            graph_this = false;
            continue;
          }
        }
        CK(cudaGraphLaunch(h->gexec, st));
      } else {
        iteration(h, flex);
      }
      CK(cudaStreamSynchronize(st));
      check_launch("CG iteration");
      launches += iteration_launches(h);
      if (timed) {
        float a = 0.f, b = 0.f, c = 0.f;
        CK(cudaEventElapsedTime(&a, h->ev[0], h->ev[1]));
        CK(cudaEventElapsedTime(&b, h->ev[2], h->ev[3]));
        CK(cudaEventElapsedTime(&c, h->ev[3], h->ev[4]));
        inf.ms_spmv += a;
        inf.ms_local += b;
        inf.ms_coarse += c;
        float d = 0.f;
        CK(cudaEventElapsedTime(&d, h->ev[0], h->ev[5]));
        inf.ms_iter += d;
      }
    }
    it += done_now;
    inf.local_launches += done_now;
    rr = h->pin[lsq::S_RR];
    if (h->pin[lsq::S_ERR] == lsq::kErrBounds)
      throw LsError(LS_ERR_INVALID, "an index out of range was met (bounds-checked build) at iteration " +
                                        std::to_string(it));
    if (h->pin[lsq::S_ERR] != 0.0)
      throw LsError(LS_ERR_DEVICE_TIMEOUT, "a bounded wait in the local-solve kernel gave up at iteration " +
                                               std::to_string(it));
    if (h->pin[lsq::S_FLAG] != 0.0 || !std::isfinite(rr))
      throw LsError(LS_ERR_NONFINITE, "CG breakdown: non-finite or non-positive p.Cp at iteration " + std::to_string(it));
    if (fixed > 0) continue;
    if (rr <= thr2) {
      const double tt = true_residual(h, mode, &launches);
      inf.relres_true = std::sqrt(tt) / gn;
      if (std::sqrt(tt) <= rtol * gn) { converged = true; break; }
      CK(cudaMemcpyAsync(h->r.p, h->w.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
      ++restarts;
      restart();
    }
  }
  // final statistics
  inf.iters = it;
  inf.restarts = restarts;
  inf.relres_recursive = std::sqrt(rr) / gn;
  if (!converged) inf.relres_true = std::sqrt(true_residual(h, mode, &launches)) / gn;
  inf.kappa_lanczos = 0.0;
  const int nh = std::min(it, h->hist_cap);
  if (restarts == 0 && nh > 0) {
    std::vector<double> al(nh), be(nh);
    CK(cudaMemcpyAsync(al.data(), h->ahist.p, sizeof(double) * nh, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(be.data(), h->bhist.p, sizeof(double) * nh, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::vector<double> d(nh), e(std::max(nh - 1, 0));
    for (int j = 0; j < nh; ++j) {
      d[j] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
      if (j + 1 < nh) e[j] = std::sqrt(std::max(be[j], 0.0)) / al[j];
    }
    const double lmax = tridiag_extreme(d, e, true), lmin = tridiag_extreme(d, e, false);
    inf.kappa_lanczos = lmin > 0 ? lmax / lmin : 0.0;
  }
  inf.n0 = h->sinfo.n0; inf.kmin = h->sinfo.kmin; inf.kmax = h->sinfo.kmax; inf.tau_used = h->sinfo.tau_used;
  inf.delta = h->sinfo.delta; inf.t_setup = h->sinfo.t_setup; inf.t_eig = h->sinfo.t_eig;
  inf.bad_subdomain = -1; inf.eig_steps_max = h->sinfo.eig_steps_max;
  inf.launches = launches;
  inf.lanes_csr = h->lanes_csr; inf.lanes_csc = h->lanes_csc; inf.normal_product = h->normal_kind; inf.local_config = h->local_cfg;
  inf.t_solve = now_s() - t0;
  if (info) *info = inf;
  if (!converged && fixed <= 0)
    return (g_err = "maximum number of iterations reached, true relative residual " +
                    std::to_string(inf.relres_true), LS_ERR_NOT_CONVERGED);
  return LS_OK;
}

// Preconditioned LSQR on min ||A' x - b'|| (b' in h->bv, result in h->x): Golub-Kahan
// bidiagonalization between R^m and R^n with the inner product of M, so the adjoint of
// A is M^{-1} A^T and each step applies the preconditioner once (Section 4.1.3 uses
// left-preconditioned LSQR); the plane-rotation recurrences run on the host, the vector
// work on the device.  Stopping: the true residual test ||A^T (b - A x)|| <= rtol ||A^T b||,
// evaluated from the first step at which LSQR's estimate of ||M^{-1} A^T r||_M has
// fallen below 10 rtol times its initial value.
ls_status lsqr_core(ls_handle* h, double rtol, ls_info* info) {
  cudaStream_t st = h->st;
  const int64_t n = h->n, m = h->m;
  const double t0 = now_s();
  ls_info inf{};
  inf.bad_subdomain = -1;
  int launches = 0;
  lsq::launch_spmv_csc(csc(h), h->bv.p, h->r.p, nullptr, site(h, lsq::S_TMP, 0), h->lanes_csc, h->grid_csc, st);
  const double gg = dev_sum(h);
  lsq::launch_dot(m, h->bv.p, h->bv.p, site(h, lsq::S_TMP, 3), st);
  const double bb = dev_sum(h);
  launches += 2;
  if (!std::isfinite(gg) || !std::isfinite(bb)) throw LsError(LS_ERR_NONFINITE, "right-hand side is not finite");
  const double gn = std::sqrt(gg);
  lsq::launch_fill(n, 0.0, h->x.p, st);
  launches += 1;
  CK(cudaMemsetAsync(h->scal.p, 0, sizeof(double) * lsq::S_NSLOT, st));
  auto finish = [&](int it, bool converged, double rel) -> ls_status {
    inf.iters = it;
    inf.relres_true = rel;
    inf.relres_recursive = rel;
    inf.n0 = h->sinfo.n0; inf.kmin = h->sinfo.kmin; inf.kmax = h->sinfo.kmax; inf.tau_used = h->sinfo.tau_used;
    inf.delta = h->sinfo.delta; inf.t_setup = h->sinfo.t_setup; inf.t_eig = h->sinfo.t_eig;
    inf.eig_steps_max = h->sinfo.eig_steps_max;
    inf.launches = launches;
    inf.lanes_csr = h->lanes_csr; inf.lanes_csc = h->lanes_csc; inf.normal_product = h->normal_kind; inf.local_config = h->local_cfg;
    inf.t_solve = now_s() - t0;
    if (info) *info = inf;
    if (!converged && h->opt.fixed_iters <= 0)
      return (g_err = "maximum number of iterations reached, true relative residual " + std::to_string(rel),
              LS_ERR_NOT_CONVERGED);
    return LS_OK;
  };
  if (gn == 0.0 || bb == 0.0) {
    CK(cudaStreamSynchronize(st));
    return finish(0, true, 0.0);
  }
  const bool timed = h->opt.time_kernels != 0;
  const int pl = balanced(h) ? kBalancedLaunches : 2 + ((h->coarse && h->n0 > 0) ? 1 : 0);
  // u = b / beta, s = A^T u, t = M^{-1} s, alpha = (s.t)^{1/2}, v = t / alpha, q = s / alpha, w = v
  double beta = std::sqrt(bb);
  lsq::launch_axpby(m, 1.0 / beta, h->bv.p, 0.0, nullptr, h->lq_u.p, st);
  lsq::launch_spmv_csc(csc(h), h->lq_u.p, h->lq_s.p, nullptr, lsq::DotSite{}, h->lanes_csc, h->grid_csc, st);
  precond(h, h->lq_s.p, h->lq_t.p, 0, true, false);
  double alpha = std::sqrt(dev_sum(h, lsq::S_RZ));
  CK(cudaMemsetAsync(h->lq_w.p, 0, sizeof(double) * n, st));
  lsq::launch_lsqr_step(n, 1.0 / alpha, 0.0, -1.0, h->lq_t.p, h->lq_s.p, h->lq_v.p, h->lq_q.p, h->x.p, h->lq_w.p,
                        st);  // v, q; w = v (x unchanged)
  launches += 3 + pl + 1;
  inf.local_launches += 1;
  std::vector<double> al{alpha}, be{beta};
  double phibar = beta, rhobar = alpha;
  const double est0 = alpha * beta;
  const int fixed = h->opt.fixed_iters;
  const int maxit = fixed > 0 ? fixed : h->opt.maxit;
  bool converged = false, checking = false, have_rel = false;
  double rel = 1.0;
  int it = 0;
  while (it < maxit) {
    if (timed) mark(h, 0);
    // beta u = A v - alpha u
    lsq::launch_spmv_csr(csr(h), h->lq_v.p, h->q.p, h->lanes_csr, h->grid_csr, st);
    if (timed) record_event(h->ev[6], st);
    lsq::launch_axpby(m, 1.0, h->q.p, -alpha, h->lq_u.p, h->lq_u.p, st);
    lsq::launch_dot(m, h->lq_u.p, h->lq_u.p, site(h, lsq::S_TMP, 3), st);
    beta = std::sqrt(dev_sum(h));
    if (!(beta > 0.0) || !std::isfinite(beta)) {
      if (beta == 0.0) { converged = true; break; }  // b lies in range(A V_k): x_k solves the problem
      throw LsError(LS_ERR_NONFINITE, "LSQR breakdown (beta) at iteration " + std::to_string(it + 1));
    }
    lsq::launch_axpby(m, 1.0 / beta, h->lq_u.p, 0.0, nullptr, h->lq_u.p, st);
    // alpha v = M^{-1} (A^T u - beta q)
    if (timed) record_event(h->ev[7], st);
    lsq::launch_spmv_csc(csc(h), h->lq_u.p, h->lq_s.p, nullptr, lsq::DotSite{}, h->lanes_csc, h->grid_csc, st);
    if (timed) mark(h, 1);
    lsq::launch_axpby(n, 1.0, h->lq_s.p, -beta, h->lq_q.p, h->lq_s.p, st);
    precond(h, h->lq_s.p, h->lq_t.p, 0, true, false, timed);
    alpha = std::sqrt(dev_sum(h, lsq::S_RZ));
    if (dev_sum(h, lsq::S_ERR) != 0.0)
      throw LsError(LS_ERR_DEVICE_TIMEOUT, "a bounded wait in the local-solve kernel gave up at iteration " +
                                               std::to_string(it + 1));
    if (!(alpha > 0.0) || !std::isfinite(alpha))
      throw LsError(LS_ERR_NONFINITE, "LSQR breakdown (alpha) at iteration " + std::to_string(it + 1));
    // plane rotation
    const double rho = std::hypot(rhobar, beta);
    const double c = rhobar / rho, sn = beta / rho;
    const double theta = sn * alpha;
    rhobar = -c * alpha;
    const double phi = c * phibar;
    phibar = sn * phibar;
    lsq::launch_lsqr_step(n, 1.0 / alpha, phi / rho, theta / rho, h->lq_t.p, h->lq_s.p, h->lq_v.p, h->lq_q.p,
                          h->x.p, h->lq_w.p, st);
    if (timed) mark(h, 5);
    ++it;
    launches += 6 + pl + 1;
    inf.local_launches += 1;
    al.push_back(alpha);
    be.push_back(beta);
    if (timed) {
      CK(cudaStreamSynchronize(st));
      float ta = 0.f, ta2 = 0.f, tb = 0.f, tc = 0.f, td = 0.f;
      CK(cudaEventElapsedTime(&ta, h->ev[0], h->ev[6]));
      CK(cudaEventElapsedTime(&ta2, h->ev[7], h->ev[1]));
      CK(cudaEventElapsedTime(&tb, h->ev[2], h->ev[3]));
      CK(cudaEventElapsedTime(&tc, h->ev[3], h->ev[4]));
      CK(cudaEventElapsedTime(&td, h->ev[0], h->ev[5]));
      inf.ms_spmv += ta + ta2; inf.ms_local += tb; inf.ms_coarse += tc; inf.ms_iter += td;
    }
    if (fixed > 0) continue;
    if (!checking && phibar * alpha * std::fabs(c) <= 10.0 * rtol * est0) checking = true;
    if (checking) {
      rel = std::sqrt(true_residual(h, 0, &launches)) / gn;
      have_rel = true;
      if (rel <= rtol) {
        converged = true;
        break;
      }
    }
  }
  if (!converged || fixed > 0 || !have_rel) rel = std::sqrt(true_residual(h, 0, &launches)) / gn;
  // kappa of M^{-1} A^T A from the bidiagonal: B_k^T B_k is the Lanczos matrix
  const int k = (int)al.size() - 1;
  if (k >= 1) {
    std::vector<double> d(k), e(std::max(k - 1, 0));
    for (int j = 0; j < k; ++j) {
      d[j] = al[j] * al[j] + be[j + 1] * be[j + 1];
      if (j + 1 < k) e[j] = al[j + 1] * be[j + 1];
    }
    const double lmax = tridiag_extreme(d, e, true), lmin = tridiag_extreme(d, e, false);
    inf.kappa_lanczos = lmin > 0 ? lmax / lmin : 0.0;
  }
  return finish(it, converged, rel);
}

// Restarted GMRES on C x = A^T b' (b' in h->bv, result in h->x), right-preconditioned in
// the flexible form (z_j = M^{-1} v_j kept): Arnoldi with classical Gram-Schmidt applied
// twice (multi-vector dot and update kernels, deterministic), Givens rotations on the
// host.  |gamma_{j+1}| = ||A^T b - C x_j||, the configs' residual; a pass (or the end of
// a cycle) updates x, and every cycle starts from the true residual, which confirms
// the pass.
ls_status gmres_core(ls_handle* h, double rtol, ls_info* info) {
  cudaStream_t st = h->st;
  const int64_t n = h->n;
  const int mr = h->opt.restart;
  const double t0 = now_s();
  ls_info inf{};
  inf.bad_subdomain = -1;
  int launches = 0;
  lsq::launch_spmv_csc(csc(h), h->bv.p, h->gm_g.p, nullptr, site(h, lsq::S_TMP, 0), h->lanes_csc, h->grid_csc, st);
  const double gg = dev_sum(h);
  launches += 1;
  if (!std::isfinite(gg)) throw LsError(LS_ERR_NONFINITE, "right-hand side is not finite");
  const double gn = std::sqrt(gg);
  lsq::launch_fill(n, 0.0, h->x.p, st);
  CK(cudaMemsetAsync(h->scal.p, 0, sizeof(double) * lsq::S_NSLOT, st));
  launches += 1;
  const bool timed = h->opt.time_kernels != 0;
  const int pl = h->opt.variant == 2 ? deflated_launches(h)
               : balanced(h) ? kBalancedLaunches : 2 + ((h->coarse && h->n0 > 0) ? 1 : 0);
  const int fixed = h->opt.fixed_iters;
  const int maxit = fixed > 0 ? fixed : h->opt.maxit;
  std::vector<double> H((size_t)(mr + 1) * mr, 0.0), cs(mr), sn(mr), gam(mr + 1), hv(2 * (size_t)(mr + 1));
  auto Hat = [&](int i, int j) -> double& { return H[(size_t)i * mr + j]; };
  double* V = h->gm_V.p;
  double* Z = h->gm_Z.p;
  double* h1 = h->gm_h.p;
  double* h2 = h->gm_h.p + (mr + 1);
  double* yv = h->gm_h.p + 2 * (mr + 1);
  int it = 0;
  bool converged = false;
  double rel = 1.0;
  while (true) {
    // r = A^T b - C x into V(:, 0)
    apply_C(h, h->x.p, h->w.p);
    lsq::launch_axpby(n, 1.0, h->gm_g.p, -1.0, h->w.p, V, st);
    lsq::launch_dot(n, V, V, site(h, lsq::S_TMP, 3), st);
    const double beta = std::sqrt(dev_sum(h));
    launches += 4;
    rel = gn > 0.0 ? beta / gn : 0.0;
    if (fixed <= 0 && beta <= rtol * gn) {
      converged = true;
      break;
    }
    if ((fixed > 0 && it >= fixed) || (fixed <= 0 && it >= maxit)) break;
    if (!std::isfinite(beta)) throw LsError(LS_ERR_NONFINITE, "GMRES: non-finite residual");
    lsq::launch_axpby(n, 1.0 / beta, V, 0.0, nullptr, V, st);
    std::fill(gam.begin(), gam.end(), 0.0);
    gam[0] = beta;
    int j = 0;
    while (j < mr) {
      double* vj = V + (int64_t)j * n;
      double* zj = Z + (int64_t)j * n;
      double* w = V + (int64_t)(j + 1) * n;
      if (timed) mark(h, 0);
      precond(h, vj, zj, 0, false, false, timed);
      if (timed) record_event(h->ev[6], st);
      apply_C(h, zj, w);
      if (timed) mark(h, 1);
      lsq::launch_multi_dot(n, V, n, j + 1, w, h->gm_part.p, h1, st);
      lsq::launch_multi_axpy(n, V, n, j + 1, h1, -1.0, w, st);
      lsq::launch_multi_dot(n, V, n, j + 1, w, h->gm_part.p, h2, st);
      lsq::launch_multi_axpy(n, V, n, j + 1, h2, -1.0, w, st);
      lsq::launch_dot(n, w, w, site(h, lsq::S_TMP, 3), st);
      CK(cudaMemcpyAsync(hv.data(), h1, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(hv.data() + (mr + 1), h2, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, st));
      const double hn = std::sqrt(dev_sum(h));  // synchronises the stream
      if (dev_sum(h, lsq::S_ERR) != 0.0)
        throw LsError(LS_ERR_DEVICE_TIMEOUT, "a bounded wait in the local-solve kernel gave up at iteration " +
                                                 std::to_string(it + 1));
      if (!std::isfinite(hn)) throw LsError(LS_ERR_NONFINITE, "GMRES breakdown at iteration " + std::to_string(it + 1));
      if (timed) {
        record_event(h->ev[5], st);
        CK(cudaStreamSynchronize(st));
        float ta = 0.f, tb = 0.f, tc = 0.f, td = 0.f;
        CK(cudaEventElapsedTime(&ta, h->ev[6], h->ev[1]));
        CK(cudaEventElapsedTime(&tb, h->ev[2], h->ev[3]));
        CK(cudaEventElapsedTime(&tc, h->ev[3], h->ev[4]));
        CK(cudaEventElapsedTime(&td, h->ev[0], h->ev[5]));
        inf.ms_spmv += ta; inf.ms_local += tb; inf.ms_coarse += tc; inf.ms_iter += td;
      }
      for (int i = 0; i <= j; ++i) Hat(i, j) = hv[i] + hv[(mr + 1) + i];
      Hat(j + 1, j) = hn;
      if (hn > 0.0) lsq::launch_axpby(n, 1.0 / hn, w, 0.0, nullptr, w, st);
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * Hat(i, j) + sn[i] * Hat(i + 1, j);
        Hat(i + 1, j) = -sn[i] * Hat(i, j) + cs[i] * Hat(i + 1, j);
        Hat(i, j) = t;
      }
      const double den = std::hypot(Hat(j, j), Hat(j + 1, j));
      cs[j] = Hat(j, j) / den;
      sn[j] = Hat(j + 1, j) / den;
      Hat(j, j) = den;
      Hat(j + 1, j) = 0.0;
      gam[j + 1] = -sn[j] * gam[j];
      gam[j] = cs[j] * gam[j];
      ++j;
      ++it;
      launches += pl + 2 + 4 * 2 + 1 + (hn > 0.0 ? 1 : 0);
      inf.local_launches += 1;
      if (fixed > 0 && it >= fixed) break;
      if (fixed <= 0 && (std::fabs(gam[j]) <= rtol * gn || it >= maxit)) break;
      if (!(hn > 0.0)) break;  // the Krylov space is invariant: the cycle's solution is exact
    }
    // x += Z y, H(0:j, 0:j) y = gamma(0:j)
    std::vector<double> y(j);
    for (int i = j - 1; i >= 0; --i) {
      double s = gam[i];
      for (int k = i + 1; k < j; ++k) s -= Hat(i, k) * y[k];
      y[i] = s / Hat(i, i);
    }
    CK(cudaMemcpyAsync(yv, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, st));
    lsq::launch_multi_axpy(n, Z, n, j, yv, 1.0, h->x.p, st);
    CK(cudaStreamSynchronize(st));
    launches += 1;
  }
  check_launch("GMRES");
  inf.iters = it;
  inf.relres_true = rel;
  inf.relres_recursive = rel;
  inf.n0 = h->sinfo.n0; inf.kmin = h->sinfo.kmin; inf.kmax = h->sinfo.kmax; inf.tau_used = h->sinfo.tau_used;
  inf.delta = h->sinfo.delta; inf.t_setup = h->sinfo.t_setup; inf.t_eig = h->sinfo.t_eig;
  inf.eig_steps_max = h->sinfo.eig_steps_max;
  inf.launches = launches;
  inf.lanes_csr = h->lanes_csr; inf.lanes_csc = h->lanes_csc; inf.normal_product = h->normal_kind; inf.local_config = h->local_cfg;
  inf.t_solve = now_s() - t0;
  if (info) *info = inf;
  if (!converged && fixed <= 0)
    return (g_err = "maximum number of iterations reached, true relative residual " + std::to_string(rel),
            LS_ERR_NOT_CONVERGED);
  return LS_OK;
}

template <class F>
ls_status guarded(F&& f) {
  try {
    g_err.clear();
    return f();
  } catch (const LsError& e) {
    g_err = e.what();
    return e.st;
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed";
    return LS_ERR_OOM;
  } catch (const std::exception& e) {
    g_err = e.what();
    return LS_ERR_CUDA;
  }
}

template <class T>
std::vector<T> to_host(const T* src, size_t count) {
  std::vector<T> v(count);
  if (count) {
    cudaError_t e = cudaMemcpy(v.data(), src, count * sizeof(T), cudaMemcpyDefault);
    if (e != cudaSuccess) throw LsError(LS_ERR_INVALID, std::string("cannot read input array: ") + cudaGetErrorString(e));
  }
  return v;
}

// f(begin, end) over [0, count) split across the host's threads.
template <class F>
void host_parallel(int64_t count, F&& f) {
  const unsigned hw = std::thread::hardware_concurrency();
  const int64_t nt = std::max<int64_t>(1, std::min<int64_t>(hw ? hw : 4, 32));
  if (count < 65536 || nt == 1) {
    f((int64_t)0, count);
    return;
  }
  std::vector<std::thread> th;
  const int64_t per = (count + nt - 1) / nt;
  for (int64_t k = 0; k < nt; ++k) {
    const int64_t a = k * per, b = std::min(count, a + per);
    if (a < b) th.emplace_back([&f, a, b]() { f(a, b); });
  }
  for (auto& t : th) t.join();
}

// A host thread that is joined when the owner leaves its scope (also by an exception).
struct HostJob {
  std::thread t;
  void join() {
    if (t.joinable()) t.join();
  }
  ~HostJob() { join(); }
};

// The CSC and sliced-ELL copies of A' take their values from the CSR values h->val.
void refresh_value_copies(ls_handle* h) {
  cudaStream_t st = h->st;
  lsq::launch_gather64(h->nnz, h->cperm.p, h->val.p, h->cval.p, st);
  lsq::launch_gather64((int64_t)h->sellA_src.n, h->sellA_src.p, h->val.p, h->sellA_val.p, st);
  lsq::launch_gather64((int64_t)h->sellB_src.n, h->sellB_src.p, h->val.p, h->sellB_val.p, st);
  if (h->nt_tiles > 0) {
    lsq::launch_gather64((int64_t)h->nt_asrc.n, h->nt_asrc.p, h->val.p, h->nt_aval.p, st);
    lsq::launch_gather64((int64_t)h->nt_bsrc.n, h->nt_bsrc.p, h->val.p, h->nt_bval.p, st);
  }
}

void release_normal_tiles(ls_handle* h) {
  h->nt_tiles = 0;
  h->nt_smem = 0;
  h->nt_lo.release(); h->nt_wid.release(); h->nt_as0.release(); h->nt_bs0.release();
  h->nt_aoff.release(); h->nt_acol.release(); h->nt_aval.release();
  h->nt_boff.release(); h->nt_brow.release(); h->nt_bval.release(); h->nt_bcid.release();
  h->nt_poff.release(); h->nt_asrc.release(); h->nt_bsrc.release();
  h->nt_cb0.release(); h->nt_cb1.release(); h->nt_part.release();
}

// Lanes per row (A) and per column (A^T) of the two sparse products, picked by timing
// every candidate kernel on the actual matrix (three launches each, CUDA events); then
// the form of the normal product: the best pair against the row tiles (when built),
// whose copies are freed if the pair wins.
void autotune_spmv(ls_handle* h) {
  cudaStream_t st = h->st;
  DevBuf<double> xa, ya;
  xa.alloc(std::max(h->m, h->n));
  ya.alloc(std::max(h->m, h->n));
  xa.zero(st);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto time_it = [&](auto&& launch) {
    launch();  // warm
    CK(cudaEventRecord(e0, st));
    for (int k = 0; k < 3; ++k) launch();
    CK(cudaEventRecord(e1, st));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    return ms;
  };
  const int forced = h->opt.spmv;
  float best = 1e30f;
  // candidates (kernel codes of kernels.h): sliced ELL, warp-stream, lanes per row
  const int cand[] = {-2, -1, -3, 1, 2, 4, 8, 16, 32};
  for (int lanes : cand) {
    if (forced != 0 && lanes != forced) continue;
    const float ms = time_it([&] { lsq::launch_spmv_csr(csr(h), xa.p, ya.p, lanes, 0, st); });
    if (ms < best) { best = ms; h->lanes_csr = lanes; }
  }
  best = 1e30f;
  for (int lanes : cand) {
    if (forced != 0 && lanes != forced) continue;
    const float ms = time_it([&] { lsq::launch_spmv_csc(csc(h), xa.p, ya.p, nullptr, lsq::DotSite{}, lanes, 0, st); });
    if (ms < best) { best = ms; h->lanes_csc = lanes; }
  }
  // The normal product runs after the local solve has streamed the factors through L2:
  // its candidates are timed one launch at a time after a write of a buffer larger than L2.
  h->normal_kind = 1;
  if (h->nt_tiles > 0) {
    DevBuf<unsigned char> flush;
    flush.alloc((size_t)256 << 20);
    auto time_cold = [&](auto&& launch) {
      launch();  // warm
      float total = 0.f;
      for (int k = 0; k < 3; ++k) {
        CK(cudaMemsetAsync(flush.p, k, flush.n, st));
        CK(cudaEventRecord(e0, st));
        launch();
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        total += ms;
      }
      return total;
    };
    float best_tiles = 1e30f;
    for (int cfg = 1; cfg <= 4; ++cfg) {
      if (h->opt.normal_kernel != 0 && cfg != h->opt.normal_kernel) continue;
      h->nt_cfg = cfg;
      const float ms = time_cold([&] { lsq::launch_normal_tiles(ntiles(h), xa.p, ya.p, nullptr, lsq::DotSite{}, st); });
      h->nt_ms[cfg] = ms / 3.f;
      if (ms < best_tiles) { best_tiles = ms; best = (float)cfg; }
    }
    h->nt_cfg = (int)best;
    const float pair = h->opt.normal_product == 2 ? 1e30f : time_cold([&] {
      lsq::launch_spmv_csr(csr(h), xa.p, ya.p, h->lanes_csr, 0, st);
      lsq::launch_spmv_csc(csc(h), ya.p, xa.p, nullptr, lsq::DotSite{}, h->lanes_csc, 0, st);
    });
    h->nt_ms[0] = h->opt.normal_product == 2 ? 0.f : pair / 3.f;
    if (best_tiles < pair) h->normal_kind = 2;
    else release_normal_tiles(h);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  check_launch("sparse-product autotuning");
}

void do_setup(ls_handle* h, const int64_t* row_ptr_in, const int32_t* col_in, const double* val_in,
              const int32_t* part_in) {
  const double t_begin = now_s();
  Phase phase("ls_setup: inputs and index sets (host)");
  cudaStream_t st = h->st;
  std::vector<int64_t> hrp = to_host(row_ptr_in, (size_t)h->m + 1);
  const int64_t nnz = hrp[h->m];
  if (nnz < 0 || hrp[0] != 0) throw LsError(LS_ERR_INVALID, "row_ptr must start at 0 and end at nnz >= 0");
  std::vector<int32_t> hcol = to_host(col_in, (size_t)nnz);
  std::vector<double> hval = to_host(val_in, (size_t)nnz);
  std::vector<int32_t> hpart = to_host(part_in, (size_t)h->n);
  for (int64_t e = 0; e < nnz; ++e)
    if (!std::isfinite(hval[e])) throw LsError(LS_ERR_NONFINITE, "A has a non-finite value at entry " + std::to_string(e));
  {
    const std::string verr = lsq::validate_inputs(h->m, h->n, hrp.data(), hcol.data(), h->N, hpart.data());
    if (!verr.empty()) throw LsError(LS_ERR_INVALID, verr);
  }
  {
    const std::string berr = lsq::validate_batch(h->m, h->n, hrp.data(), hcol.data(), h->N, hpart.data(), h->nprob,
                                                 h->h_m_off.data(), h->h_n_off.data(), h->h_N_off, h->prob_of_sub);
    if (!berr.empty()) throw LsError(LS_ERR_INVALID, berr);
  }
  // Work with A' = P A, rows ordered by first column (min ||Ax - b|| = min ||PAx - Pb||):
  // neighbouring rows then touch neighbouring entries of x and of A p.
  {
    std::vector<int32_t> perm;
    lsq::order_rows_by_first_column(h->m, h->n, hrp.data(), hcol.data(), perm);
    std::vector<int64_t> rp2(h->m + 1, 0), emap(nnz);
    std::vector<int32_t> c2(nnz);
    std::vector<double> v2(nnz);
    for (int64_t r2 = 0; r2 < h->m; ++r2) rp2[r2 + 1] = rp2[r2] + (hrp[perm[r2] + 1] - hrp[perm[r2]]);
    host_parallel(h->m, [&](int64_t a, int64_t b) {
      for (int64_t r2 = a; r2 < b; ++r2) {
        const int32_t r = perm[r2];
        const int64_t len = hrp[r + 1] - hrp[r];
        for (int64_t k = 0; k < len; ++k) {
          c2[rp2[r2] + k] = hcol[hrp[r] + k];
          v2[rp2[r2] + k] = hval[hrp[r] + k];
          emap[rp2[r2] + k] = hrp[r] + k;
        }
      }
    });
    h->perm.upload(perm, st);
    h->entmap.upload(emap, st);
    CK(cudaStreamSynchronize(st));
    h->h_perm.swap(perm);
    hrp.swap(rp2);
    hcol.swap(c2);
    hval.swap(v2);
  }
  // Optional column equilibration: the preconditioner is built for A S.
  std::vector<double> hval_orig, colscale;
  if (h->opt.equilibrate) {
    colscale.assign(h->n, 0.0);
    for (int64_t e = 0; e < nnz; ++e) colscale[hcol[e]] += hval[e] * hval[e];
    for (auto& s : colscale) s = s > 0.0 ? 1.0 / std::sqrt(s) : 1.0;
    hval_orig = hval;
    for (int64_t e = 0; e < nnz; ++e) hval[e] *= colscale[hcol[e]];
  }
  lsq::HostSets hs;
  std::string err = lsq::build_host_sets(h->m, h->n, hrp.data(), hcol.data(), h->N, hpart.data(), h->coarse, hs);
  if (!err.empty()) throw LsError(LS_ERR_INVALID, err);
  h->nnz = nnz;
  const int N = h->N;
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->dev));
  (void)sms;
  h->lanes_csr = pow2_lanes((double)nnz / (double)h->m);
  h->lanes_csc = pow2_lanes((double)nnz / (double)h->n);

  // matrix copies
  phase.next("ls_setup: matrix copies");
  h->row_ptr.upload(hrp, st);
  h->col.upload(hcol, st);
  h->val.upload(hval, st);
  h->col_ptr.upload(hs.csc_ptr, st);
  h->crow.upload(hs.csc_row, st);
  std::vector<double> cv(nnz);
  host_parallel(nnz, [&](int64_t a, int64_t b) {
    for (int64_t t = a; t < b; ++t) cv[t] = hval[hs.csc_perm[t]];
  });
  h->cval.upload(cv, st);
  h->cperm.upload(hs.csc_perm, st);
  h->part.upload(hpart, st);
  // The copies that only the sparse-product autotuner needs (sliced ELL of A and A^T,
  // the row tiles of the one-pass normal product: not on batched handles, whose solves
  // run the multi right-hand-side products) are built by a host thread while the device
  // runs the factorisations and eigensolves; the autotuning runs at the end of setup.
  const bool want_tiles =
      h->opt.normal_product == 2 || (h->opt.normal_product == 0 && h->opt.spmv == 0 && h->nprob == 1);
  int smem_optin = 0;
  CK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev));
  const int tile_cap = smem_optin / 8 - 128;
  if (h->opt.normal_product == 2) {
    // one row alone must fit a tile (its padded row and its column span)
    for (int64_t r = 0; r < h->m; ++r)
      if (hrp[r + 1] > hrp[r] && 32 + ((hcol[hrp[r + 1] - 1] - hcol[hrp[r]] + 2) & ~1) > tile_cap)
        throw LsError(LS_ERR_UNSUPPORTED, "normal_product = 2: a row's column span does not fit a block's shared memory");
  }
  lsq::SellHost sa, sb;
  lsq::NormalTilesHost nt;
  bool nt_ok = false, job_failed = false;
  HostJob job;  // declared after everything it reads: joined first on every way out
  job.t = std::thread([&]() {
    try {
      lsq::build_sell(h->m, hrp.data(), hcol.data(), hval.data(), 256, sa);
      lsq::build_sell(h->n, hs.csc_ptr.data(), hs.csc_row.data(), cv.data(), 256, sb);
      // where every stored copy of an entry comes from (A' CSR slot), for ls_update_values
      for (auto& e : sb.src)
        if (e >= 0) e = hs.csc_perm[e];
      if (want_tiles) nt_ok = lsq::build_normal_tiles(h->m, h->n, hrp.data(), hcol.data(), hval.data(), tile_cap, sms, nt);
    } catch (...) {
      job_failed = true;
    }
  });

  // local plan
  phase.next("ls_setup: local matrices and Cholesky factors");
  h->total_local = hs.om_off[N];
  h->total_blocks = hs.blk_off[N];
  h->fac_elems = hs.fac_elems;
  h->max_nb = hs.max_nb;
  h->wmax = 0;
  for (int i = 0; i < h->N; ++i)
    for (int64_t b = hs.blk_off[i]; b < hs.blk_off[i + 1]; ++b)
      h->wmax = std::max<int>(h->wmax, (int)(b - hs.blk_off[i]) - hs.blk_tf[b] + 1);
  {
    // the local solve keeps one subdomain's right-hand side in shared memory
    int optin = 0;
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev));
    const size_t need = lsq::local_solve_smem(h->opt.factor_prec, h->max_nb, 1);
    if (need > (size_t)optin)
      throw LsError(LS_ERR_UNSUPPORTED, "largest subdomain (" + std::to_string((int64_t)h->max_nb * 32) +
                                            " padded columns) needs " + std::to_string(need) +
                                            " B of shared memory in the local solve; the device allows " +
                                            std::to_string(optin) + " B: use more subdomains");
  }
  h->om_off.upload(hs.om_off, st);
  h->om_glob.upload(hs.om_glob, st);
  h->om_int.upload(hs.om_int, st);
  h->blk_off.upload(hs.blk_off, st);
  h->blk_tf.upload(hs.blk_tf, st);
  {
    std::vector<int64_t> po(hs.blk_poff);
    po.push_back(hs.fac_elems);
    h->blk_poff.upload(po, st);
  }
  h->map_ptr.upload(hs.map_ptr, st);
  h->map_idx.upload(hs.map_idx, st);
  h->int_off.upload(hs.int_off, st);
  h->int_loc.upload(hs.int_loc, st);
  h->jj_of.upload(hs.jj_of, st);
  h->nI.upload(hs.nI, st);
  {
    std::vector<int32_t> ig(hs.int_off[N]);
    for (int i = 0; i < N; ++i)
      for (int64_t a = hs.int_off[i]; a < hs.int_off[i + 1]; ++a)
        ig[a] = hs.om_glob[hs.om_off[i] + hs.int_loc[a]];
    h->int_glob.upload(ig, st);
    if (h->opt.variant == 2) {
      // RAS: the local-solution entry that column j takes from its own subdomain
      std::vector<int64_t> own(h->n, 0);
      for (int i = 0; i < N; ++i)
        for (int64_t a = hs.int_off[i]; a < hs.int_off[i + 1]; ++a) own[ig[a]] = hs.om_off[i] + hs.int_loc[a];
      h->own.upload(own, st);
    }
  }
  DevBuf<int32_t> row_sub;
  {
    std::vector<int32_t> rs(h->total_local);
    for (int i = 0; i < N; ++i)
      for (int64_t e = hs.om_off[i]; e < hs.om_off[i + 1]; ++e) rs[e] = i;
    row_sub.upload(rs, st);
  }
  h->h_om_off = hs.om_off;
  h->h_om_paper = hs.om_paper;
  h->h_xi_off = hs.xi_off;
  h->h_xi = hs.xi;
  h->h_nI = hs.nI;

  lsq::BandPlan plan{N, h->om_off.p, h->om_glob.p, h->om_int.p, h->blk_off.p, h->blk_tf.p, h->blk_poff.p, row_sub.p};

  // assemble C_ii and C~_ii (Algorithm 1 steps 6-7), shifts, factors
  DevBuf<double> Cst, Ctst, Bst;
  Cst.alloc(h->fac_elems); Cst.zero(st);
  Ctst.alloc(h->fac_elems); Ctst.zero(st);
  lsq::launch_assemble(plan, csr(h), csc(h), h->part.p, h->total_local, Cst.p, Ctst.p, st);
  check_launch("assembly");
  DevBuf<double> cn2, ctn2, sdev;
  cn2.alloc(N); ctn2.alloc(N);
  lsq::launch_norms(plan, Cst.p, Ctst.p, cn2.p, ctn2.p, st);
  std::vector<double> hcn2(N), hctn2(N);
  CK(cudaMemcpyAsync(hcn2.data(), cn2.p, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hctn2.data(), ctn2.p, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  check_launch("norms");
  // delta_q = delta_rel ||C_q||_F for each independent problem q (Section 4.1.2)
  std::vector<double> hdsub(N);
  h->h_delta.assign(h->nprob, 0.0);
  for (int q = 0; q < h->nprob; ++q) {
    double cf2 = 0.0;
    for (int i = h->h_N_off[q]; i < h->h_N_off[q + 1]; ++i) cf2 += hcn2[i];
    h->h_delta[q] = h->opt.delta_rel * std::sqrt(cf2);
    for (int i = h->h_N_off[q]; i < h->h_N_off[q + 1]; ++i) hdsub[i] = h->h_delta[q];
  }
  const double delta = h->h_delta[0];
  h->dsub.upload(hdsub, st);
  std::vector<double> hs_shift(N);
  for (int i = 0; i < N; ++i) hs_shift[i] = h->opt.s_rel * std::sqrt(hctn2[i]);
  sdev.upload(hs_shift, st);
  h->eqs.alloc(h->total_local);
  Bst.alloc(h->fac_elems);  // prep always writes B = C~_ii + s I
  lsq::launch_prep(plan, h->dsub.p, sdev.p, Cst.p, h->eqs.p, Ctst.p, Bst.p, st);
  check_launch("prep");
  DevBuf<double> dinv, Bidiag, idiag;
  DevBuf<int> status;
  dinv.alloc((size_t)h->total_blocks * 1024);
  status.alloc(N);
  idiag.alloc((size_t)h->total_blocks * 32);
  lsq::launch_band_cholesky(plan, Cst.p, idiag.p, dinv.p, status.p, st);
  std::vector<int> hst(N);
  CK(cudaMemcpyAsync(hst.data(), status.p, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  check_launch("local Cholesky");
  for (int i = 0; i < N; ++i)
    if (hst[i]) {
      h->sinfo.bad_subdomain = i;
      throw LsError(LS_ERR_FACTOR, "Cholesky of C_ii failed in subdomain " + std::to_string(i) + " at local row " +
                                       std::to_string(hst[i] - 1));
    }
  // solve storage in the factor precision: column-major panels + inverse diagonal tiles
  h->prec = h->opt.factor_prec;
  {
    void* dst = nullptr;
    if (h->prec == LS_PREC_F64) { h->L64.alloc(h->fac_elems); dst = h->L64.p; }
    else if (h->prec == LS_PREC_F32) { h->L32.alloc(h->fac_elems); dst = h->L32.p; }
    else {
      h->L16.alloc(h->fac_elems);
      h->tsc.alloc(std::max<int64_t>(h->fac_elems / 1024, 1));
      dst = h->L16.p;
    }
    lsq::launch_to_solve_layout(h->prec, h->total_blocks, h->blk_poff.p, Cst.p, dinv.p, dst,
                                h->prec == LS_PREC_BF16 ? h->tsc.p : nullptr, st);
    CK(cudaStreamSynchronize(st));
    check_launch("solve storage");
    Cst.release();
    idiag.release();
  }

  h->sinfo.delta = delta;
  h->kwant_cap = h->opt.nev_max + 1;
  h->h_k.assign(N, 0);
  h->h_steps.assign(N, 0);
  h->coff.alloc(N + 1);
  h->zoff.alloc(N + 1);
  {
    std::vector<int32_t> zc(N + 1, 0);
    std::vector<int64_t> zz(N + 1, 0);
    h->coff.upload(zc, st);
    h->zoff.upload(zz, st);
  }
  h->n0 = 0;
  if (h->coarse) {
    const double te0 = now_s();
    phase.next("ls_setup: local eigensolves and coarse operator");
    Bidiag.alloc((size_t)h->total_blocks * 32);
    lsq::launch_band_cholesky(plan, Bst.p, Bidiag.p, dinv.p, status.p, st);
    CK(cudaMemcpyAsync(hst.data(), status.p, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    check_launch("Cholesky of C~_ii + s I");
    for (int i = 0; i < N; ++i)
      if (hst[i]) {
        h->sinfo.bad_subdomain = i;
        throw LsError(LS_ERR_FACTOR, "Cholesky of C~_ii + s I failed in subdomain " + std::to_string(i));
      }
    const int kw = h->kwant_cap;
    int K = std::max(48, 2 * kw + 24);
    K += K & 1;
    if (K > 160) throw LsError(LS_ERR_UNSUPPORTED, "nev_max too large for the device eigensolver (max 67)");
    const int keep = kw + (K - kw) / 2;
    const int64_t vs = (int64_t)h->max_nb * 32;
    DevBuf<double> V, V2, H, S, vec, lam;
    DevBuf<int> nconv, steps, est;
    V.alloc((size_t)N * K * vs); V2.alloc((size_t)N * K * vs);
    H.alloc((size_t)N * K * K); S.alloc((size_t)N * K * K);
    vec.alloc((size_t)N * 2 * vs);
    lam.alloc((size_t)N * kw); lam.zero(st);
    nconv.alloc(N); steps.alloc(N); est.alloc(N);
    lsq::EigArgs ea{};
    ea.P = plan; ea.Bfac = Bst.p; ea.Bidiag = Bidiag.p; ea.Ct = Ctst.p; ea.delta = h->dsub.p;
    ea.kwant_cap = kw; ea.Kmax = K; ea.keep = keep; ea.maxit = h->opt.eig_maxit; ea.tol = h->opt.eig_tol;
    ea.V = V.p; ea.V2 = V2.p; ea.vstride = vs; ea.H = H.p; ea.S = S.p; ea.vec = vec.p; ea.lam = lam.p;
    ea.nconv = nconv.p; ea.steps = steps.p; ea.status = est.p;
    lsq::launch_lanczos(ea, st);
    h->h_lam.assign((size_t)N * kw, 0.0);
    CK(cudaMemcpyAsync(h->h_lam.data(), lam.p, sizeof(double) * N * kw, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h->h_steps.data(), steps.p, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hst.data(), est.p, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    check_launch("local eigensolves");
    for (int i = 0; i < N; ++i) {
      h->sinfo.eig_steps_max = std::max(h->sinfo.eig_steps_max, h->h_steps[i]);
      if (hst[i]) {
        h->sinfo.bad_subdomain = i;
        throw LsError(LS_ERR_EIGEN, "eigensolve of subdomain " + std::to_string(i) + " did not converge in " +
                                        std::to_string(h->h_steps[i]) + " steps");
      }
    }
    // threshold 1/tau (Lemma 2.4 / eq. (3.6)); tau <= 0: max_i lambda_{i, nev_max+1}
    // (per independent problem when batched)
    h->h_thr.assign(h->nprob, 0.0);
    double thr_max = 0.0;
    for (int q = 0; q < h->nprob; ++q) {
      double thr = 0.0;
      if (h->tau > 0) {
        thr = 1.0 / h->tau;
      } else {
        for (int i = h->h_N_off[q]; i < h->h_N_off[q + 1]; ++i) {
          const int64_t ni = hs.om_off[i + 1] - hs.om_off[i];
          if (ni > h->opt.nev_max) thr = std::max(thr, h->h_lam[(size_t)i * kw + h->opt.nev_max]);
        }
      }
      h->h_thr[q] = thr;
      thr_max = std::max(thr_max, thr);
    }
    h->sinfo.tau_used = thr_max > 0 ? 1.0 / thr_max : INFINITY;
    std::vector<int32_t> hcoff(N + 1, 0);
    std::vector<int64_t> hzoff(N + 1, 0), hwoff(N + 1, 0);
    int kmin = 1 << 30, kmax = 0;
    for (int i = 0; i < N; ++i) {
      const int64_t ni = hs.om_off[i + 1] - hs.om_off[i];
      const int lim = (int)std::min<int64_t>(std::min<int64_t>(kw, ni), h->opt.nev_max);
      const double thr = h->h_thr[h->prob_of_sub[i]];
      int k = 0;
      while (k < lim && h->h_lam[(size_t)i * kw + k] > thr) ++k;
      h->h_k[i] = k;
      kmin = std::min(kmin, k); kmax = std::max(kmax, k);
      hcoff[i + 1] = hcoff[i] + k;
      hzoff[i + 1] = hzoff[i] + (int64_t)k * hs.nI[i];
      hwoff[i + 1] = hwoff[i] + (int64_t)k * (hs.xi_off[i + 1] - hs.xi_off[i]);
    }
    h->n0 = hcoff[N];
    h->sinfo.kmin = kmin; h->sinfo.kmax = kmax; h->sinfo.n0 = (int)h->n0;
    h->coff.upload(hcoff, st);
    h->zoff.upload(hzoff, st);
    h->Z.alloc(std::max<int64_t>(hzoff[N], 1));
    lsq::launch_eigvec(ea, h->coff.p, h->zoff.p, h->int_off.p, h->int_loc.p, h->Z.p, st);
    check_launch("coarse basis");
    V.release(); V2.release(); H.release(); S.release(); vec.release();
    if (h->n0 > 0) {
      DevBuf<int64_t> woff, xi_off, poff;
      DevBuf<int32_t> xi, xi_sub, pi, pj, ppi, ppj;
      DevBuf<double> W;
      woff.upload(hwoff, st);
      xi_off.upload(hs.xi_off, st);
      xi.upload(hs.xi, st);
      {
        std::vector<int32_t> xs(hs.xi_off[N]);
        for (int i = 0; i < N; ++i)
          for (int64_t a = hs.xi_off[i]; a < hs.xi_off[i + 1]; ++a) xs[a] = i;
        xi_sub.upload(xs, st);
      }
      W.alloc(std::max<int64_t>(hwoff[N], 1));
      lsq::launch_coarse_w(N, xi_off.p, xi.p, h->coff.p, woff.p, h->zoff.p, h->nI.p, csr(h), h->part.p, h->jj_of.p,
                           h->Z.p, W.p, hs.xi_off[N], xi_sub.p, st);
      pi.upload(hs.pair_i, st); pj.upload(hs.pair_j, st); poff.upload(hs.pair_off, st);
      ppi.upload(hs.pair_pi, st); ppj.upload(hs.pair_pj, st);
      // C_00 in one dense block per problem, each padded to a multiple of 32
      const int Q = h->nprob;
      h->h_cb_base.assign(Q, 0); h->h_cb_ld.assign(Q, 0); h->h_cb_c0.assign(Q, 0); h->h_n0q.assign(Q, 0);
      int64_t base = 0, ldmax = 0;
      for (int q = 0; q < Q; ++q) {
        h->h_cb_c0[q] = hcoff[h->h_N_off[q]];
        h->h_n0q[q] = hcoff[h->h_N_off[q + 1]] - hcoff[h->h_N_off[q]];
        h->h_cb_ld[q] = (h->h_n0q[q] + 31) / 32 * 32;
        h->h_cb_base[q] = base;
        base += h->h_cb_ld[q] * h->h_cb_ld[q];
        ldmax = std::max(ldmax, h->h_cb_ld[q]);
      }
      h->xinv_elems = base;
      h->n0p = h->h_cb_ld[0];
      h->cb_prob_of_sub.upload(h->prob_of_sub, st);
      h->cb_base.upload(h->h_cb_base, st);
      h->cb_ld.upload(h->h_cb_ld, st);
      h->cb_c0.upload(h->h_cb_c0, st);
      h->Xinv.alloc((size_t)base);
      h->Xinv.zero(st);
      for (int q = 0; q < Q; ++q)
        if (h->h_cb_ld[q] > h->h_n0q[q])
          k_set_diag<<<32, 256, 0, st>>>(h->Xinv.p + h->h_cb_base[q], h->h_cb_ld[q], h->h_n0q[q], h->h_cb_ld[q], 1.0);
      const lsq::CoarseBlocks cb{h->cb_prob_of_sub.p, h->cb_base.p, h->cb_ld.p, h->cb_c0.p};
      lsq::launch_coarse_pairs((int)hs.pair_i.size(), pi.p, pj.p, poff.p, ppi.p, ppj.p, h->coff.p, woff.p, h->zoff.p,
                               h->nI.p, W.p, h->Z.p, h->dsub.p, cb, h->Xinv.p, st);
      check_launch("coarse operator");
      W.release();
      DevBuf<double> Y, dinvc;
      Y.alloc((size_t)ldmax * ldmax);
      dinvc.alloc((size_t)(ldmax / 32) * 1024);
      DevBuf<int> cstat;
      cstat.alloc(Q);
      cstat.zero(st);
      for (int q = 0; q < Q; ++q)
        if (h->h_n0q[q] > 0)
          lsq::dense_spd_inverse(h->h_cb_ld[q], h->Xinv.p + h->h_cb_base[q], Y.p, dinvc.p, cstat.p + q, st);
      std::vector<int> hcst(Q);
      CK(cudaMemcpyAsync(hcst.data(), cstat.p, sizeof(int) * Q, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      check_launch("coarse factorization");
      for (int q = 0; q < Q; ++q)
        if (hcst[q])
          throw LsError(LS_ERR_FACTOR, "Cholesky of C_00 failed at row " + std::to_string(hcst[q] - 1) +
                                           (Q > 1 ? " of problem " + std::to_string(q) : std::string()));
    }
    h->sinfo.t_eig = now_s() - te0;
  } else {
    h->sinfo.tau_used = 0.0;
  }
  Bst.release(); Ctst.release(); Bidiag.release();

  if (h->opt.equilibrate) {
    // the operator is A itself; M^{-1} = S M_S^{-1} S with S folded into the local
    // gather/scatter scales and into the rows of the coarse basis
    CK(cudaMemcpyAsync(h->val.p, hval_orig.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, st));
    refresh_value_copies(h);
    DevBuf<double> sdev;
    sdev.upload(colscale, st);
    k_scale_by_gather<<<1024, 256, 0, st>>>(h->total_local, h->om_glob.p, sdev.p, h->eqs.p);
    if (h->n0 > 0) k_scale_zbar<<<N, 256, 0, st>>>(h->coff.p, h->zoff.p, h->int_off.p, h->int_glob.p, sdev.p, h->Z.p);
    CK(cudaStreamSynchronize(st));
    check_launch("column equilibration");
  }

  // work vectors
  const int64_t mm = std::max(h->m, h->n);
  h->x.alloc(h->n); h->r.alloc(h->n); h->r_old.alloc(h->n); h->z.alloc(h->n); h->p.alloc(h->n);
  h->q.alloc(mm); h->w.alloc(h->n); h->ybuf.alloc(h->total_local);
  h->r0.alloc(std::max<int64_t>(h->n0p, 1)); h->r0.zero(st);
  h->y0.alloc(std::max<int64_t>(h->n0p, 1)); h->y0.zero(st);
  h->tv.alloc(h->n); h->bv.alloc(h->m);
  if (h->opt.variant == 1 || h->opt.variant == 2) {
    h->bal_y.alloc(h->n); h->bal_t.alloc(h->n); h->bal_u.alloc(h->n); h->bal_v.alloc(h->n);
  }
  if (h->opt.solver == 2) {
    const int mr = h->opt.restart;
    h->gm_V.alloc((size_t)h->n * (mr + 1));
    h->gm_Z.alloc((size_t)h->n * mr);
    h->gm_g.alloc(h->n);
    h->gm_h.alloc(3 * (size_t)(mr + 1));
    h->gm_part.alloc((size_t)lsq::multi_dot_grid(h->n) * (mr + 1));
  }
  if (h->opt.solver == 1) {
    h->lq_u.alloc(h->m);
    h->lq_v.alloc(h->n); h->lq_q.alloc(h->n); h->lq_s.alloc(h->n); h->lq_t.alloc(h->n); h->lq_w.alloc(h->n);
  }
  h->parts.alloc(2 * (size_t)lsq::kMaxGrid);
  h->counters.alloc(8); h->counters.zero(st);
  h->scal.alloc(lsq::S_NSLOT); h->scal.zero(st);
  h->hist_cap = std::max(h->opt.maxit, h->opt.fixed_iters) + 8;
  h->ahist.alloc(h->hist_cap); h->bhist.alloc(h->hist_cap);
  h->ctr.alloc(1);
  CK(cudaHostAlloc((void**)&h->pin, sizeof(double) * lsq::S_NSLOT, cudaHostAllocDefault));
  if (h->opt.time_kernels)
    for (auto& e : h->ev) CK(cudaEventCreate(&e));
  std::memset(h->pin, 0, sizeof(double) * lsq::S_NSLOT);
  phase.next("ls_setup: sparse-product copies and autotuning");
  job.join();
  if (job_failed) throw LsError(LS_ERR_OOM, "host memory for the sparse-product copies");
  h->sellA_src.upload(sa.src, st);
  h->sellB_src.upload(sb.src, st);
  h->sellA.nslices = sa.nslices;
  h->sellA_off.upload(sa.off, st); h->sellA_perm.upload(sa.perm, st);
  h->sellA_col.upload(sa.col, st); h->sellA_val.upload(sa.val, st);
  h->sellB.nslices = sb.nslices;
  h->sellB_off.upload(sb.off, st); h->sellB_perm.upload(sb.perm, st);
  h->sellB_col.upload(sb.col, st); h->sellB_val.upload(sb.val, st);
  if (nt_ok) {
    h->nt_lo.upload(nt.lo, st); h->nt_wid.upload(nt.wid, st);
    h->nt_as0.upload(nt.as0, st); h->nt_bs0.upload(nt.bs0, st);
    h->nt_aoff.upload(nt.aoff, st); h->nt_acol.upload(nt.acol, st); h->nt_aval.upload(nt.aval, st);
    h->nt_boff.upload(nt.boff, st); h->nt_brow.upload(nt.brow, st); h->nt_bval.upload(nt.bval, st);
    h->nt_bcid.upload(nt.bcid, st); h->nt_poff.upload(nt.poff, st);
    h->nt_asrc.upload(nt.asrc, st); h->nt_bsrc.upload(nt.bsrc, st);
    h->nt_cb0.upload(nt.cb_t0, st); h->nt_cb1.upload(nt.cb_t1, st);
    h->nt_part.alloc((size_t)nt.poff[nt.ntiles]);
    h->nt_tiles = nt.ntiles;
    h->nt_smem = nt.smem_doubles;
    const int64_t st6[6] = {nt.ntiles, (int64_t)nt.aval.size(), (int64_t)nt.bval.size(), nt.as0[nt.ntiles],
                            nt.bs0[nt.ntiles], nt.poff[nt.ntiles]};
    for (int k = 0; k < 6; ++k) h->nt_stats[k] = st6[k];
  }
  CK(cudaStreamSynchronize(st));  // the host copies go out of scope
  if (h->nt_tiles > 0 && !lsq::normal_tiles_prepare(ntiles(h))) release_normal_tiles(h);
  if (h->nt_tiles == 0 && h->opt.normal_product == 2)
    throw LsError(LS_ERR_UNSUPPORTED, "normal_product = 2: the row tiles do not fit a block's shared memory");
  if (h->opt.equilibrate) refresh_value_copies(h);  // the copies above hold the scaled values
  autotune_spmv(h);
  {
    int optin = 0;
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev));
    h->r.zero(st);
    choose_local_config(h, optin);
  }
  block_plan(h);
  CK(cudaStreamSynchronize(st));
  h->sinfo.t_setup = now_s() - t_begin;
  h->sinfo.bad_subdomain = -1;
  h->sinfo.lanes_csr = h->lanes_csr;
  h->sinfo.lanes_csc = h->lanes_csc;
  h->sinfo.normal_product = h->normal_kind;
  h->sinfo.local_config = h->local_cfg;
}

}  // namespace

namespace {

// Orders one call's device work, which runs on the handle's stream, between the work
// the caller queued on its own stream before the call and what it queues there after:
// an event recorded on the caller's stream that the handle's stream waits for at entry,
// and one recorded on the handle's stream that the caller's waits for at exit.
struct CallerOrder {
  ls_handle* h;
  cudaStream_t caller;
  bool joined = false;
  CallerOrder(ls_handle* h_, void* s) : h(h_), caller(static_cast<cudaStream_t>(s)) {
    if (caller == h->st) return;
    if (!h->ev_join) CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    CK(cudaEventRecord(h->ev_join, caller));
    CK(cudaStreamWaitEvent(h->st, h->ev_join, 0));
    joined = true;
  }
  ~CallerOrder() {
    if (joined && cudaEventRecord(h->ev_join, h->st) == cudaSuccess) cudaStreamWaitEvent(caller, h->ev_join, 0);
  }
};

}  // namespace

extern "C" {

void ls_default_options(ls_options* o) {
  if (!o) return;
  o->nev_max = 16;
  o->delta_rel = 1e-10;
  o->s_rel = 1e-8;
  o->factor_prec = LS_PREC_F64;
  o->maxit = 1000;
  o->coarse = 1;
  o->fixed_iters = 0;
  o->eig_maxit = 3000;
  o->eig_tol = 1e-11;
  o->use_graph = 1;
  o->time_kernels = 0;
  o->equilibrate = 0;
  o->variant = 0;
  o->solver = 0;
  o->restart = 100;
  o->spmv = 0;
  o->test_stall = 0;
  o->block_kernel = 0;
  o->normal_product = 0;
  o->normal_kernel = 0;
  o->local_config = 0;
}

const char* ls_last_error(void) { return g_err.c_str(); }

namespace {

ls_status setup_entry(int32_t nprob, const int64_t* m_off, const int64_t* n_off, int64_t m, int64_t n,
                      const int64_t* row_ptr, const int32_t* col, const double* val, int32_t nparts,
                      const int32_t* part, int overlap, double tau, const ls_options* opt, void* stream,
                      ls_handle** out) {
  if (out) *out = nullptr;
  return guarded([&]() -> ls_status {
    if (!out || !row_ptr || !part || (!col && m > 0) || (!val && m > 0))
      throw LsError(LS_ERR_INVALID, "null pointer argument");
    if (m < 1 || n < 1 || m < n) throw LsError(LS_ERR_INVALID, "need m >= n >= 1");
    if (nparts < 1 || nparts > n) throw LsError(LS_ERR_INVALID, "nparts must lie in [1, n]");
    if (overlap != 1) throw LsError(LS_ERR_UNSUPPORTED, "only overlap = 1 is defined for the splitting");
    std::unique_ptr<ls_handle> h(new ls_handle());
    ls_default_options(&h->opt);
    if (opt) h->opt = *opt;
    if (h->opt.factor_prec < 0 || h->opt.factor_prec > 2) throw LsError(LS_ERR_INVALID, "bad factor_prec");
    if (h->opt.maxit < 1 && h->opt.fixed_iters < 1) throw LsError(LS_ERR_INVALID, "maxit must be positive");
    if (h->opt.nev_max < 0) throw LsError(LS_ERR_INVALID, "nev_max must be >= 0");
    if (h->opt.variant < 0 || h->opt.variant > 2) throw LsError(LS_ERR_INVALID, "variant must be 0, 1 or 2");
    if (h->opt.solver < 0 || h->opt.solver > 2) throw LsError(LS_ERR_INVALID, "solver must be 0, 1 or 2");
    if (h->opt.variant == 2 && h->opt.solver != 2)
      throw LsError(LS_ERR_INVALID, "the deflated RAS variant is not symmetric: it needs solver = 2 (GMRES)");
    if (h->opt.solver == 2 && (h->opt.restart < 1 || h->opt.restart > 1000))
      throw LsError(LS_ERR_INVALID, "restart must lie in [1, 1000]");
    if (h->opt.test_stall != 0 && h->opt.test_stall != 1) throw LsError(LS_ERR_INVALID, "test_stall must be 0 or 1");
    if (h->opt.block_kernel < 0 || h->opt.block_kernel > 2) throw LsError(LS_ERR_INVALID, "block_kernel must be 0, 1 or 2");
    if (h->opt.normal_product < 0 || h->opt.normal_product > 2)
      throw LsError(LS_ERR_INVALID, "normal_product must be 0, 1 or 2");
    if (h->opt.local_config < 0 || h->opt.local_config > 3) throw LsError(LS_ERR_INVALID, "local_config must lie in [0, 3]");
    if (h->opt.normal_kernel < 0 || h->opt.normal_kernel > 4)
      throw LsError(LS_ERR_INVALID, "normal_kernel must lie in [0, 4]");
    if (h->opt.spmv != 0 && !lsq::valid_spmv_code(h->opt.spmv))
      throw LsError(LS_ERR_INVALID, "spmv must be 0 or a sparse-product kernel code");
    if (h->opt.variant != 0 && nprob > 1)
      throw LsError(LS_ERR_UNSUPPORTED, "the balanced and deflated variants are implemented for single-problem handles");
    if (!(tau < 1.0)) throw LsError(tau >= 1.0 ? LS_ERR_UNSUPPORTED : LS_ERR_INVALID,
                                    "tau >= 1 keeps the eigenvalue-1 cluster, which the device Lanczos cannot resolve");
    h->tau = tau;
    CK(cudaGetDevice(&h->dev));
    if (stream) {
      h->st = (cudaStream_t)stream;
    } else {
      CK(cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking));
      h->own_stream = true;
    }
    h->m = m; h->n = n; h->N = nparts;
    h->nprob = nprob;
    if (m_off && n_off) {
      h->h_m_off.assign(m_off, m_off + nprob + 1);
      h->h_n_off.assign(n_off, n_off + nprob + 1);
    } else {
      h->h_m_off = {0, m};
      h->h_n_off = {0, n};
    }
    h->coarse = h->opt.coarse != 0 && h->opt.nev_max > 0;
    h->sinfo.bad_subdomain = -1;
    try {
      do_setup(h.get(), row_ptr, col, val, part);
    } catch (...) {
      cudaStreamSynchronize(h->st);
      throw;
    }
    *out = h.release();
    return LS_OK;
  });
}

}  // namespace

ls_status ls_setup(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                   int32_t nparts, const int32_t* part, int overlap, double tau, const ls_options* opt, void* stream,
                   ls_handle** out) {
  return setup_entry(1, nullptr, nullptr, m, n, row_ptr, col, val, nparts, part, overlap, tau, opt, stream, out);
}

ls_status ls_setup_batched(int32_t nprob, const int64_t* m_off, const int64_t* n_off, const int64_t* row_ptr,
                           const int32_t* col, const double* val, int32_t nparts, const int32_t* part, int overlap,
                           double tau, const ls_options* opt, void* stream, ls_handle** out) {
  if (nprob < 1 || !m_off || !n_off) {
    if (out) *out = nullptr;
    g_err = "nprob must be positive and m_off, n_off non-null";
    return LS_ERR_INVALID;
  }
  return setup_entry(nprob, m_off, n_off, m_off[nprob], n_off[nprob], row_ptr, col, val, nparts, part, overlap, tau,
                     opt, stream, out);
}

ls_status ls_solve(ls_handle* h, const double* b, int nrhs, double rtol, double* x, ls_info* info, void* stream) {
  return guarded([&]() -> ls_status {
    if (!h || !b || !x || nrhs < 1) throw LsError(LS_ERR_INVALID, "null handle/pointer or nrhs < 1");
    if (!(rtol > 0) && h->opt.fixed_iters <= 0) throw LsError(LS_ERR_INVALID, "rtol must be positive");
    CK(cudaSetDevice(h->dev));
    Phase phase("ls_solve");
    CallerOrder order(h, stream);
    if (nrhs > 1 || h->nprob > 1) {
      if (h->opt.solver != 0)
        throw LsError(LS_ERR_UNSUPPORTED, "the LSQR and GMRES outer solvers take one right-hand side of a single "
                                          "problem");
      return block_solve(h, b, nrhs, rtol, x, info);
    }
    ls_status last = LS_OK;
    for (int k = 0; k < nrhs; ++k) {
      // b' = P b for the row-reordered device matrix
      CK(cudaMemcpyAsync(h->q.p, b + (int64_t)k * h->m, sizeof(double) * h->m, cudaMemcpyDefault, h->st));
      lsq::launch_gather(h->m, h->perm.p, h->q.p, h->bv.p, h->st);
      ls_status s = h->opt.solver == 1 ? lsqr_core(h, rtol, info)
                  : h->opt.solver == 2 ? gmres_core(h, rtol, info) : solve_core(h, 0, rtol, info);
      CK(cudaMemcpyAsync(x + (int64_t)k * h->n, h->x.p, sizeof(double) * h->n, cudaMemcpyDefault, h->st));
      CK(cudaStreamSynchronize(h->st));
      if (s != LS_OK) last = s;
    }
    return last;
  });
}

ls_status ls_backward(ls_handle* h, const double* b, const double* x, const double* grad_x, int nrhs, double rtol,
                      double* grad_b, double* grad_vals, ls_info* info, void* stream) {
  return guarded([&]() -> ls_status {
    if (!h || !b || !x || !grad_x || nrhs < 1) throw LsError(LS_ERR_INVALID, "null handle/pointer or nrhs < 1");
    CK(cudaSetDevice(h->dev));
    Phase phase("ls_backward");
    CallerOrder order(h, stream);
    if (h->nprob > 1) return block_backward(h, b, x, grad_x, nrhs, rtol, grad_b, grad_vals, info);
    cudaStream_t st = h->st;
    ls_status last = LS_OK;
    DevBuf<double> xk, lam, mu, tmp, gperm, gout;
    xk.alloc(h->n); lam.alloc(h->n); mu.alloc(h->m); tmp.alloc(h->m);
    if (grad_vals) { gperm.alloc(h->nnz); gout.alloc(h->nnz); }
    for (int k = 0; k < nrhs; ++k) {
      CK(cudaMemcpyAsync(h->tv.p, grad_x + (int64_t)k * h->n, sizeof(double) * h->n, cudaMemcpyDefault, st));
      ls_status s = solve_core(h, 1, rtol, info);
      if (s != LS_OK) last = s;
      CK(cudaMemcpyAsync(lam.p, h->x.p, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, st));
      lsq::launch_spmv_csr(csr(h), lam.p, mu.p, h->lanes_csr, h->grid_csr, st);  // mu' = A' lambda
      if (grad_b) {  // grad_b = A lambda = P^T mu'
        lsq::launch_scatter_idx(h->m, h->perm.p, nullptr, mu.p, tmp.p, 0, st);
        CK(cudaMemcpyAsync(grad_b + (int64_t)k * h->m, tmp.p, sizeof(double) * h->m, cudaMemcpyDefault, st));
      }
      if (grad_vals) {
        CK(cudaMemcpyAsync(xk.p, x + (int64_t)k * h->n, sizeof(double) * h->n, cudaMemcpyDefault, st));
        CK(cudaMemcpyAsync(tmp.p, b + (int64_t)k * h->m, sizeof(double) * h->m, cudaMemcpyDefault, st));
        lsq::launch_gather(h->m, h->perm.p, tmp.p, h->bv.p, st);  // b' = P b
        lsq::launch_spmv_csr(csr(h), xk.p, h->q.p, h->lanes_csr, h->grid_csr, st);
        lsq::launch_axpby(h->m, 1.0, h->bv.p, -1.0, h->q.p, h->q.p, st);  // rho' = b' - A' x
        lsq::launch_grad_vals(csr(h), h->q.p, lam.p, mu.p, xk.p, gperm.p, k > 0 ? 1 : 0, st);
      }
      check_launch("backward");
    }
    if (grad_vals) {  // entries of A' back to the caller's CSR order
      lsq::launch_scatter_idx(h->nnz, nullptr, h->entmap.p, gperm.p, gout.p, 0, st);
      CK(cudaMemcpyAsync(grad_vals, gout.p, sizeof(double) * h->nnz, cudaMemcpyDefault, st));
    }
    CK(cudaStreamSynchronize(st));
    check_launch("backward");
    return last;
  });
}

ls_status ls_update_values(ls_handle* h, const double* val) {
  return guarded([&]() -> ls_status {
    if (!h || !val) throw LsError(LS_ERR_INVALID, "null argument");
    CK(cudaSetDevice(h->dev));
    cudaStream_t st = h->st;
    const int64_t nnz = h->nnz;
    DevBuf<double> tmp;
    tmp.alloc(nnz);
    CK(cudaMemcpyAsync(tmp.p, val, sizeof(double) * nnz, cudaMemcpyDefault, st));
    lsq::launch_gather64(nnz, h->entmap.p, tmp.p, h->val.p, st);  // A' = P A, CSR
    refresh_value_copies(h);
    CK(cudaStreamSynchronize(st));
    check_launch("value update");
    return LS_OK;
  });
}

void ls_free(ls_handle* h) { delete h; }

ls_status ls_handle_info(const ls_handle* h, ls_info* info) {
  if (!h || !info) return LS_ERR_INVALID;
  *info = h->sinfo;
  return LS_OK;
}

ls_status ls_apply_preconditioner(ls_handle* h, const double* r, double* z, int which) {
  return guarded([&]() -> ls_status {
    if (!h || !r || !z || which < 0 || which > 2) throw LsError(LS_ERR_INVALID, "bad arguments");
    if (h->nprob > 1) throw LsError(LS_ERR_UNSUPPORTED, "single-vector preconditioner apply on a batched handle");
    CK(cudaSetDevice(h->dev));
    CK(cudaMemsetAsync(h->scal.p + lsq::S_ERR, 0, sizeof(double), h->st));
    CK(cudaMemcpyAsync(h->tv.p, r, sizeof(double) * h->n, cudaMemcpyDefault, h->st));
    if (which == 2) {
      // the coarse term Q r alone
      if (h->coarse && h->n0 > 0) coarse_term(h, h->tv.p, h->w.p);
      else CK(cudaMemsetAsync(h->w.p, 0, sizeof(double) * h->n, h->st));
    } else {
      precond(h, h->tv.p, h->w.p, which, false, false);
    }
    CK(cudaMemcpyAsync(z, h->w.p, sizeof(double) * h->n, cudaMemcpyDefault, h->st));
    CK(cudaStreamSynchronize(h->st));
    check_launch("preconditioner");
    double err = 0.0;
    CK(cudaMemcpy(&err, h->scal.p + lsq::S_ERR, sizeof(double), cudaMemcpyDeviceToHost));
    if (err == lsq::kErrBounds)
      throw LsError(LS_ERR_INVALID, "an index out of range was met (bounds-checked build) in the preconditioner apply");
    if (err != 0.0) throw LsError(LS_ERR_DEVICE_TIMEOUT, "a bounded wait in the local-solve kernel gave up");
    return LS_OK;
  });
}

ls_status ls_apply_normal(ls_handle* h, const double* p, double* w) {
  return guarded([&]() -> ls_status {
    if (!h || !p || !w) throw LsError(LS_ERR_INVALID, "bad arguments");
    CK(cudaSetDevice(h->dev));
    CK(cudaMemcpyAsync(h->tv.p, p, sizeof(double) * h->n, cudaMemcpyDefault, h->st));
    normal_product(h, h->tv.p, h->w.p, nullptr, lsq::DotSite{}, h->st);
    CK(cudaMemcpyAsync(w, h->w.p, sizeof(double) * h->n, cudaMemcpyDefault, h->st));
    CK(cudaStreamSynchronize(h->st));
    check_launch("normal-equations product");
    return LS_OK;
  });
}

ls_status ls_query(const ls_handle* h, int kind, int i, void* out, int64_t cap) {
  return guarded([&]() -> ls_status {
    if (!h || !out) throw LsError(LS_ERR_INVALID, "null argument");
    const int N = h->N;
    auto need = [&](int64_t k) {
      if (cap < k) throw LsError(LS_ERR_INVALID, "output capacity too small: need " + std::to_string(k));
    };
    if (kind == LS_Q_SIZES) {
      need((int64_t)N * 4);
      int64_t* o = (int64_t*)out;
      for (int s = 0; s < N; ++s) {
        o[4 * s + 0] = h->h_om_off[s + 1] - h->h_om_off[s];
        o[4 * s + 1] = h->h_nI[s];
        o[4 * s + 2] = h->h_xi_off[s + 1] - h->h_xi_off[s];
        o[4 * s + 3] = h->h_k.empty() ? 0 : h->h_k[s];
      }
      return LS_OK;
    }
    if (kind == LS_Q_STORAGE) {
      need(8);
      int64_t* o = (int64_t*)out;
      int64_t zel = 0;
      for (int s = 0; s < N; ++s) zel += (int64_t)(h->h_k.empty() ? 0 : h->h_k[s]) * h->h_nI[s];
      o[0] = h->fac_elems; o[1] = h->total_local; o[2] = h->total_blocks; o[3] = zel;
      o[4] = h->n0; o[5] = h->n0p; o[6] = h->nnz; o[7] = h->prec;
      return LS_OK;
    }
    if (kind == LS_Q_NORMAL) {
      need(12);
      int64_t* o = (int64_t*)out;
      for (int k = 0; k < 6; ++k) o[k] = h->nt_tiles > 0 ? h->nt_stats[k] : 0;
      o[6] = h->nt_tiles > 0 ? h->nt_cfg : 0;
      for (int k = 0; k < 5; ++k) o[7 + k] = (int64_t)(h->nt_ms[k] * 1e6f);
      return LS_OK;
    }
    if (kind == LS_Q_BATCH) {
      const int64_t k = (int64_t)h->blk.h_its.size();
      if (k == 0) throw LsError(LS_ERR_INVALID, "no multi right-hand-side solve has run");
      need(2 * k);
      double* o = (double*)out;
      for (int64_t a = 0; a < k; ++a) {
        o[a] = h->blk.h_its[a];
        o[k + a] = h->blk.h_rel[a];
      }
      return LS_OK;
    }
    if (kind == LS_Q_EIGSTEPS) {
      need(N);
      for (int s = 0; s < N; ++s) ((int32_t*)out)[s] = h->h_steps.empty() ? 0 : h->h_steps[s];
      return LS_OK;
    }
    if (i < 0 || i >= N) throw LsError(LS_ERR_INVALID, "subdomain index out of range");
    if (kind == LS_Q_OMEGA) {
      const int64_t k = h->h_om_off[i + 1] - h->h_om_off[i];
      need(k);
      std::memcpy(out, h->h_om_paper.data() + h->h_om_off[i], sizeof(int32_t) * k);
    } else if (kind == LS_Q_XI) {
      const int64_t k = h->h_xi_off[i + 1] - h->h_xi_off[i];
      need(k);
      // internal rows are those of A' = P A: report the caller's row numbers, ascending
      int32_t* o = (int32_t*)out;
      for (int64_t a = 0; a < k; ++a) o[a] = h->h_perm[h->h_xi[h->h_xi_off[i] + a]];
      std::sort(o, o + k);
    } else if (kind == LS_Q_EIGVALS) {
      if (h->h_lam.empty()) throw LsError(LS_ERR_INVALID, "no eigensolve was run");
      const int64_t ni = h->h_om_off[i + 1] - h->h_om_off[i];
      const int64_t k = std::min<int64_t>(h->kwant_cap, ni);
      need(k);
      std::memcpy(out, h->h_lam.data() + (size_t)i * h->kwant_cap, sizeof(double) * k);
    } else if (kind == LS_Q_ZBAR) {
      const int64_t k = (int64_t)h->h_k[i] * h->h_nI[i];
      need(k);
      if (k) {
        int64_t off = 0;
        for (int s = 0; s < i; ++s) off += (int64_t)h->h_k[s] * h->h_nI[s];
        CK(cudaSetDevice(h->dev));
        CK(cudaMemcpy(out, h->Z.p + off, sizeof(double) * k, cudaMemcpyDeviceToHost));
      }
    } else {
      throw LsError(LS_ERR_INVALID, "unknown query kind");
    }
    return LS_OK;
  });
}

ls_status ls_build_index_sets(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col, int32_t nparts,
                              const int32_t* part, int64_t* omega_total, int64_t* xi_total, int64_t* omega_off,
                              int32_t* omega, int32_t* n_interior, int64_t* xi_off, int32_t* xi) {
  return guarded([&]() -> ls_status {
    if (!row_ptr || !col || !part) throw LsError(LS_ERR_INVALID, "null pointer argument");
    lsq::HostSets hs;
    std::string err = lsq::build_host_sets(m, n, row_ptr, col, nparts, part, false, hs);
    if (!err.empty()) throw LsError(LS_ERR_INVALID, err);
    if (omega_total) *omega_total = hs.om_off[nparts];
    if (xi_total) *xi_total = hs.xi_off[nparts];
    if (omega) {
      std::memcpy(omega, hs.om_paper.data(), sizeof(int32_t) * hs.om_paper.size());
      std::memcpy(omega_off, hs.om_off.data(), sizeof(int64_t) * hs.om_off.size());
      std::memcpy(n_interior, hs.nI.data(), sizeof(int32_t) * hs.nI.size());
      std::memcpy(xi_off, hs.xi_off.data(), sizeof(int64_t) * hs.xi_off.size());
      std::memcpy(xi, hs.xi.data(), sizeof(int32_t) * hs.xi.size());
    }
    return LS_OK;
  });
}

}  // extern "C"
