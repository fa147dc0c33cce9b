// Host construction of the index sets (Section 3, Algorithm 1 steps 3-5) and of the
// storage plans used by the device kernels.
#include "host_sets.h"

#include <algorithm>
#include <atomic>
#include <thread>

namespace lsq {

namespace {

struct Local {
  std::vector<int32_t> om;     // ascending
  std::vector<uint8_t> isint;
  std::vector<int32_t> paper;  // [interior ascending, overlap ascending]
  std::vector<int32_t> xi;     // ascending
  std::vector<int32_t> tf;     // per block row
  int32_t nI = 0;
};

template <class F>
void parallel_for(int count, F&& f) {
  unsigned hw = std::thread::hardware_concurrency();
  int nt = (int)std::max(1u, std::min(hw ? hw : 4u, 32u));
  nt = std::min(nt, std::max(1, count));
  std::atomic<int> next(0);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t]() {
      f.init(t);
      for (;;) {
        int i = next.fetch_add(1);
        if (i >= count) break;
        f.run(t, i);
      }
    });
  for (auto& x : th) x.join();
}

}  // namespace

void build_sell(int64_t nrows, const int64_t* ptr, const int32_t* idx, const double* val, int window,
                SellHost& out) {
  out = SellHost();
  const int64_t ns = (nrows + 31) / 32;
  out.nslices = ns;
  out.perm.assign(ns * 32, -1);
  std::vector<int32_t> order(nrows);
  for (int64_t r = 0; r < nrows; ++r) order[r] = (int32_t)r;
  for (int64_t w0 = 0; w0 < nrows; w0 += window) {
    const int64_t w1 = std::min(nrows, w0 + window);
    std::stable_sort(order.begin() + w0, order.begin() + w1, [&](int32_t a, int32_t b) {
      return (ptr[a + 1] - ptr[a]) > (ptr[b + 1] - ptr[b]);
    });
  }
  out.off.assign(ns + 1, 0);
  for (int64_t s = 0; s < ns; ++s) {
    int64_t wmax = 0;
    for (int l = 0; l < 32; ++l) {
      const int64_t k = s * 32 + l;
      if (k < nrows) {
        out.perm[k] = order[k];
        wmax = std::max(wmax, ptr[order[k] + 1] - ptr[order[k]]);
      }
    }
    out.off[s + 1] = out.off[s] + 32 * wmax;
  }
  out.col.assign(out.off[ns], 0);
  out.val.assign(out.off[ns], 0.0);
  out.src.assign(out.off[ns], -1);
  for (int64_t s = 0; s < ns; ++s)
    for (int l = 0; l < 32; ++l) {
      const int32_t r = out.perm[s * 32 + l];
      if (r < 0) continue;
      for (int64_t e = ptr[r], k = 0; e < ptr[r + 1]; ++e, ++k) {
        out.col[out.off[s] + 32 * k + l] = idx[e];
        out.val[out.off[s] + 32 * k + l] = val[e];
        out.src[out.off[s] + 32 * k + l] = e;
      }
    }
}

void order_rows_by_first_column(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col,
                                std::vector<int32_t>& perm) {
  // stable counting sort on the key col[row_ptr[r]] (n for an empty row)
  std::vector<int64_t> cnt(n + 2, 0);
  auto key = [&](int64_t r) -> int64_t { return row_ptr[r + 1] > row_ptr[r] ? col[row_ptr[r]] : n; };
  for (int64_t r = 0; r < m; ++r) cnt[key(r) + 1]++;
  for (int64_t k = 0; k <= n; ++k) cnt[k + 1] += cnt[k];
  perm.assign(m, 0);
  for (int64_t r = 0; r < m; ++r) perm[cnt[key(r)]++] = (int32_t)r;
}

std::string validate_inputs(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col, int N,
                            const int32_t* part) {
  if (m < 1 || n < 1) return "m and n must be positive";
  if (N < 1 || N > n) return "nparts must lie in [1, n]";
  if (n > INT32_MAX || m > INT32_MAX) return "m and n must fit in int32";
  if (row_ptr[0] != 0) return "row_ptr[0] must be 0";
  for (int64_t r = 0; r < m; ++r)
    if (row_ptr[r + 1] < row_ptr[r]) return "row_ptr must be nondecreasing";
  for (int64_t r = 0; r < m; ++r) {
    for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
      int32_t c = col[e];
      if (c < 0 || c >= n) return "column index out of range in row " + std::to_string(r);
      if (e > row_ptr[r] && c <= col[e - 1])
        return "column indices must be strictly increasing within row " + std::to_string(r);
    }
  }
  for (int64_t j = 0; j < n; ++j)
    if (part[j] < 0 || part[j] >= N) return "part[" + std::to_string(j) + "] out of range";
  return std::string();
}

std::string validate_batch(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col, int N,
                           const int32_t* part, int nprob, const int64_t* m_off, const int64_t* n_off,
                           std::vector<int32_t>& N_off, std::vector<int32_t>& prob_of_sub) {
  if (nprob < 1) return "nprob must be positive";
  if (m_off[0] != 0 || n_off[0] != 0 || m_off[nprob] != m || n_off[nprob] != n)
    return "problem offsets must start at 0 and end at m and n";
  for (int q = 0; q < nprob; ++q) {
    const int64_t mq = m_off[q + 1] - m_off[q], nq = n_off[q + 1] - n_off[q];
    if (nq < 1 || mq < nq) return "problem " + std::to_string(q) + " needs m_q >= n_q >= 1";
    for (int64_t r = m_off[q]; r < m_off[q + 1]; ++r)
      for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e)
        if (col[e] < n_off[q] || col[e] >= n_off[q + 1])
          return "row " + std::to_string(r) + " of problem " + std::to_string(q) + " has a column outside it";
  }
  N_off.assign(nprob + 1, 0);
  prob_of_sub.assign(N, -1);
  for (int q = 0; q < nprob; ++q) {
    int lo = INT32_MAX, hi = -1;
    for (int64_t j = n_off[q]; j < n_off[q + 1]; ++j) {
      lo = std::min(lo, part[j]);
      hi = std::max(hi, part[j]);
    }
    if (lo != N_off[q])
      return "subdomain ids of problem " + std::to_string(q) + " must start at " + std::to_string(N_off[q]);
    N_off[q + 1] = hi + 1;
    for (int i = lo; i <= hi; ++i) prob_of_sub[i] = q;
  }
  if (N_off[nprob] != N) return "subdomain ids must run through 0 .. nparts-1 in problem order";
  for (int64_t j = 0; j < n; ++j) {
    const int q = prob_of_sub[part[j]];
    if (j < n_off[q] || j >= n_off[q + 1]) return "subdomain " + std::to_string(part[j]) + " spans two problems";
  }
  return std::string();
}

std::string build_host_sets(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col,
                            int N, const int32_t* part, bool with_pairs, HostSets& hs) {
  if (m < 1 || n < 1) return "m and n must be positive";
  if (N < 1 || N > n) return "nparts must lie in [1, n]";
  if (n > INT32_MAX || m > INT32_MAX) return "m and n must fit in int32";
  if (row_ptr[0] != 0) return "row_ptr[0] must be 0";
  for (int64_t r = 0; r < m; ++r)
    if (row_ptr[r + 1] < row_ptr[r]) return "row_ptr must be nondecreasing";
  const int64_t nnz = row_ptr[m];
  for (int64_t r = 0; r < m; ++r) {
    for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
      int32_t c = col[e];
      if (c < 0 || c >= n) return "column index out of range in row " + std::to_string(r);
      if (e > row_ptr[r] && c <= col[e - 1])
        return "column indices must be strictly increasing within row " + std::to_string(r);
    }
  }
  for (int64_t j = 0; j < n; ++j)
    if (part[j] < 0 || part[j] >= N) return "part[" + std::to_string(j) + "] out of range";

  hs = HostSets();
  hs.m = m; hs.n = n; hs.nnz = nnz; hs.N = N;

  // CSC of the pattern (rows ascending inside each column) and the CSR slot of each entry.
  hs.csc_ptr.assign(n + 1, 0);
  for (int64_t e = 0; e < nnz; ++e) hs.csc_ptr[col[e] + 1]++;
  for (int64_t j = 0; j < n; ++j) hs.csc_ptr[j + 1] += hs.csc_ptr[j];
  hs.csc_row.resize(nnz);
  hs.csc_perm.resize(nnz);
  {
    std::vector<int64_t> pos(hs.csc_ptr.begin(), hs.csc_ptr.end() - 1);
    for (int64_t r = 0; r < m; ++r)
      for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
        int64_t s = pos[col[e]]++;
        hs.csc_row[s] = (int32_t)r;
        hs.csc_perm[s] = e;
      }
  }

  // Interior sets Omega_I,i (ascending) by counting sort of the partition.
  std::vector<int64_t> ioff(N + 1, 0);
  for (int64_t j = 0; j < n; ++j) ioff[part[j] + 1]++;
  for (int i = 0; i < N; ++i) ioff[i + 1] += ioff[i];
  for (int i = 0; i < N; ++i)
    if (ioff[i + 1] == ioff[i]) return "subdomain " + std::to_string(i) + " owns no column";
  std::vector<int32_t> interior(n);
  hs.jj_of.resize(n);
  {
    std::vector<int64_t> pos(ioff.begin(), ioff.end() - 1);
    for (int64_t j = 0; j < n; ++j) {
      int p = part[j];
      hs.jj_of[j] = (int32_t)(pos[p] - ioff[p]);
      interior[pos[p]++] = (int32_t)j;
    }
  }

  std::vector<Local> loc(N);
  struct Worker {
    const int64_t* row_ptr; const int32_t* col; const int32_t* part;
    const HostSets* hs; const std::vector<int64_t>* ioff; const std::vector<int32_t>* interior;
    std::vector<Local>* loc; int64_t m, n;
    std::vector<std::vector<int32_t>> row_stamp, col_stamp, col_pos;
    void init(int t) {
      if ((int)row_stamp.size() <= t) return;
      row_stamp[t].assign(m, -1);
      col_stamp[t].assign(n, -1);
      col_pos[t].assign(n, -1);
    }
    void run(int t, int i) {
      auto& rs = row_stamp[t];
      auto& cs = col_stamp[t];
      auto& cp = col_pos[t];
      Local& L = (*loc)[i];
      const int64_t b0 = (*ioff)[i], b1 = (*ioff)[i + 1];
      // Xi_i: rows with a stored entry in an interior column (Algorithm 1, step 3).
      for (int64_t a = b0; a < b1; ++a) {
        int32_t j = (*interior)[a];
        for (int64_t e = hs->csc_ptr[j]; e < hs->csc_ptr[j + 1]; ++e) {
          int32_t r = hs->csc_row[e];
          if (rs[r] != i) { rs[r] = i; L.xi.push_back(r); }
        }
      }
      std::sort(L.xi.begin(), L.xi.end());
      // Omega_i: all columns of A(Xi_i, :), plus interior columns without entries.
      for (int32_t r : L.xi)
        for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
          int32_t c = col[e];
          if (cs[c] != i) { cs[c] = i; L.om.push_back(c); }
        }
      for (int64_t a = b0; a < b1; ++a) {
        int32_t j = (*interior)[a];
        if (cs[j] != i) { cs[j] = i; L.om.push_back(j); }
      }
      std::sort(L.om.begin(), L.om.end());
      const int64_t ni = (int64_t)L.om.size();
      L.isint.resize(ni);
      L.nI = (int32_t)(b1 - b0);
      L.paper.reserve(ni);
      for (int64_t a = b0; a < b1; ++a) L.paper.push_back((*interior)[a]);
      for (int64_t k = 0; k < ni; ++k) {
        int32_t c = L.om[k];
        cp[c] = (int32_t)k;
        L.isint[k] = (part[c] == i);
        if (part[c] != i) L.paper.push_back(c);
      }
      // Envelope of C_ii = A(:, Omega_i)^T A(:, Omega_i): first coupled local column
      // of every local row (Cholesky fill stays to the right of it).
      const int64_t nb = (ni + kTile - 1) / kTile;
      L.tf.assign(nb, 0);
      for (int64_t b = 0; b < nb; ++b) {
        int64_t f = b * kTile;
        for (int64_t k = b * kTile; k < std::min(ni, (b + 1) * kTile); ++k) {
          int32_t g = L.om[k];
          for (int64_t e = hs->csc_ptr[g]; e < hs->csc_ptr[g + 1]; ++e) {
            int32_t r = hs->csc_row[e];
            for (int64_t e2 = row_ptr[r]; e2 < row_ptr[r + 1]; ++e2) {
              int32_t c = col[e2];
              if (cs[c] == i && cp[c] < f) f = cp[c];
            }
          }
        }
        L.tf[b] = (int32_t)(f / kTile);
      }
    }
  } w;
  w.row_ptr = row_ptr; w.col = col; w.part = part; w.hs = &hs; w.ioff = &ioff;
  w.interior = &interior; w.loc = &loc; w.m = m; w.n = n;
  {
    unsigned hw = std::thread::hardware_concurrency();
    int nt = (int)std::max(1u, std::min(hw ? hw : 4u, 32u));
    w.row_stamp.resize(nt); w.col_stamp.resize(nt); w.col_pos.resize(nt);
  }
  parallel_for(N, w);

  // Concatenate the per-subdomain results in subdomain order.
  hs.om_off.assign(N + 1, 0);
  hs.xi_off.assign(N + 1, 0);
  hs.blk_off.assign(N + 1, 0);
  hs.int_off = ioff;
  hs.nI.resize(N);
  for (int i = 0; i < N; ++i) {
    hs.om_off[i + 1] = hs.om_off[i] + (int64_t)loc[i].om.size();
    hs.xi_off[i + 1] = hs.xi_off[i] + (int64_t)loc[i].xi.size();
    hs.blk_off[i + 1] = hs.blk_off[i] + (int64_t)loc[i].tf.size();
    hs.nI[i] = loc[i].nI;
    hs.max_nb = std::max(hs.max_nb, (int)loc[i].tf.size());
    hs.max_ni = std::max(hs.max_ni, (int64_t)loc[i].om.size());
  }
  hs.om_glob.resize(hs.om_off[N]);
  hs.om_int.resize(hs.om_off[N]);
  hs.om_paper.resize(hs.om_off[N]);
  hs.xi.resize(hs.xi_off[N]);
  hs.blk_tf.resize(hs.blk_off[N]);
  hs.blk_poff.resize(hs.blk_off[N]);
  hs.int_loc.resize(ioff[N]);
  int64_t poff = 0;
  for (int i = 0; i < N; ++i) {
    const Local& L = loc[i];
    std::copy(L.om.begin(), L.om.end(), hs.om_glob.begin() + hs.om_off[i]);
    std::copy(L.isint.begin(), L.isint.end(), hs.om_int.begin() + hs.om_off[i]);
    std::copy(L.paper.begin(), L.paper.end(), hs.om_paper.begin() + hs.om_off[i]);
    std::copy(L.xi.begin(), L.xi.end(), hs.xi.begin() + hs.xi_off[i]);
    int64_t q = ioff[i];
    for (size_t k = 0; k < L.om.size(); ++k)
      if (L.isint[k]) hs.int_loc[q++] = (int32_t)k;
    for (size_t b = 0; b < L.tf.size(); ++b) {
      hs.blk_tf[hs.blk_off[i] + b] = L.tf[b];
      hs.blk_poff[hs.blk_off[i] + b] = poff;
      poff += (int64_t)kTile * ((int64_t)b - L.tf[b] + 1) * kTile;
    }
  }
  hs.fac_elems = poff;

  // Transposed scatter map (deterministic order: ascending subdomain).
  hs.map_ptr.assign(n + 1, 0);
  for (int64_t e = 0; e < hs.om_off[N]; ++e) hs.map_ptr[hs.om_glob[e] + 1]++;
  for (int64_t j = 0; j < n; ++j) hs.map_ptr[j + 1] += hs.map_ptr[j];
  hs.map_idx.resize(hs.om_off[N]);
  {
    std::vector<int64_t> pos(hs.map_ptr.begin(), hs.map_ptr.end() - 1);
    for (int64_t e = 0; e < hs.om_off[N]; ++e) hs.map_idx[pos[hs.om_glob[e]]++] = e;
  }

  if (with_pairs) {
    // Rows shared by Xi_i and Xi_j: per row, the (subdomain, position) list.
    std::vector<int64_t> rptr(m + 1, 0);
    for (int64_t e = 0; e < hs.xi_off[N]; ++e) rptr[hs.xi[e] + 1]++;
    for (int64_t r = 0; r < m; ++r) rptr[r + 1] += rptr[r];
    std::vector<int32_t> rsub(hs.xi_off[N]), rpos(hs.xi_off[N]);
    {
      std::vector<int64_t> pos(rptr.begin(), rptr.end() - 1);
      for (int i = 0; i < N; ++i)
        for (int64_t a = hs.xi_off[i]; a < hs.xi_off[i + 1]; ++a) {
          int64_t s = pos[hs.xi[a]]++;
          rsub[s] = i;
          rpos[s] = (int32_t)(a - hs.xi_off[i]);
        }
    }
    std::vector<int64_t> keys;
    for (int64_t r = 0; r < m; ++r)
      for (int64_t a = rptr[r]; a < rptr[r + 1]; ++a)
        for (int64_t b = a; b < rptr[r + 1]; ++b) keys.push_back((int64_t)rsub[a] * N + rsub[b]);
    std::vector<int64_t> uk(keys);
    std::sort(uk.begin(), uk.end());
    uk.erase(std::unique(uk.begin(), uk.end()), uk.end());
    const int64_t np = (int64_t)uk.size();
    hs.pair_i.resize(np); hs.pair_j.resize(np);
    for (int64_t p = 0; p < np; ++p) { hs.pair_i[p] = (int32_t)(uk[p] / N); hs.pair_j[p] = (int32_t)(uk[p] % N); }
    hs.pair_off.assign(np + 1, 0);
    std::vector<int64_t> kid(keys.size());
    for (size_t t = 0; t < keys.size(); ++t) {
      kid[t] = std::lower_bound(uk.begin(), uk.end(), keys[t]) - uk.begin();
      hs.pair_off[kid[t] + 1]++;
    }
    for (int64_t p = 0; p < np; ++p) hs.pair_off[p + 1] += hs.pair_off[p];
    hs.pair_pi.resize(keys.size()); hs.pair_pj.resize(keys.size());
    std::vector<int64_t> pos(hs.pair_off.begin(), hs.pair_off.end() - 1);
    size_t t = 0;
    for (int64_t r = 0; r < m; ++r)
      for (int64_t a = rptr[r]; a < rptr[r + 1]; ++a)
        for (int64_t b = a; b < rptr[r + 1]; ++b, ++t) {
          int64_t s = pos[kid[t]]++;
          hs.pair_pi[s] = rpos[a];
          hs.pair_pj[s] = rpos[b];
        }
  }
  return std::string();
}

}  // namespace lsq
