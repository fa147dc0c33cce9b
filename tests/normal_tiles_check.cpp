// Host check of the row-tile plan of the one-pass normal product (normal_tiles.cpp):
// for several matrices, the plan's invariants (every stored entry once in each copy,
// windows within the cap, the reduction table covering every window) and a plain
// emulation of the two tile sweeps and the per-column reduction against w = A^T (A p)
// computed from its definition.  Prints one line per case; exit code 0 when all pass.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "../paper_2107_09006_gb300/csrc/normal_tiles.h"

namespace {

struct Csr {
  int64_t m = 0, n = 0;
  std::vector<int64_t> rp{0};
  std::vector<int32_t> col;
  std::vector<double> val;
  void add_row(std::vector<int32_t> cols, std::mt19937_64& g) {
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    std::normal_distribution<double> nd;
    for (int32_t c : cols) {
      col.push_back(c);
      val.push_back(nd(g));
    }
    rp.push_back((int64_t)col.size());
    ++m;
  }
};

// rows of k entries within `radius` columns of a centre that walks across [0, n), plus
// empty rows every `empty_every` rows and no entries in columns [hole_lo, hole_hi)
Csr banded(int64_t n, int64_t m, int k, int radius, int empty_every, int hole_lo, int hole_hi, uint64_t seed) {
  std::mt19937_64 g(seed);
  Csr A;
  A.n = n;
  for (int64_t r = 0; r < m; ++r) {
    std::vector<int32_t> cols;
    if (!(empty_every > 0 && r % empty_every == 0)) {
      const int64_t centre = r * n / m;
      for (int t = 0; t < k; ++t) {
        int64_t c = centre + (int64_t)(g() % (2 * radius + 1)) - radius;
        c = std::min<int64_t>(std::max<int64_t>(c, 0), n - 1);
        if (c >= hole_lo && c < hole_hi) continue;
        cols.push_back((int32_t)c);
      }
    }
    A.add_row(cols, g);
  }
  return A;
}

std::vector<double> normal_product(const Csr& A, const std::vector<double>& p) {
  std::vector<double> q(A.m, 0.0), w(A.n, 0.0);
  for (int64_t r = 0; r < A.m; ++r)
    for (int64_t e = A.rp[r]; e < A.rp[r + 1]; ++e) q[r] += A.val[e] * p[A.col[e]];
  for (int64_t r = 0; r < A.m; ++r)
    for (int64_t e = A.rp[r]; e < A.rp[r + 1]; ++e) w[A.col[e]] += A.val[e] * q[r];
  return w;
}

// the two sweeps of one tile and the per-column sum, as the kernels order them
std::vector<double> tiles_product(const lsq::NormalTilesHost& T, int64_t n, const std::vector<double>& p,
                                  const char** why) {
  std::vector<double> part((size_t)T.poff[T.ntiles], 0.0);
  for (int t = 0; t < T.ntiles; ++t) {
    const int W = T.wid[t];
    const int R = (T.as0[t + 1] - T.as0[t]) * 32;
    if (((W + 1) & ~1) + R > T.smem_doubles) { *why = "tile exceeds its shared-memory size"; return {}; }
    std::vector<double> pw(W), sv(R, 0.0);
    for (int i = 0; i < W; ++i) pw[i] = p[T.lo[t] + i];
    for (int s = T.as0[t]; s < T.as0[t + 1]; ++s) {
      const int64_t e0 = T.aoff[s];
      const int K = (int)((T.aoff[s + 1] - e0) / 32);
      for (int l = 0; l < 32; ++l) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k) {
          const int c = T.acol[e0 + 32 * k + l];
          if (c >= std::max(W, 1)) { *why = "row-copy column outside the window"; return {}; }
          acc = std::fma(T.aval[e0 + 32 * k + l], W ? pw[c] : 0.0, acc);
        }
        sv[(s - T.as0[t]) * 32 + l] = acc;
      }
    }
    std::vector<int> seen(W, 0);
    for (int s = T.bs0[t]; s < T.bs0[t + 1]; ++s) {
      const int64_t e0 = T.boff[s];
      const int K = (int)((T.boff[s + 1] - e0) / 32);
      for (int l = 0; l < 32; ++l) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k) {
          const int j = T.brow[e0 + 32 * k + l];
          if (j >= R) { *why = "column-copy row outside the tile"; return {}; }
          acc = std::fma(T.bval[e0 + 32 * k + l], sv[j], acc);
        }
        const int c = T.bcid[(size_t)s * 32 + l];
        if (c != 0xFFFF) {
          if (c >= W) { *why = "column id outside the window"; return {}; }
          pw[c] = acc;
          ++seen[c];
        }
      }
    }
    for (int i = 0; i < W; ++i)
      if (seen[i] != 1) { *why = "a window column is not written exactly once"; return {}; }
    for (int i = 0; i < W; ++i) part[T.poff[t] + i] = pw[i];
  }
  std::vector<double> w(n, 0.0);
  std::vector<char> covered(n, 0);
  for (int t = 0; t < T.ntiles; ++t)
    for (int i = 0; i < T.wid[t]; ++i) covered[T.lo[t] + i] = 1;
  for (int64_t c = 0; c < n; ++c) {
    const int64_t b = c / lsq::kNormalColBlock;
    int hits = 0;
    for (int t = T.cb_t0[b]; t <= T.cb_t1[b]; ++t) {
      const int64_t off = c - T.lo[t];
      if (off >= 0 && off < T.wid[t]) { w[c] += part[T.poff[t] + off]; ++hits; }
    }
    if (covered[c] && hits == 0) { *why = "the column-block table misses a window"; return {}; }
  }
  return w;
}

bool check(const char* name, const Csr& A, int cap, int sms, bool expect_ok) {
  lsq::NormalTilesHost T;
  const bool ok = lsq::build_normal_tiles(A.m, A.n, A.rp.data(), A.col.data(), A.val.data(), cap, sms, T);
  if (ok != expect_ok) {
    std::printf("FAIL %s: build returned %d, expected %d\n", name, ok, expect_ok);
    return false;
  }
  if (!ok) {
    std::printf("ok   %s: refused as expected\n", name);
    return true;
  }
  // every stored entry exactly once in each copy, with its value
  std::vector<int> ca(A.col.size(), 0), cb(A.col.size(), 0);
  for (size_t e = 0; e < T.asrc.size(); ++e)
    if (T.asrc[e] >= 0) {
      ca[T.asrc[e]]++;
      if (T.aval[e] != A.val[T.asrc[e]]) { std::printf("FAIL %s: row-copy value\n", name); return false; }
    } else if (T.aval[e] != 0.0) { std::printf("FAIL %s: nonzero padding\n", name); return false; }
  for (size_t e = 0; e < T.bsrc.size(); ++e)
    if (T.bsrc[e] >= 0) {
      cb[T.bsrc[e]]++;
      if (T.bval[e] != A.val[T.bsrc[e]]) { std::printf("FAIL %s: column-copy value\n", name); return false; }
    } else if (T.bval[e] != 0.0) { std::printf("FAIL %s: nonzero padding\n", name); return false; }
  for (size_t e = 0; e < A.col.size(); ++e)
    if (ca[e] != 1 || cb[e] != 1) { std::printf("FAIL %s: entry %zu stored %d / %d times\n", name, e, ca[e], cb[e]); return false; }
  if (T.smem_doubles > cap) { std::printf("FAIL %s: tile above the cap\n", name); return false; }
  std::mt19937_64 g(7);
  std::normal_distribution<double> nd;
  std::vector<double> p(A.n);
  for (auto& x : p) x = nd(g);
  const char* why = nullptr;
  const std::vector<double> wt = tiles_product(T, A.n, p, &why);
  if (why) { std::printf("FAIL %s: %s\n", name, why); return false; }
  const std::vector<double> wr = normal_product(A, p);
  double err = 0.0, nrm = 0.0;
  for (int64_t c = 0; c < A.n; ++c) {
    err = std::max(err, std::fabs(wt[c] - wr[c]));
    nrm = std::max(nrm, std::fabs(wr[c]));
  }
  const double rel = nrm > 0 ? err / nrm : err;
  std::printf("%s %s: %d tiles, max |w - A^T A p| / max|A^T A p| = %.2e\n", rel <= 1e-13 ? "ok  " : "FAIL", name,
              T.ntiles, rel);
  return rel <= 1e-13;
}

}  // namespace

int main() {
  bool all = true;
  all &= check("banded", banded(5000, 24000, 8, 40, 0, 0, 0, 1), 4096, 152, true);
  all &= check("empty rows and columns", banded(3000, 15000, 6, 25, 7, 1000, 1064, 2), 2048, 152, true);
  {
    std::mt19937_64 g(3);
    Csr A = banded(2000, 8000, 6, 20, 0, 0, 0, 3);
    std::vector<int32_t> all_cols(2000);
    for (int c = 0; c < 2000; ++c) all_cols[c] = c;
    A.add_row(all_cols, g);  // a row over the whole width: its tile's window is all of A
    all &= check("one full-width row", A, 4096, 152, true);
  }
  {
    std::mt19937_64 g(4);
    Csr A = banded(40000, 60000, 4, 10, 0, 0, 0, 4);
    A.add_row({0, 39999}, g);  // its window alone exceeds the cap
    all &= check("a row wider than the cap", A, 8192, 152, false);
  }
  {
    std::mt19937_64 g(5);
    Csr A;
    A.n = 1;
    A.add_row({0}, g);
    all &= check("1 x 1", A, 4096, 152, true);
  }
  {
    // rows in no particular order: windows are wide, tiles many
    std::mt19937_64 g(6);
    Csr A;
    A.n = 3000;
    for (int r = 0; r < 6000; ++r) {
      const int c0 = (int)(g() % 3000);
      A.add_row({c0, std::min(c0 + 3, 2999)}, g);
    }
    all &= check("unsorted rows", A, 8192, 152, true);
  }
  std::printf(all ? "ALL OK\n" : "SOME FAILED\n");
  return all ? 0 : 1;
}
