// Row tiles of A for the one-pass normal-equations product (layout in normal_tiles.h).
#include "normal_tiles.h"

#include <algorithm>
#include <atomic>
#include <climits>
#include <numeric>
#include <thread>

namespace lsq {
namespace {

struct Span {
  int64_t r0, r1;  // rows [r0, r1)
  int64_t lo, hi;  // columns [lo, hi] of their entries (hi < lo: none)
};

int64_t pad32(int64_t x) { return (x + 31) / 32 * 32; }
int64_t even(int64_t x) { return (x + 1) & ~int64_t(1); }

// Greedy split into tiles: a tile takes the next row while its rows (padded to 32) plus
// its even window width stay within cap and its row count within rmax.  False when a
// single row does not fit.
bool split(int64_t m, const int64_t* rp, const int32_t* col, int64_t cap, int64_t rmax, std::vector<Span>& t) {
  t.clear();
  int64_t r = 0;
  while (r < m) {
    Span s{r, r, INT64_MAX, -1};
    for (; r < m; ++r) {
      int64_t lo = s.lo, hi = s.hi;
      if (rp[r + 1] > rp[r]) {
        lo = std::min<int64_t>(lo, col[rp[r]]);
        hi = std::max<int64_t>(hi, col[rp[r + 1] - 1]);
      }
      const int64_t rows = r + 1 - s.r0;
      const int64_t win = hi >= lo ? hi - lo + 1 : 0;
      if (rows > rmax || rows > 65536 || win > 65535 || pad32(rows) + even(win) > cap) {
        if (rows == 1) return false;
        break;
      }
      s.lo = lo;
      s.hi = hi;
    }
    s.r1 = r;
    t.push_back(s);
  }
  return true;
}

template <class F>
void for_tiles(int T, F&& f) {
  const unsigned hw = std::thread::hardware_concurrency();
  const int nt = std::max(1, std::min<int>(T, (int)std::min(hw ? hw : 4u, 32u)));
  std::atomic<int> next(0);
  std::vector<std::thread> th;
  for (int k = 0; k < nt; ++k)
    th.emplace_back([&]() {
      for (int t; (t = next.fetch_add(1)) < T;) f(t);
    });
  for (auto& x : th) x.join();
}

// The two orders of one tile: its rows by decreasing length and its window columns by
// decreasing entry count (both stable), so that the 32 lanes of a slice have about the
// same number of entries.
struct TileOrder {
  int R = 0, W = 0;
  std::vector<int32_t> rows;  // position j -> row offset within the tile
  std::vector<int32_t> cols;  // slice position -> window column
  std::vector<int32_t> cnt;   // window column -> entries in this tile
};

void tile_order(const Span& s, const int64_t* rp, const int32_t* col, TileOrder& o) {
  o.R = (int)(s.r1 - s.r0);
  o.W = s.hi >= s.lo ? (int)(s.hi - s.lo + 1) : 0;
  auto len = [&](int a) { return rp[s.r0 + a + 1] - rp[s.r0 + a]; };
  o.rows.resize(o.R);
  std::iota(o.rows.begin(), o.rows.end(), 0);
  std::stable_sort(o.rows.begin(), o.rows.end(), [&](int a, int b) { return len(a) > len(b); });
  o.cnt.assign(o.W, 0);
  for (int64_t e = rp[s.r0]; e < rp[s.r1]; ++e) o.cnt[col[e] - s.lo]++;
  o.cols.resize(o.W);
  std::iota(o.cols.begin(), o.cols.end(), 0);
  std::stable_sort(o.cols.begin(), o.cols.end(), [&](int a, int b) { return o.cnt[a] > o.cnt[b]; });
}

}  // namespace

bool build_normal_tiles(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                        int cap, int sms, NormalTilesHost& out) {
  out = NormalTilesHost();
  if (m < 1 || n < 1 || cap < 64) return false;
  std::vector<Span> sp;
  if (!split(m, row_ptr, col, cap, INT64_MAX, sp)) return false;
  // Equal row counts, the tile count a multiple of the SM count, where the cap allows.
  const int64_t unit = std::max(1, sms);
  const int64_t waves = ((int64_t)sp.size() + unit - 1) / unit;
  const int64_t rmax = pad32((m + waves * unit - 1) / (waves * unit));
  if (!split(m, row_ptr, col, cap, rmax, sp)) return false;
  const int T = (int)sp.size();

  std::vector<TileOrder> ord(T);
  for_tiles(T, [&](int t) { tile_order(sp[t], row_ptr, col, ord[t]); });

  // Slice counts and entry counts (padding included), then the global offsets.
  out.ntiles = T;
  out.as0.assign(T + 1, 0);
  out.bs0.assign(T + 1, 0);
  out.poff.assign(T + 1, 0);
  out.lo.resize(T);
  out.wid.resize(T);
  std::vector<int64_t> ea(T + 1, 0), eb(T + 1, 0);
  for (int t = 0; t < T; ++t) {
    const TileOrder& o = ord[t];
    const int sa = (o.R + 31) / 32, sb = (o.W + 31) / 32;
    int64_t na = 0, nb = 0;
    for (int s = 0; s < sa; ++s) {
      const int64_t r = sp[t].r0 + o.rows[32 * s];
      na += 32 * (row_ptr[r + 1] - row_ptr[r]);
    }
    for (int s = 0; s < sb; ++s) nb += 32 * (int64_t)o.cnt[o.cols[32 * s]];
    out.as0[t + 1] = out.as0[t] + sa;
    out.bs0[t + 1] = out.bs0[t] + sb;
    ea[t + 1] = ea[t] + na;
    eb[t + 1] = eb[t] + nb;
    out.lo[t] = o.W > 0 ? sp[t].lo : 0;
    out.wid[t] = o.W;
    out.poff[t + 1] = out.poff[t] + o.W;
    out.smem_doubles = std::max<int>(out.smem_doubles, (int)(even(o.W) + pad32(o.R)));
  }
  const int64_t SA = out.as0[T], SB = out.bs0[T];
  out.aoff.assign(SA + 1, 0);
  out.boff.assign(SB + 1, 0);
  out.acol.assign(ea[T], 0);
  out.aval.assign(ea[T], 0.0);
  out.asrc.assign(ea[T], -1);
  out.brow.assign(eb[T], 0);
  out.bval.assign(eb[T], 0.0);
  out.bsrc.assign(eb[T], -1);
  out.bcid.assign(SB * 32, 0xFFFF);
  out.aoff[SA] = ea[T];
  out.boff[SB] = eb[T];

  for_tiles(T, [&](int t) {
    const Span& s = sp[t];
    const TileOrder& o = ord[t];
    // row slices: entry k of slice lane l is entry k of the row at position 32 sl + l
    int64_t e = ea[t];
    for (int sl = 0; sl < (o.R + 31) / 32; ++sl) {
      out.aoff[out.as0[t] + sl] = e;
      const int64_t r_first = s.r0 + o.rows[32 * sl];
      const int64_t width = row_ptr[r_first + 1] - row_ptr[r_first];
      for (int64_t k = 0; k < width; ++k)
        for (int l = 0; l < 32; ++l, ++e) {
          const int j = 32 * sl + l;
          if (j >= o.R) continue;
          const int64_t r = s.r0 + o.rows[j];
          if (k >= row_ptr[r + 1] - row_ptr[r]) continue;
          const int64_t src = row_ptr[r] + k;
          out.acol[e] = (uint16_t)(col[src] - s.lo);
          out.aval[e] = val[src];
          out.asrc[e] = src;
        }
    }
    // column lists in increasing row position j, then the column slices
    std::vector<int32_t> start(o.W + 1, 0), cur;
    for (int c = 0; c < o.W; ++c) start[c + 1] = start[c] + o.cnt[c];
    cur.assign(start.begin(), start.end() - 1);
    std::vector<int32_t> lj(start[o.W]);
    std::vector<int64_t> ls(start[o.W]);
    for (int j = 0; j < o.R; ++j) {
      const int64_t r = s.r0 + o.rows[j];
      for (int64_t q = row_ptr[r]; q < row_ptr[r + 1]; ++q) {
        const int c = (int)(col[q] - s.lo);
        lj[cur[c]] = j;
        ls[cur[c]++] = q;
      }
    }
    e = eb[t];
    for (int sl = 0; sl < (o.W + 31) / 32; ++sl) {
      const int64_t gs = out.bs0[t] + sl;
      out.boff[gs] = e;
      for (int l = 0; l < 32; ++l)
        if (32 * sl + l < o.W) out.bcid[gs * 32 + l] = (uint16_t)o.cols[32 * sl + l];
      const int width = o.cnt[o.cols[32 * sl]];
      for (int k = 0; k < width; ++k)
        for (int l = 0; l < 32; ++l, ++e) {
          const int qpos = 32 * sl + l;
          if (qpos >= o.W) continue;
          const int c = o.cols[qpos];
          if (k >= o.cnt[c]) continue;
          const int idx = start[c] + k;
          out.brow[e] = (uint16_t)lj[idx];
          out.bval[e] = val[ls[idx]];
          out.bsrc[e] = ls[idx];
        }
    }
  });

  // tiles whose window meets each block of 256 columns (the reduction's search range)
  const int64_t ncb = (n + kNormalColBlock - 1) / kNormalColBlock;
  out.cb_t0.assign(ncb, INT32_MAX);
  out.cb_t1.assign(ncb, -1);
  for (int t = 0; t < T; ++t) {
    if (out.wid[t] == 0) continue;
    const int64_t b0 = out.lo[t] / kNormalColBlock, b1 = (out.lo[t] + out.wid[t] - 1) / kNormalColBlock;
    for (int64_t b = b0; b <= b1; ++b) {
      out.cb_t0[b] = std::min(out.cb_t0[b], t);
      out.cb_t1[b] = std::max(out.cb_t1[b], t);
    }
  }
  for (int64_t b = 0; b < ncb; ++b)
    if (out.cb_t1[b] < 0) out.cb_t0[b] = 0;
  return true;
}

}  // namespace lsq
