// Host-side plan of the one-pass normal-equations product w = A^T (A p).
//
// The paper applies C = A^T A only as A^T (A .) and never forms it (Section 4.1.3).  The
// two-product form reads A twice (once as CSR for q = A p, once as CSC for w = A^T q) and
// gathers p and q from global memory.  The row-tile form reads each entry once per
// direction from a tile-local copy and does both gathers in shared memory:
//
//   tile t = consecutive rows [r0, r1) of A (rows ordered by first column, so a tile's
//   entries fall in a narrow column window [lo_t, lo_t + W_t));
//   s_j   = sum_k a_{jk} p_k             for the tile's rows (p window in shared memory),
//   u_t,c = sum_j a_{jc} s_j             for the window's columns (s in shared memory),
//   w_c   = sum_t u_t,c                  over the tiles whose window holds c, in tile order.
//
// Every sum has a fixed order, so the product is bitwise repeatable.  Both tile-local
// copies are sliced ELL (slices of 32 rows or 32 window columns, entry k of slice lane l
// at offset 32 k + l, padding with value 0), with 16-bit window-local column and
// tile-local row indices.
#pragma once
#include <cstdint>
#include <vector>

namespace lsq {

constexpr int kNormalColBlock = 256;  // columns per entry of the reduction's tile-range table

struct NormalTilesHost {
  int ntiles = 0;
  int smem_doubles = 0;               // max over tiles of even(W_t) + rows_t padded to 32
  std::vector<int64_t> lo;            // [T] first column of the window
  std::vector<int32_t> wid;           // [T] window width W_t (0: no entries)
  std::vector<int32_t> as0, bs0;      // [T+1] first row slice / first column slice of tile t
  std::vector<int64_t> aoff, boff;    // [SA+1] / [SB+1] entry offset of each slice
  std::vector<uint16_t> acol;         // row slices: window-local column of each entry
  std::vector<uint16_t> brow;         // column slices: tile-local row position of each entry
  std::vector<uint16_t> bcid;         // [SB*32] window column of each column-slice lane (0xFFFF: none)
  std::vector<double> aval, bval;
  std::vector<int64_t> asrc, bsrc;    // CSR slot each stored entry copies (-1: padding)
  std::vector<int64_t> poff;          // [T+1] offset of tile t's partial window
  std::vector<int32_t> cb_t0, cb_t1;  // [ceil(n/256)] first / last tile whose window meets the block
};

// Builds the tiles of the m x n CSR matrix (column indices strictly increasing in each
// row).  cap: most doubles of shared memory one tile may use (even window width + rows
// padded to 32); sms: the SM count: where the cap allows, tiles hold equal row counts and
// their number is a multiple of it.  Returns false (out left empty) when a single row
// alone exceeds the cap, or m or the window would overflow the 16-bit local indices.
bool build_normal_tiles(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                        int cap, int sms, NormalTilesHost& out);

}  // namespace lsq
