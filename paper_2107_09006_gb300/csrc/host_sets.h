// Host-side index sets and storage plans of the Schwarz preconditioner.
//
// Everything here is integer bookkeeping built from the sparsity pattern of A and
// the column partition (Section 3 of arXiv 2107.09006): the sets Xi_i and
// Omega_i = [Omega_I,i, Omega_Gamma,i], the block-envelope plan in which each
// local matrix C_ii is stored and factored, the deterministic transposed scatter
// map for sum_i R_i^T y_i, and the row pairs that couple subdomains in the coarse
// operator C_00 = (A R_0^T)^T (A R_0^T).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace lsq {

constexpr int kTile = 32;  // rows/columns of one tile of the block-envelope storage

struct HostSets {
  int64_t m = 0, n = 0, nnz = 0;
  int N = 0;

  // CSC copy of the pattern: csc_ptr[n+1], csc_row[nnz], csc_perm[nnz] = CSR slot.
  std::vector<int64_t> csc_ptr;
  std::vector<int32_t> csc_row;
  std::vector<int64_t> csc_perm;

  // Omega_i in factor order (ascending global column); om_off[N+1].
  std::vector<int64_t> om_off;
  std::vector<int32_t> om_glob;
  std::vector<uint8_t> om_int;        // 1 if the local position is interior
  std::vector<int32_t> om_paper;      // Omega_i in [Omega_I, Omega_Gamma] order
  std::vector<int32_t> nI;            // n_I,i
  std::vector<int64_t> xi_off;        // Xi_i ascending; xi_off[N+1]
  std::vector<int32_t> xi;

  // Block-envelope plan: block row b of subdomain i is global block blk_off[i] + b.
  // It stores tile columns [blk_tf[.], b] as a row-major 32 x width panel starting
  // at element blk_poff[.] of the storage (width = (b - tf + 1) * 32).
  std::vector<int64_t> blk_off;       // N+1
  std::vector<int32_t> blk_tf;        // first tile column of each block row
  std::vector<int64_t> blk_poff;      // element offset of each panel
  int64_t fac_elems = 0;              // elements of one whole storage
  int max_nb = 0;                     // most block rows of one subdomain
  int64_t max_ni = 0;

  // Interior positions: int_loc[int_off[i] ..] = local positions of Omega_I,i
  // (ascending); jj_of[j] = index of column j inside Omega_I of part[j].
  std::vector<int64_t> int_off;
  std::vector<int32_t> int_loc;
  std::vector<int32_t> jj_of;

  // Transposed scatter map: for column j, map_idx[map_ptr[j] ..] lists the positions
  // om_off[i] + k with Omega_i[k] = j, in increasing subdomain order.
  std::vector<int64_t> map_ptr;
  std::vector<int64_t> map_idx;

  // Coarse coupling: for each pair (i <= j) of subdomains with Xi_i and Xi_j sharing
  // rows, the positions of every shared row inside Xi_i and Xi_j.
  std::vector<int32_t> pair_i, pair_j;
  std::vector<int64_t> pair_off;
  std::vector<int32_t> pair_pi, pair_pj;
};

// Sliced-ELL copy of a CSR matrix: slices of 32 rows, rows ordered by decreasing length
// inside windows of `window` rows (stable), entries column-major inside a slice, zero
// padding with column 0; perm maps slice rows to matrix rows (-1 for padding rows).
struct SellHost {
  int64_t nslices = 0;
  std::vector<int64_t> off;
  std::vector<int32_t> perm, col;
  std::vector<double> val;
  std::vector<int64_t> src;  // source CSR slot of every stored entry (-1: padding)
};
void build_sell(int64_t nrows, const int64_t* ptr, const int32_t* idx, const double* val, int window,
                SellHost& out);

// Checks sizes, the CSR pattern (sorted, in range) and the partition ids; "" if valid.
std::string validate_inputs(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col, int N,
                            const int32_t* part);

// Batched problems: checks that A is block diagonal over the nprob problems (rows
// [m_off[q], m_off[q+1]) touch only columns [n_off[q], n_off[q+1])), that every problem
// has m_q >= n_q >= 1, and that the subdomain ids of problem q form one range
// [N_off[q], N_off[q+1]) in problem order; fills N_off and prob_of_sub.  "" if valid.
std::string validate_batch(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col, int N,
                           const int32_t* part, int nprob, const int64_t* m_off, const int64_t* n_off,
                           std::vector<int32_t>& N_off, std::vector<int32_t>& prob_of_sub);

// Row order by first stored column (stable; empty rows last): perm[new] = old row.
// Rows of a least-squares problem may be permuted freely; this order keeps the
// vector entries that neighbouring rows and columns touch close in memory.
void order_rows_by_first_column(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col,
                                std::vector<int32_t>& perm);

// Validates the CSR pattern and the partition and fills hs.  Returns an empty
// string on success, else the reason the input is invalid.  col must be strictly
// increasing within each row; part[j] must lie in [0, N).
std::string build_host_sets(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col,
                            int N, const int32_t* part, bool with_pairs, HostSets& hs);

}  // namespace lsq
