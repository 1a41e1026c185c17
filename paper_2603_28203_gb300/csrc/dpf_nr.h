// Internal definitions of the batched Newton-Raphson solver (Alg. 2) shared
// by its host analysis (dpf_nr_symbolic.cpp) and its CUDA part (dpf_nr.cu).
//
// The Newton system J_f dx = -f of Alg. 2 is written per bus as 2x2 blocks:
// block row i holds the (P_i, Q_i) equations, block column j the (theta_j,
// |V|_j) unknowns.  Equations and unknowns that Alg. 2 leaves out (P and Q at
// the slack, Q at pv buses; theta at the slack, |V| at pv and slack buses)
// become identity rows and columns with a zero right-hand side, so that every
// case of a batch has the same block pattern: that of Y_bus.  The blocks are
// factorised as A = L U with unit block-lower L and block-upper U, pivoting
// only inside the 2x2 diagonal blocks (inverted), in a fill-reducing order
// found on the host.
#pragma once

#include <stdint.h>

#include <vector>

#include "dpf_internal.h"

namespace dpf {

enum { NR_U = 0, NR_DIAG = 1, NR_L = 2 };

struct NrSymbolic {
  int n = 0;                       // block rows (buses)
  std::vector<int32_t> order;      // order[r] = internal bus at elimination step r
  std::vector<int32_t> rank;       // rank[i] = elimination step of internal bus i
  // filled block pattern of L + U in elimination order, CSR by rows with
  // sorted columns: row r = its L columns (< r), r itself, its U columns (> r)
  std::vector<int32_t> row_ptr, col, diag;  // diag[r]: position of (r, r)
  std::vector<int32_t> ymap;       // Y_bus CSR entry (internal order) of a position, -1 for fill
  std::vector<int32_t> level;      // elimination-tree height of every row (leaves 0)
  int n_levels = 0;
  // factorisation schedule: positions grouped by the level of their pivot
  // p = min(row, col), 8 ints per target:
  //   {pos, pair_begin, pair_end, kind, dpos, dpair_begin, dpair_end, r}
  // kind NR_U: a U position; NR_DIAG: the diagonal of row r (its inverse
  // is stored; the forward substitution of row r, over its L positions from
  // dpos = row_ptr[r] up to the diagonal, follows); NR_L: an L
  // position, which also needs the pivot's diagonal block: position dpos
  // with its own update range
  std::vector<int32_t> lvl_ptr;    // [n_levels + 1] into targets
  std::vector<int32_t> targets;    // 8 ints per target
  std::vector<int32_t> pairs;      // 2 ints per pair: L(i,k) position, U(k,j) position
  // triangular solves: rows grouped by level, 4 ints per row:
  // {r, first U position of row r, end of row r, 0}
  std::vector<int32_t> rlvl_ptr;   // [n_levels + 1]
  std::vector<int32_t> rows;       // [4 n]
};

// Minimum-degree order of Y_bus's graph, the filled pattern it produces, the
// elimination tree's levels and the update lists.  Host only; fails with
// DPF_E_UNSUPPORTED when the update lists would exceed `max_pairs`.
int nr_symbolic(const dpf_ybus* y, int64_t max_pairs, NrSymbolic* s);

}  // namespace dpf
