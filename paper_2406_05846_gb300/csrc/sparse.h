// Sparse factor of the y-solve's Schur complement (host side).
//
// After the star elimination of the A_mom rows, the y-solve works on the
// Gram S = A_o diag(omega) A_o^T of the other rows (A_ineq, A_eq, phi_0,
// A_sen). Its rows are taken in the canonical order of the row reduction:
// cliques N..1, natural row order inside a clique. The pivot-skipping
// Cholesky in that order decides which rows are dependent (they are dropped
// from the SDP) and factorises the rest, S_KK = L L^T. In this order S is
// block tridiagonal by clique (the rows of clique k meet only each other and
// the consensus rows of clique k-1), so L is block bidiagonal: a row of
// clique k has entries only in columns of clique k and, for its consensus
// rows, of clique k+1 (the group eliminated just before it).
//
// The symbolic analysis below finds the pattern of L (elimination tree and
// row patterns, no pivoting) once per distinct row structure; a dropped row
// keeps its place in the pattern with zero entries and a zero inverse pivot.
#pragma once
#include <cstdint>
#include <vector>

#include "internal.h"

namespace strom {

constexpr int kSpBlock = 32;        // rows per block of the sparse substitution
constexpr int kSpMaxGroups = 1024;  // clique groups (horizon N) of one instance

struct SpSymbolic {
  int32_t n = 0;        // canonical positions (other rows of one instance)
  int32_t n_tail = 0;   // positions [0, n_tail) belong to cliques N..2; the first clique's group comes last
  int32_t ngroups = 0;  // groups in canonical order (clique N-1 first)
  std::vector<int32_t> grp_ptr;    // [ngroups + 1] canonical position of each group's first row
  std::vector<int32_t> can_local;  // [n] instance-local row id of each canonical position
  // strictly lower part of L by rows (forward solve) and by columns
  // (backward solve), entries sorted inside a row / column
  std::vector<int64_t> fptr;  // [n + 1]
  std::vector<int32_t> fcol;  // [nnz]
  std::vector<int64_t> bptr;  // [n + 1]
  std::vector<int32_t> brow;  // [nnz]
  std::vector<int32_t> fmap;  // [nnz] column position of each forward entry
  // entries of S to assemble (lower triangle): rows (instance-local ids) and
  // the column position of the entry in L's pattern (-1: the diagonal)
  std::vector<int32_t> s_ri, s_rj;  // s_rj = canonical position of the column (for the diagonal: of the row)
  std::vector<int64_t> s_dst;
  int64_t ns_tail = 0;    // entries of s_* whose column lies in the tail (they come first)
  // level schedules inside each group: forward (rows in increasing order of
  // dependency depth, counting dependencies inside the group only) and
  // backward (the same on the columns, dependencies on later rows)
  std::vector<int32_t> flev_ptr, flev_rows;  // levels of all groups, concatenated
  std::vector<int32_t> flev_grp;             // [ngroups + 1] first level of each group
  std::vector<int32_t> blev_ptr, blev_rows;
  std::vector<int32_t> blev_grp;
  // blocks of the substitution: each group cut into runs of kSpBlock positions
  // from its first row (the last run of a group may be shorter). The entries
  // of row i in columns of earlier blocks come first in the row ([fptr[i],
  // fsplit[i])); those of column j in rows of later blocks come last
  // ([bsplit[j], bptr[j + 1])); the rest form the block's dense diagonal part.
  std::vector<int64_t> fsplit, bsplit;  // [n]
  // entries of row i in columns of the previous group (in elimination order)
  // are [fptr[i], fgrp[i]); entries of column j in rows of the next group
  // are [bgrp[j], bptr[j + 1]) (the substitution gathers them at once when
  // a group starts, not block by block)
  std::vector<int64_t> fgrp, bgrp;      // [n]
  std::vector<int32_t> blk_grp;         // [ngroups + 1] first block of each group
  int32_t nblk = 0;
  int64_t nnz_tail_b = 0;  // column entries of tail columns (they come first)
  int32_t max_col = 0;     // longest column of L (strictly lower entries)
  int32_t max_span = 0;    // max over columns j of (last row - j)
  int32_t max_group = 0;
  int64_t nnz_ = 0;        // strictly lower entries of L (fcol / brow may be released once on the device)
  int64_t nnz() const { return nnz_; }
};

// Symbolic analysis of the Schur complement of one instance (its other rows,
// omega, and A's rows). Throws StatusError when the structure is not block
// bidiagonal in the canonical order (an SDP outside the chain form).
SpSymbolic* sparse_symbolic(const Sdp& q);

// true when two SDPs have the same rows and sparsity (same symbolic factor)
bool same_structure(const Sdp& a, const Sdp& b);

}  // namespace strom
