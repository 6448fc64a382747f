// Device-side view of the sparse factor of the y-solve (sparse.cu); the host
// side and the structure of the factor are described in sparse.h.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace strom {

// one symbolic pattern (shared by the instances of one row structure)
struct SpPatDev {
  int32_t n, n_tail, ngroups, max_group;
  const int64_t* fptr;       // [n + 1] rows of L (strictly lower part)
  const int32_t* fcol;       // [nnz]
  const int64_t* bptr;       // [n + 1] columns of L (strictly lower part)
  const int32_t* brow;       // [nnz]
  const int32_t* grp_ptr;    // [ngroups + 1]
  const int32_t* flev_ptr;   // forward levels (rows), inside each group
  const int32_t* flev_rows;
  const int32_t* flev_grp;   // [ngroups + 1]
  const int32_t* blev_ptr;   // backward levels (columns), inside each group
  const int32_t* blev_rows;
  const int32_t* blev_grp;
  const int32_t* can_local;  // [n] instance-local row id of each position
  const int64_t* fsplit;     // [n] row i: entries in earlier blocks are [fptr[i], fsplit[i])
  const int64_t* bsplit;     // [n] column j: entries in later blocks are [bsplit[j], bptr[j + 1])
  const int64_t* fgrp;       // [n] row i: entries in the previous group are [fptr[i], fgrp[i])
  const int64_t* bgrp;       // [n] column j: entries in the next group are [bgrp[j], bptr[j + 1])
  const int32_t* blk_grp;    // [ngroups + 1] first block of each group
  int32_t nblk, tail_blk;    // blocks; blocks of the tail groups
  // factorisation only (device copies exist while a factorisation runs)
  const int32_t* fmap;       // forward entry -> column position
  const int32_t* s_ri;       // entries of S to assemble
  const int32_t* s_rj;
  const int64_t* s_dst;
  int64_t ns, ns_tail, tail_fwd, tail_bwd;  // tail_fwd = fptr[n_tail], tail_bwd = bptr[n_tail]
};

// where instance i's values live. L is stored twice: by rows (fval, the
// forward solve) and by columns (bval, the factorisation and the backward
// solve). An entry whose column is in the shared tail is at
// fval[f_tail + e] / bval[b_tail + e], any other entry at fval[f_own + e] /
// bval[b_own + e] (e its position in the row or column order); the same for
// dinv / sdiag with positions and d_tail / d_own. Without a shared tail
// each pair is equal.
struct SpInstDev {
  int32_t pat;
  int32_t pad;
  int64_t f_tail, f_own, b_tail, b_own, d_tail, d_own;
  int64_t v_tail, v_own;  // inverses of the diagonal blocks: block t at dinvb[v + t * 1024]
  int64_t w_off;    // working vector of the solves: position p at w[w_off + p]
  int64_t row_off;  // first global row of the instance
};

struct SpDev {
  const SpPatDev* pats;
  const SpInstDev* inst;
  int32_t ninst;
  int32_t tile_r;           // instances per CTA in the solves (same pattern; shared tail)
  double* fval;
  double* bval;
  double* dinv;             // 1 / L_jj, 0 for a dropped row
  double* dinvb;            // per block: the inverse of its diagonal part, dropped rows zeroed
  double* sdiag;            // S_jj (the reference of the pivot test)
  double* w;
  uint8_t* keep;            // [m_total] row keep flags
  const uint8_t* inst_active;  // nullable
  // factor-time smem sizing
  int32_t max_col, max_span, max_group;
};

struct YsolveDev;
// S values into bval / sdiag (after zeroing the instances' own part), the
// left-looking pivot-skipping Cholesky of each listed instance on bval, then
// the row-order copy fval.
// first_only: the tail columns are shared and already factorised by their
// owner; only the columns from n_tail on are computed.
// max_ns / max_nnz: the most entries of S to assemble / of L for one listed
// instance; max_blk: the most blocks of one listed instance
void sparse_factor(const SpDev& d, const YsolveDev& y, const int32_t* ilist_dev, int nlist, bool first_only,
                   double rank_tol, cudaStream_t st, int64_t max_ns, int64_t max_nnz, int max_blk);
// y = S^{-1} t on the kept rows: t = r + A rho on the other rows (rho from
// the star elimination), then the forward and backward substitutions, y
// scattered to the rows; the star rows are done by the caller.
// max_n: the most positions of one instance
void sparse_solve(const SpDev& d, const YsolveDev& y, const double* r, const double* rho, double* yout,
                  cudaStream_t st, int max_n);
void sparse_configure(const SpDev& d);

}  // namespace strom
