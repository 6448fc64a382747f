// Device-side view of the y-solve data (factor.cu).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace strom {

struct YsolveDev {
  // A (CSR over the whole batch) and A^T (CSR over svec positions)
  const int64_t* rowptr;
  const int32_t* col;
  const double* val;
  const int64_t* atptr;
  const int32_t* atrow;
  const double* atval;
  const int8_t* row_kind;
  const int32_t* row_inst;
  // star elimination
  int64_t nclass;
  const int64_t* star_rep;
  const double* star_c;
  const double* star_d;
  const int32_t* star_ptr;
  const int64_t* star_row;
  const double* star_inv_s2;
  const int32_t* star_inst;
  const double* omega;
  const double* inv_rep_s;
  // groups of other rows, one per (instance, clique). Group g owns the
  // entries [grp_beg[g], grp_beg[g] + capacity) of oth_rows; its first
  // grp_len[g] entries are its rows (all of them before the row reduction,
  // the kept ones after it) and the rest hold -1.
  int64_t noth;              // capacity of oth_rows
  const int64_t* oth_rows;
  const int64_t* grp_beg;
  const int32_t* grp_len;
  const int64_t* dropped;    // rows removed by the row reduction (y = 0 there)
  int64_t ndropped;
  const int32_t* inst_grp;   // [ninst+1] first group of each instance
  const int32_t* coup_n;     // [ngroups] consensus rows of the previous group coupled to this one
  // factor storage
  double* fac;
  double* lt;                // row-major copies of the L_g (same offsets as fac)
  const int64_t* fac_off;
  double* coup;
  const int64_t* coup_off;
  double* diag0;             // [noth]
  uint8_t* keep;             // [m_total]
  uint8_t* keep_oth;         // [noth] keep flag of each other row, group order
  double* yo;                // [noth] work vector of the chain solve, group order
  double* inv_piv;           // [noth] 1 / pivot of each kept other row, 0 if dropped
  double* dinv;              // inverses of the 32 x 32 diagonal blocks of every L_g
  const int64_t* dinv_off;   // [ngroups]
  const uint8_t* inst_active;  // nullable
  int tile_r;                // > 1: multi-right-hand-side solve over tiles of this many instances (shared tail)
};

// glist / ilist (device, nullable): factorise only these groups / instances;
// first_only: only the first group of each listed instance (its later groups
// are shared with an instance factorised before)
// zsave / zuse: see chain_factor_kernel (the first group's Schur update, saved
// by the instance that owns a shared chain and reused by the others)
void ysolve_factor(const YsolveDev& d, int ngroups, int ninst, double rank_tol, cudaStream_t st,
                   const int32_t* glist = nullptr, const int32_t* ilist = nullptr, bool first_only = false,
                   double* zsave = nullptr, const double* zuse = nullptr);
// dynamic shared memory limits of the chain solves for groups up to max_group rows
void ysolve_configure(int max_group);
// the star elimination of the A_mom rows before (rho) and after (their y)
// the solve on the other rows; shared by the dense and the sparse factor
void ysolve_star_pre(const YsolveDev& d, const double* r, double* rho, cudaStream_t st);
void ysolve_star_post(const YsolveDev& d, const double* r, double* y, cudaStream_t st);
void ysolve_apply(const YsolveDev& d, int ninst, int max_group, const double* r, double* y, double* rho,
                  cudaStream_t st);

}  // namespace strom
