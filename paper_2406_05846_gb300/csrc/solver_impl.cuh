// Host-side solver object shared by solver.cu and serve.cu.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include <memory>

#include "admm.cuh"
#include "common.cuh"
#include "factor.cuh"
#include "sparse.cuh"
#include "sparse.h"

namespace strom {
// one symbolic pattern of the sparse factor with its device copies; the
// arrays only the factorisation reads (fac_*) may be dropped between
// factorisations when several patterns would not fit together
struct SpPatHost {
  std::unique_ptr<SpSymbolic> sym;
  DevBuf<int64_t> fptr, bptr, fsplit, bsplit, fgrp, bgrp;
  DevBuf<int32_t> fcol, brow, grp_ptr, blk_grp, can_local;
  DevBuf<int64_t> s_dst;
  DevBuf<int32_t> fmap, s_ri, s_rj;
  bool fac_on_device = false;
};
struct SparseState {
  std::vector<std::unique_ptr<SpPatHost>> pats;
  std::vector<int32_t> inst_pat;       // pattern of each instance
  std::vector<SpInstDev> inst_h;
  std::vector<SpPatDev> pats_h;
  DevBuf<SpPatDev> pats_dev;
  DevBuf<SpInstDev> inst_dev;
  DevBuf<double> fval, bval, dinv, dinvb, sdiag, w;
  bool keep_fac = true;                // factorisation arrays stay on the device
  int max_n = 0;
  SpDev dev{};
  int64_t fval_entries = 0;            // values stored (all instances)
  double symbolic_s = 0.0;             // host time of the symbolic analysis
};
struct InstMeta {
  int N, nv, dx, du;
  int64_t nsvec, m;
  std::vector<int32_t> block_n, block_clique;
  std::vector<int64_t> block_off;  // local
  std::vector<int8_t> block_kind;
  std::vector<double> b;
};
}  // namespace strom

using namespace strom;  // internal header: the solver object is written in strom's vocabulary

struct strom_solver {
  strom_options opt{};
  int ninst = 0;
  std::vector<strom::InstMeta> meta;
  std::vector<int64_t> svec_off, row_off;  // [ninst+1]
  int64_t nsvec = 0, m = 0;
  int nblk = 0, ngroups = 0, max_group = 0;
  std::vector<int64_t> inst_blk_off;  // [ninst+1] first global block of instance
  std::vector<int64_t> m_kept;
  std::vector<int64_t> inst_nnz_off;  // [ninst+1] first nonzero of each instance in the batch CSR
  std::vector<int32_t> inst_grp_h;    // [ninst+1] first factor group of each instance
  // other-row groups before the row reduction (host copies)
  std::vector<int64_t> full_oth;      // all other rows, group by group
  std::vector<int64_t> grp_beg_h;     // [ngroups] first entry of each group in full_oth
  std::vector<int32_t> grp_full_len;  // [ngroups]
  std::vector<int32_t> grp_full_cons; // [ngroups] consensus rows closing each group
  std::vector<int32_t> grp_len_h, coup_n_h;      // current (compacted) lengths
  std::vector<std::vector<int64_t>> dropped_h;   // per instance
  // shared tail: instance 0 owns the factor of its cliques 2..N and every
  // other instance's groups after its first point to it
  bool shared_tail = false;
  std::vector<uint8_t> tail_keep;     // keep flags of instance 0's rows (local row order)
  std::vector<int32_t> row_clique_h0; // clique of each row of instance 0
  DevBuf<double> zshared;             // Schur update of instance 0's first group, all consensus rows
  // device data
  DevBuf<int64_t> rowptr, atptr, star_rep, star_row, oth_rows, grp_beg, fac_off, coup_off, blk_off, lam_off, dropped,
      vstore_off;
  DevBuf<float> vstore;     // FP32 eigenvectors of every block, kept for the warm start
  DevBuf<double> vstore64;  // FP64 eigenvectors (polish / FP64 mode)
  DevBuf<int32_t> iters64;  // consecutive FP64 iterations of each instance
  DevBuf<double> eta_ref;   // stall checkpoints of the mixed-precision FP32 phase
  DevBuf<int32_t> it_ref;
  DevBuf<int32_t> col, atrow, row_inst, star_ptr, star_inst, inst_grp, coup_n, grp_len, blk_n, blk_list, blk_inst;
  DevBuf<int32_t> inst_svec_chunk, inst_row_chunk, iters, n_active;
  DevBuf<double> val, atval, b, C, omega, inv_rep_s, star_c, star_d, star_inv_s2, fac, lt, coup, diag0;
  DevBuf<double> X, S, Xb, y, yh, r, rho, norm_b, norm_C, sigma, stats, part_svec, part_rows, blk_inv_sigma;
  DevBuf<double> vscratch, tmp_svec, lam, topvec, yo, inv_piv, dinv;
  DevBuf<int64_t> dinv_off;
  DevBuf<int8_t> row_kind;
  DevBuf<uint8_t> keep, keep_oth, inst_active, inst_flag, inst_prec, blk_act32, blk_act64;
  DevBuf<Chunk> svec_chunks, row_chunks;
  PsdClasses cls;
  YsolveDev yd{};
  AdmmDev ad{};
  AdmmParams prm{};
  int factor_kind = STROM_FACTOR_DENSE;  // the factorisation in use (DENSE or SPARSE)
  strom::SparseState sp;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  cudaGraph_t graph_def = nullptr;
  int64_t graph_kernels = 0;  // kernel nodes of one captured iteration
  ~strom_solver() {
    if (graph) cudaGraphExecDestroy(graph);
    if (graph_def) cudaGraphDestroy(graph_def);
    if (stream) cudaStreamDestroy(stream);
  }
};


namespace strom {
// solver internals used by the serving loop (solver.cu)
void reset_instances(strom_solver* s, const std::vector<int>& inst);
void factor_instances(strom_solver* s, const std::vector<int>& inst, bool tail = false);
void eig_instances(strom_solver* s, const std::vector<int>& inst, bool use_Z, std::vector<double>& lam,
                   std::vector<double>& topvec, std::vector<int64_t>& lam_off);
int run_iterations(strom_solver* s, int iters, cudaStream_t user, int32_t* n_active);
// sparse factor (sparse_solver.cu)
void sparse_setup(strom_solver* s, const strom_sdp* const* sdps, int count);
void sparse_factor_instances(strom_solver* s, const std::vector<int>& inst, bool tail);
// y = (A_K A_K^T)^{-1} r with the factor in use; yd.inst_active selects instances
void ysolve_run(strom_solver* s, const YsolveDev& yd, const double* r, double* y, double* rho, cudaStream_t st);
}  // namespace strom
