// Device-side view of the batched sGS-ADMM state (admm.cu).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace strom {

struct Chunk {
  int64_t begin, end;
  int32_t inst, pad;
};

struct AdmmDev {
  int ninst, nblk;
  int n_svec_chunks, n_row_chunks;
  const Chunk* svec_chunks;
  const Chunk* row_chunks;
  const int32_t* inst_svec_chunk;  // [ninst+1]
  const int32_t* inst_row_chunk;   // [ninst+1]
  // data
  const int64_t* rowptr;
  const int32_t* col;
  const double* val;
  const int64_t* atptr;
  const int32_t* atrow;
  const double* atval;
  const double* b;
  const double* C;
  const uint8_t* keep;
  const double* norm_b;
  const double* norm_C;
  // state
  double* X;
  double* S;
  double* sigma;
  uint8_t* inst_active;
  uint8_t* inst_flag;   // 0 running, 1 converged, 2 numerical, 3 maxiter
  uint8_t* inst_prec;
  int32_t* iters;
  int32_t* iters64;     // consecutive iterations projected with the FP64 eigensolver
  double* eta_ref;      // mixed precision: eta at the last stall checkpoint of the FP32 phase
  int32_t* it_ref;      // and its iteration (-1 at allocation)
  double* stats;        // [ninst * 8]: eta_p, eta_d, eta_g, pobj, dobj
  double* part_svec;
  double* part_rows;
  int32_t* n_active;
  // per block
  const int32_t* blk_inst;
  uint8_t* blk_act32;
  uint8_t* blk_act64;
  double* blk_inv_sigma;
};

struct AdmmParams {
  double tol;
  int maxiter;
  int sigma_every;
  double sigma_ratio, sigma_factor, sigma_min, sigma_max;
  int precision;
  double polish_eta;
};

void admm_residual_rhs(const AdmmDev& d, const double* S, double* r, cudaStream_t st);
void admm_xb(const AdmmDev& d, const double* y, double* Xb, cudaStream_t st);
void admm_xupdate(const AdmmDev& d, const double* y, double tau, cudaStream_t st);
void admm_primal_res(const AdmmDev& d, const double* y, cudaStream_t st);
void admm_finalize(const AdmmDev& d, const AdmmParams& p, cudaStream_t st);
void admm_block_mode(const AdmmDev& d, cudaStream_t st);
void csr_spmv(const int64_t* ptr, const int32_t* idx, const double* val, int64_t nrows, const double* x,
              double* out, cudaStream_t st);

}  // namespace strom
