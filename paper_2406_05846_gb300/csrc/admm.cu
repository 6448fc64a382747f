// Per-iteration kernels of Algorithm 1 (sGS-ADMM) on a batch of SDPs.
//
// Work is cut into fixed chunks that never cross an instance boundary; each
// chunk is one CTA and writes its partial sums to its own slot, and a
// single-CTA finalize kernel adds the slots of each instance in a fixed order.
// The result of every instance is therefore bit-identical whether it is
// solved alone or inside a batch.
#include <cuda_runtime.h>

#include "admm.cuh"
#include "common.cuh"

namespace strom {
namespace {

constexpr int CT = 256;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int N>
__device__ void block_sum2(double& a, double& b, double* red) {
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { red[2 * w] = a; red[2 * w + 1] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int i = 0; i < N / 32; ++i) { sa += red[2 * i]; sb += red[2 * i + 1]; }
    a = sa;
    b = sb;
  }
}

// r_j = b_j / sigma - A_j . (X / sigma + S - C)         (Steps 1 and 3)
__global__ void __launch_bounds__(CT) residual_rhs_kernel(AdmmDev d, const double* __restrict__ S, double* __restrict__ r) {
  const Chunk ch = d.row_chunks[blockIdx.x];
  if (!d.inst_active[ch.inst]) return;
  const double is = 1.0 / d.sigma[ch.inst];
  for (int64_t j = ch.begin + threadIdx.x; j < ch.end; j += CT) {
    double acc = 0.0;
    for (int64_t e = d.rowptr[j]; e < d.rowptr[j + 1]; ++e) {
      const int32_t p = d.col[e];
      acc += d.val[e] * (d.X[p] * is + S[p] - d.C[p]);
    }
    r[j] = d.b[j] * is - acc;
  }
}

// X_b = X + sigma (A^T y - C)                            (Step 2)
__global__ void __launch_bounds__(CT) xb_kernel(AdmmDev d, const double* __restrict__ y, double* __restrict__ Xb) {
  const Chunk ch = d.svec_chunks[blockIdx.x];
  if (!d.inst_active[ch.inst]) return;
  const double sg = d.sigma[ch.inst];
  for (int64_t p = ch.begin + threadIdx.x; p < ch.end; p += CT) {
    double aty = 0.0;
    for (int64_t e = d.atptr[p]; e < d.atptr[p + 1]; ++e) aty += d.atval[e] * y[d.atrow[e]];
    Xb[p] = d.X[p] + sg * (aty - d.C[p]);
  }
}

// R_d = S + A^T y - C,  X+ = X + tau sigma R_d; partial ||R_d||^2 and <C, X+>   (Step 4)
__global__ void __launch_bounds__(CT) xupdate_kernel(AdmmDev d, const double* __restrict__ y, double tau) {
  __shared__ double red[2 * CT / 32];
  const Chunk ch = d.svec_chunks[blockIdx.x];
  double s_rd = 0.0, s_cx = 0.0;
  if (d.inst_active[ch.inst]) {
    const double ts = tau * d.sigma[ch.inst];
    for (int64_t p = ch.begin + threadIdx.x; p < ch.end; p += CT) {
      double aty = 0.0;
      for (int64_t e = d.atptr[p]; e < d.atptr[p + 1]; ++e) aty += d.atval[e] * y[d.atrow[e]];
      const double c = d.C[p];
      const double rd = d.S[p] + aty - c;
      const double x = d.X[p] + ts * rd;
      d.X[p] = x;
      s_rd += rd * rd;
      s_cx += c * x;
    }
  }
  block_sum2<CT>(s_rd, s_cx, red);
  if (threadIdx.x == 0) {
    d.part_svec[2 * blockIdx.x] = s_rd;
    d.part_svec[2 * blockIdx.x + 1] = s_cx;
  }
}

// partial ||A_K X - b_K||^2 and <b, y> over the kept rows
__global__ void __launch_bounds__(CT) primal_res_kernel(AdmmDev d, const double* __restrict__ y) {
  __shared__ double red[2 * CT / 32];
  const Chunk ch = d.row_chunks[blockIdx.x];
  double s_rp = 0.0, s_by = 0.0;
  if (d.inst_active[ch.inst]) {
    for (int64_t j = ch.begin + threadIdx.x; j < ch.end; j += CT) {
      if (!d.keep[j]) continue;
      double acc = 0.0;
      for (int64_t e = d.rowptr[j]; e < d.rowptr[j + 1]; ++e) acc += d.val[e] * d.X[d.col[e]];
      const double rp = acc - d.b[j];
      s_rp += rp * rp;
      s_by += d.b[j] * y[j];
    }
  }
  block_sum2<CT>(s_rp, s_by, red);
  if (threadIdx.x == 0) {
    d.part_rows[2 * blockIdx.x] = s_rp;
    d.part_rows[2 * blockIdx.x + 1] = s_by;
  }
}

// mixed precision: stall test of the FP32 phase (see finalize_kernel)
constexpr int kStallWindow = 200;
constexpr double kStallEta = 1e-4;
constexpr double kStallRatio = 0.95;

// per instance: eta_p, eta_d, eta_g (eq. kkt-residual), stop test, sigma rule
__global__ void __launch_bounds__(1024) finalize_kernel(AdmmDev d, AdmmParams prm) {
  __shared__ int cnt[32];
  int active_here = 0;
  for (int i = threadIdx.x; i < d.ninst; i += blockDim.x) {
    if (!d.inst_active[i]) continue;
    double rd = 0.0, cx = 0.0, rp = 0.0, by = 0.0;
    for (int c = d.inst_svec_chunk[i]; c < d.inst_svec_chunk[i + 1]; ++c) {
      rd += d.part_svec[2 * c];
      cx += d.part_svec[2 * c + 1];
    }
    for (int c = d.inst_row_chunk[i]; c < d.inst_row_chunk[i + 1]; ++c) {
      rp += d.part_rows[2 * c];
      by += d.part_rows[2 * c + 1];
    }
    const double ep = sqrt(rp) / (1.0 + d.norm_b[i]);
    const double ed = sqrt(rd) / (1.0 + d.norm_C[i]);
    const double eg = fabs(cx - by) / (1.0 + fabs(cx) + fabs(by));
    const int it = d.iters[i] + 1;
    d.iters[i] = it;
    // this iteration's projection used the FP64 eigensolver iff the instance
    // was in FP64 mode before the switches below
    d.iters64[i] = (d.inst_prec[i] == STROM_PREC_FP64) ? d.iters64[i] + 1 : 0;
    double* st = d.stats + 8 * (int64_t)i;
    st[0] = ep; st[1] = ed; st[2] = eg; st[3] = cx; st[4] = by;
    const double eta = fmax(ep, fmax(ed, eg));
    if (!(eta == eta) || isinf(eta)) {  // NaN / Inf: freeze with an error flag
      d.inst_active[i] = 0;
      d.inst_flag[i] = 2;
      continue;
    }
    if (eta <= prm.tol) {
      if (prm.precision == STROM_PREC_MIXED && d.inst_prec[i] == STROM_PREC_FP32) {
        // mixed precision: an instance retires only on an iterate whose
        // projection used the FP64 eigensolver (the final polish)
        d.inst_prec[i] = STROM_PREC_FP64;
        ++active_here;
        continue;
      }
      d.inst_active[i] = 0;
      d.inst_flag[i] = 1;
      continue;
    }
    if (it >= prm.maxiter) {
      d.inst_active[i] = 0;
      d.inst_flag[i] = 3;
      continue;
    }
    if (prm.precision == STROM_PREC_MIXED && d.inst_prec[i] == STROM_PREC_FP32) {
      if (eta <= prm.polish_eta) {
        d.inst_prec[i] = STROM_PREC_FP64;
      } else if (it % kStallWindow == 0) {
        // the FP32 eigensolver's rounding (about 1e-6 relative) can stall
        // the residuals above polish_eta: below kStallEta, an FP32 phase
        // that gains less than 5 % over a window switches to FP64 too. The
        // checkpoint of the previous window counts only if it is this
        // run's (it_ref == it - window), so a reset needs no clearing.
        if (d.it_ref[i] == it - kStallWindow && eta <= kStallEta && eta > kStallRatio * d.eta_ref[i])
          d.inst_prec[i] = STROM_PREC_FP64;
        d.eta_ref[i] = eta;
        d.it_ref[i] = it;
      }
    }
    if (prm.sigma_every > 0 && it % prm.sigma_every == 0) {
      const double epg = fmax(ep, eg);
      double sg = d.sigma[i];
      if (epg > prm.sigma_ratio * ed) sg /= prm.sigma_factor;
      else if (ed > prm.sigma_ratio * epg) sg *= prm.sigma_factor;
      d.sigma[i] = fmin(fmax(sg, prm.sigma_min), prm.sigma_max);
    }
    ++active_here;
  }
  for (int o = 16; o > 0; o >>= 1) active_here += __shfl_xor_sync(0xffffffffu, active_here, o);
  if ((threadIdx.x & 31) == 0) cnt[threadIdx.x >> 5] = active_here;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += cnt[w];
    *d.n_active = s;
  }
}

// per-block view of the instance mode for the projection kernels
__global__ void block_mode_kernel(AdmmDev d) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= d.nblk) return;
  const int i = d.blk_inst[b];
  const uint8_t a = d.inst_active[i];
  d.blk_act32[b] = a && d.inst_prec[i] == STROM_PREC_FP32;
  d.blk_act64[b] = a && d.inst_prec[i] == STROM_PREC_FP64;
  d.blk_inv_sigma[b] = 1.0 / d.sigma[i];
}

// plain operator kernels (kernel-level entry points)
__global__ void spmv_kernel(const int64_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                            const double* __restrict__ val, int64_t nrows, const double* __restrict__ x,
                            double* __restrict__ out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nrows) return;
  double acc = 0.0;
  for (int64_t e = ptr[j]; e < ptr[j + 1]; ++e) acc += val[e] * x[idx[e]];
  out[j] = acc;
}

}  // namespace

void admm_residual_rhs(const AdmmDev& d, const double* S, double* r, cudaStream_t st) {
  residual_rhs_kernel<<<d.n_row_chunks, CT, 0, st>>>(d, S, r);
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
}
void admm_xb(const AdmmDev& d, const double* y, double* Xb, cudaStream_t st) {
  xb_kernel<<<d.n_svec_chunks, CT, 0, st>>>(d, y, Xb);
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
}
void admm_xupdate(const AdmmDev& d, const double* y, double tau, cudaStream_t st) {
  xupdate_kernel<<<d.n_svec_chunks, CT, 0, st>>>(d, y, tau);
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
}
void admm_primal_res(const AdmmDev& d, const double* y, cudaStream_t st) {
  primal_res_kernel<<<d.n_row_chunks, CT, 0, st>>>(d, y);
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
}
void admm_finalize(const AdmmDev& d, const AdmmParams& p, cudaStream_t st) {
  finalize_kernel<<<1, 1024, 0, st>>>(d, p);
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
}
void admm_block_mode(const AdmmDev& d, cudaStream_t st) {
  block_mode_kernel<<<ceil_div(d.nblk, 256), 256, 0, st>>>(d);
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
}
void csr_spmv(const int64_t* ptr, const int32_t* idx, const double* val, int64_t nrows, const double* x,
              double* out, cudaStream_t st) {
  if (nrows == 0) return;
  spmv_kernel<<<ceil_div(nrows, 256), 256, 0, st>>>(ptr, idx, val, nrows, x, out);
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
}

}  // namespace strom
