// y-solve with the pre-factorised A A^T (Sec. 4, hybrid sparse linear system
// solver; eq. cholesky), done entirely on the GPU.
//
// Structure used (exact algebra, no approximation):
//  * Each A_mom row ties a duplicate entry p of a monomial to its
//    representative r: a_p = s_p e_p - s_r e_r. The rows of one monomial form
//    a "star" whose Gram block is D + s_r^2 1 1^T (D = diag(s_p^2)); it is
//    inverted by the Sherman-Morrison formula. These rows are always
//    independent (each owns the entry p).
//  * Eliminating the stars leaves, on the other rows (A_ineq, A_eq, phi_0,
//    A_sen), the Schur complement S = A_o diag(omega) A_o^T with
//    omega_r = 1 / (s_r^2 * #occurrences of the monomial) at representatives
//    and omega = 1 on localizing entries. Ordered by clique, S is block
//    tridiagonal and the coupling between cliques k and k+1 runs only through
//    the consensus rows of clique k (the last rows of its group).
//  * S is factorised in the order cliques N..1 (natural order inside a
//    clique) by a Cholesky that skips a row whose pivot is at most
//    rank_tol * S_ii: that row is linearly dependent on the rows before it
//    and is removed from the SDP (y = 0 there). Factor blocks: a dense lower
//    triangular L_k per clique and a coupling E_k = L_k^{-1} S[G_k, cons_{k-1}].
// All arithmetic is FP64.
#include <cuda_runtime.h>

#include "common.cuh"
#include "factor.cuh"

namespace strom {
namespace {

constexpr int FT = 256;       // threads per factorisation CTA
constexpr int SOLVE_T = 256;  // threads per chain-solve CTA

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// S_ij = sum_p omega_p A_ip A_jp over two sorted CSR rows
__device__ double sdot(const YsolveDev& d, int64_t ri, int64_t rj) {
  int64_t a = d.rowptr[ri], ae = d.rowptr[ri + 1];
  int64_t b = d.rowptr[rj], be = d.rowptr[rj + 1];
  double s = 0.0;
  while (a < ae && b < be) {
    const int ca = d.col[a], cb = d.col[b];
    if (ca == cb) { s += d.omega[ca] * d.val[a] * d.val[b]; ++a; ++b; }
    else if (ca < cb) ++a;
    else ++b;
  }
  return s;
}

// One CTA per (instance, clique): dense lower D_k = S[G_k, G_k], its diagonal,
// and the coupling right-hand side B_k = S[G_k, cons_{k-1}].
__global__ void __launch_bounds__(FT) assemble_kernel(YsolveDev d, const int32_t* __restrict__ glist) {
  const int g = glist ? glist[blockIdx.x] : blockIdx.x;  // global group id
  const int64_t g0 = d.grp_beg[g];
  const int m = d.grp_len[g];
  double* L = d.fac + d.fac_off[g];
  double* diag0 = d.diag0 + g0;
  for (int64_t idx = threadIdx.x; idx < (int64_t)m * m; idx += FT) {
    const int i = (int)(idx % m), j = (int)(idx / m);  // column-major: i row, j col
    double v = 0.0;
    if (i >= j) v = sdot(d, d.oth_rows[g0 + i], d.oth_rows[g0 + j]);
    L[idx] = v;
    if (i == j) diag0[i] = v;
  }
  const int cprev = d.coup_n[g];
  if (cprev > 0) {
    const int64_t pg0 = d.grp_beg[g - 1];
    const int pm = d.grp_len[g - 1];
    double* B = d.coup + d.coup_off[g];
    for (int64_t idx = threadIdx.x; idx < (int64_t)m * cprev; idx += FT) {
      const int i = (int)(idx % m), c = (int)(idx / m);
      B[idx] = sdot(d, d.oth_rows[g0 + i], d.oth_rows[pg0 + pm - cprev + c]);
    }
  }
}

// One CTA per instance: the chain factorisation, cliques N..1.
// zsave (nullable): store the Schur update E^T E that the first group receives
// (shared with the instances that reuse this chain's later groups);
// zuse (nullable, with first_only): apply that stored update instead of E^T E
__global__ void __launch_bounds__(FT) chain_factor_kernel(YsolveDev d, double rank_tol, const int32_t* __restrict__ ilist,
                                                          int first_only, double* zsave, const double* zuse) {
  const int inst = ilist ? ilist[blockIdx.x] : blockIdx.x;
  const int gbeg = d.inst_grp[inst], gend = d.inst_grp[inst + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ double s_piv;
  __shared__ int s_keep;
  // first_only: the groups after the first are shared with another instance
  // and already factorised; only the first clique's group is done here
  for (int g = first_only ? gbeg : gend - 1; g >= gbeg; --g) {
    const int64_t g0 = d.grp_beg[g];
    const int m = d.grp_len[g];
    double* L = d.fac + d.fac_off[g];
    // Schur update from the clique factored just before: D[cons, cons] -= E^T E
    if (g + 1 < gend) {
      const int cn = d.coup_n[g + 1];
      const int nm = d.grp_len[g + 1];
      const double* E = d.coup + d.coup_off[g + 1];
      const bool use_z = (zuse != nullptr) && first_only && g == gbeg;
      for (int pair = warp; pair < cn * cn; pair += FT / 32) {
        const int a = pair % cn, b = pair / cn;
        if (a < b) continue;
        double sum = 0.0;
        if (use_z) {
          sum = (lane == 0) ? zuse[(int64_t)b * cn + a] : 0.0;
        } else {
          for (int r = lane; r < nm; r += 32) sum += E[(int64_t)a * nm + r] * E[(int64_t)b * nm + r];
          sum = warp_sum(sum);
        }
        if (lane == 0) {
          const int i = m - cn + a, j = m - cn + b;
          L[(int64_t)j * m + i] -= sum;
          if (zsave != nullptr && g == gbeg) {
            zsave[(int64_t)b * cn + a] = sum;
            zsave[(int64_t)a * cn + b] = sum;
          }
        }
      }
      __syncthreads();
    }
    // pivot-skipping right-looking Cholesky
    for (int j = 0; j < m; ++j) {
      if (threadIdx.x == 0) {
        const double piv = L[(int64_t)j * m + j];
        const double ref = d.diag0[g0 + j];
        const int keep = (ref > 0.0) && (piv > rank_tol * ref);
        s_keep = keep;
        s_piv = keep ? sqrt(piv) : 1.0;
        d.keep[d.oth_rows[g0 + j]] = (uint8_t)keep;
        d.keep_oth[g0 + j] = (uint8_t)keep;
        d.inv_piv[g0 + j] = keep ? 1.0 / sqrt(piv) : 0.0;
        L[(int64_t)j * m + j] = s_piv;
      }
      __syncthreads();
      const int keep = s_keep;
      const double inv = 1.0 / s_piv;
      double* colj = L + (int64_t)j * m;
      for (int i = j + 1 + threadIdx.x; i < m; i += FT) colj[i] = keep ? colj[i] * inv : 0.0;
      __syncthreads();
      if (keep) {
        for (int l = j + 1 + warp; l < m; l += FT / 32) {
          const double ljl = colj[l];
          if (ljl == 0.0) continue;
          double* coll = L + (int64_t)l * m;
          for (int i = l + lane; i < m; i += 32) coll[i] -= colj[i] * ljl;
        }
      }
      __syncthreads();
    }
    // row-major copy of L_g for the backward substitution: lt[j * m + i] = L[j][i]
    {
      double* LT = d.lt + d.fac_off[g];
      for (int64_t idx = threadIdx.x; idx < (int64_t)m * m; idx += FT) {
        const int i = (int)(idx % m), j = (int)(idx / m);  // writes are coalesced in i
        LT[(int64_t)j * m + i] = (i <= j) ? L[(int64_t)i * m + j] : 0.0;
      }
      __syncthreads();
    }
    // inverses of the 32 x 32 diagonal blocks of L_g, with every dropped row j
    // replaced by e_j in L and by 0 in the inverse (so w_j = y_j = 0 there);
    // stored column-major per block: Dinv[t][j] at t * 32 + j.
    {
      const int nb = (m + 31) / 32;
      double* Dg = d.dinv + d.dinv_off[g];
      for (int b = warp; b < nb; b += FT / 32) {
        const int jb = b * 32, je = min(jb + 32, m), bs = je - jb;
        double* Db = Dg + (int64_t)b * 1024;
        // lane k solves Ltilde x = e_k (forward substitution) for column k
        const int k = lane;
        double x[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) x[i] = 0.0;
        if (k < bs && d.keep[d.oth_rows[g0 + jb + k]]) {
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            if (i < bs && i >= k) {
              const int row = jb + i;
              double acc = (i == k) ? 1.0 : 0.0;
              if (d.keep[d.oth_rows[g0 + row]]) {
#pragma unroll
                for (int c = 0; c < 32; ++c)
                  if (c >= k && c < i) acc -= L[(int64_t)(jb + c) * m + row] * x[c];
                x[i] = acc / L[(int64_t)row * m + row];
              } else {
                x[i] = 0.0;
              }
            }
          }
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) Db[(int64_t)k * 32 + i] = x[i];  // Dinv[i][k]
      }
      __syncthreads();
    }
    // coupling E_g = L_g^{-1} B_g (one warp per right-hand side)
    const int cprev = d.coup_n[g];
    if (cprev > 0) {
      double* B = d.coup + d.coup_off[g];
      for (int c = warp; c < cprev; c += FT / 32) {
        double* e = B + (int64_t)c * m;
        for (int j = 0; j < m; ++j) {
          const double* colj = L + (int64_t)j * m;
          double ej = 0.0;
          if (lane == 0) ej = d.keep[d.oth_rows[g0 + j]] ? e[j] / colj[j] : 0.0;
          ej = __shfl_sync(0xffffffffu, ej, 0);
          if (lane == 0) e[j] = ej;
          if (ej != 0.0)
            for (int i = j + 1 + lane; i < m; i += 32) e[i] -= colj[i] * ej;
          __syncwarp();
        }
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// solve kernels
// ---------------------------------------------------------------------------

// rho at every representative with duplicates:
// rho_r = c * sum_p r_p / s_p^2 / (1 + c d) / s_r   (c = s_r^2, d = sum 1/s_p^2)
__global__ void star_pre_kernel(YsolveDev d, const double* __restrict__ r, double* __restrict__ rho) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.nclass) return;
  if (d.inst_active && !d.inst_active[d.star_inst[c]]) return;
  double acc = 0.0;
  for (int32_t q = d.star_ptr[c]; q < d.star_ptr[c + 1]; ++q) acc += r[d.star_row[q]] * d.star_inv_s2[q];
  const double cc = d.star_c[c];
  const int64_t rep = d.star_rep[c];
  rho[rep] = cc * acc / (1.0 + cc * d.star_d[c]) * d.inv_rep_s[rep];
}

// t_i = r_i + sum_p A_ip rho_p for every other row (written into yo, group order)
__global__ void other_rhs_kernel(YsolveDev d, const double* __restrict__ r, const double* __restrict__ rho,
                                 double* __restrict__ yo) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= d.noth) return;
  const int64_t row = d.oth_rows[q];
  if (row < 0) return;  // unused capacity after the row reduction
  if (d.inst_active && !d.inst_active[d.row_inst[row]]) return;
  double t = r[row];
  for (int64_t e = d.rowptr[row]; e < d.rowptr[row + 1]; ++e) t += d.val[e] * rho[d.col[e]];
  yo[q] = d.keep_oth[q] ? t : 0.0;
}

// y = 0 on the rows removed by the row reduction
__global__ void zero_rows_kernel(const int64_t* __restrict__ rows, int64_t n, double* __restrict__ y) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) y[rows[q]] = 0.0;
}

// block forward / backward substitution along the chain; one CTA per instance.
// The right-hand side arrives in yo (other rows, group order) and the
// solution is written back to yo and scattered to y. Each 32 x 32 diagonal
// block is applied through its precomputed inverse (a parallel product),
// so no step of the substitution is a sequential chain of 32 divisions.
__global__ void __launch_bounds__(SOLVE_T) chain_solve_kernel(YsolveDev d, double* __restrict__ yo, double* __restrict__ y) {
  const int inst = blockIdx.x;
  if (d.inst_active && !d.inst_active[inst]) return;
  const int gbeg = d.inst_grp[inst], gend = d.inst_grp[inst + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  extern __shared__ double sh[];  // [max group size]
  // forward: groups gend-1 .. gbeg,  w_g = L_g^{-1} (t_g - F_g w_{g+1})
  for (int g = gend - 1; g >= gbeg; --g) {
    const int64_t g0 = d.grp_beg[g];
    const int m = d.grp_len[g];
    const double* L = d.fac + d.fac_off[g];
    for (int i = threadIdx.x; i < m; i += SOLVE_T) sh[i] = yo[g0 + i];
    __syncthreads();
    if (g + 1 < gend) {
      const int cn = d.coup_n[g + 1];
      const int64_t ng0 = d.grp_beg[g + 1];
      const int nm = d.grp_len[g + 1];
      const double* E = d.coup + d.coup_off[g + 1];
      // one warp per output, lanes over rows; the butterfly sum has a fixed
      // order, the same in the multi-right-hand-side kernel
      for (int a = warp; a < cn; a += SOLVE_T / 32) {
        double acc = 0.0;
        for (int rr = lane; rr < nm; rr += 32) acc += E[(int64_t)a * nm + rr] * yo[ng0 + rr];
        acc = warp_sum(acc);
        if (lane == 0) sh[m - cn + a] -= acc;
      }
      __syncthreads();
    }
    const double* Dg = d.dinv + d.dinv_off[g];
    for (int jb = 0; jb < m; jb += 32) {
      const int je = min(jb + 32, m), bs = je - jb;
      const double* Db = Dg + (int64_t)(jb / 32) * 1024;
      // w_b = Dinv_b t_b, one thread per output (Dinv column-major: coalesced in j)
      {
        double w = 0.0;
        if (threadIdx.x < bs) {
          const int j = threadIdx.x;
          for (int t = 0; t < bs; ++t) w += Db[t * 32 + j] * sh[jb + t];
        }
        __syncthreads();
        if (threadIdx.x < bs) sh[jb + threadIdx.x] = w;
      }
      __syncthreads();
      if (je - jb == 32) {
        for (int i = je + threadIdx.x; i < m; i += SOLVE_T) {
          const double* Li = L + (int64_t)jb * m + i;
          double lv[32];
#pragma unroll
          for (int t = 0; t < 32; ++t) lv[t] = Li[(int64_t)t * m];  // 32 independent loads in flight
          double acc = 0.0;  // one chain in t order: the same arithmetic as the multi-RHS kernel
#pragma unroll
          for (int t = 0; t < 32; ++t) acc += lv[t] * sh[jb + t];
          sh[i] -= acc;
        }
      } else {
        for (int i = je + threadIdx.x; i < m; i += SOLVE_T) {
          double acc = 0.0;
          for (int jj = jb; jj < je; ++jj) acc += L[(int64_t)jj * m + i] * sh[jj];
          sh[i] -= acc;
        }
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < m; i += SOLVE_T) yo[g0 + i] = sh[i];
    __syncthreads();
  }
  // backward: groups gbeg .. gend-1,  y_g = L_g^{-T} (w_g - E_g y_{g-1}[cons])
  for (int g = gbeg; g < gend; ++g) {
    const int64_t g0 = d.grp_beg[g];
    const int m = d.grp_len[g];
    const double* L = d.fac + d.fac_off[g];
    const double* Dg = d.dinv + d.dinv_off[g];
    const int cprev = d.coup_n[g];
    const double* E = d.coup + d.coup_off[g];
    const int64_t pcons0 = (g > gbeg) ? d.grp_beg[g - 1] + d.grp_len[g - 1] - cprev : 0;  // consensus rows ending group g-1
    for (int i = threadIdx.x; i < m; i += SOLVE_T) {
      double w = yo[g0 + i];
      for (int c = 0; c < cprev; ++c) w -= E[(int64_t)c * m + i] * yo[pcons0 + c];
      sh[i] = w;
    }
    __syncthreads();
    const int nb = (m + 31) / 32;
    const double* LT = d.lt + d.fac_off[g];  // row-major copy: LT[j * m + i] = L[j][i]
    for (int b = nb - 1; b >= 0; --b) {
      const int jb = b * 32, je = min(jb + 32, m), bs = je - jb;
      // y_b = Dinv_b^T w_b, one thread per output (no cross-lane reductions)
      const double* Db = Dg + (int64_t)b * 1024;
      double v = 0.0;
      if (threadIdx.x < bs) {
        const int j = threadIdx.x;
        for (int t = 0; t < bs; ++t) v += Db[(int64_t)j * 32 + t] * sh[jb + t];
      }
      __syncthreads();
      if (threadIdx.x < bs) sh[jb + threadIdx.x] = v;
      __syncthreads();
      // upward update: w_i -= sum_{j in block} L[j][i] y_j for i < jb (coalesced in i)
      if (bs == 32) {
        for (int i = threadIdx.x; i < jb; i += SOLVE_T) {
          const double* Li = LT + (int64_t)jb * m + i;
          double lv[32];
#pragma unroll
          for (int t = 0; t < 32; ++t) lv[t] = Li[(int64_t)t * m];
          double acc = 0.0;
#pragma unroll
          for (int t = 0; t < 32; ++t) acc += lv[t] * sh[jb + t];
          sh[i] -= acc;
        }
      } else {
        for (int i = threadIdx.x; i < jb; i += SOLVE_T) {
          double acc = 0.0;
          for (int jj = jb; jj < je; ++jj) acc += LT[(int64_t)jj * m + i] * sh[jj];
          sh[i] -= acc;
        }
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < m; i += SOLVE_T) {
      yo[g0 + i] = sh[i];
      y[d.oth_rows[g0 + i]] = sh[i];
    }
    __syncthreads();
  }
}


// ---------------------------------------------------------------------------
// Multi-right-hand-side chain solve for instances that share the factor of
// cliques 2..N: one CTA serves a tile of R instances. For a shared group each
// element of L (L^T, E, the 32x32 inverses) is loaded once and applied to the
// R right-hand sides (columns) held in shared memory as sh[i * R + r], and
// every barrier is paid once per R instances. The first clique's group has a
// factor per instance and is done column by column.
// ---------------------------------------------------------------------------

// one column (stride R in sh) through a per-instance group, forward
template <int R>
__device__ void column_forward(const YsolveDev& d, int g, double* sh, int r, const double* __restrict__ yo,
                               int ngrp_next) {
  const int m = d.grp_len[g];
  const double* L = d.fac + d.fac_off[g];
  const double* Dg = d.dinv + d.dinv_off[g];
  (void)ngrp_next;
  for (int jb = 0; jb < m; jb += 32) {
    const int je = min(jb + 32, m), bs = je - jb;
    const double* Db = Dg + (int64_t)(jb / 32) * 1024;
    double w = 0.0;
    if (threadIdx.x < bs) {
      const int j = threadIdx.x;
      for (int t = 0; t < bs; ++t) w += Db[t * 32 + j] * sh[(jb + t) * R + r];
    }
    __syncthreads();
    if (threadIdx.x < bs) sh[(jb + threadIdx.x) * R + r] = w;
    __syncthreads();
    for (int i = je + threadIdx.x; i < m; i += SOLVE_T) {
      double acc = 0.0;
      for (int jj = jb; jj < je; ++jj) acc += L[(int64_t)jj * m + i] * sh[jj * R + r];
      sh[i * R + r] -= acc;
    }
    __syncthreads();
  }
}

// one column (stride R in sh) through a per-instance group, backward
template <int R>
__device__ void column_backward(const YsolveDev& d, int g, double* sh, int r) {
  const int m = d.grp_len[g];
  const double* LT = d.lt + d.fac_off[g];
  const double* Dg = d.dinv + d.dinv_off[g];
  const int nb = (m + 31) / 32;
  for (int b = nb - 1; b >= 0; --b) {
    const int jb = b * 32, je = min(jb + 32, m), bs = je - jb;
    const double* Db = Dg + (int64_t)b * 1024;
    double v = 0.0;
    if (threadIdx.x < bs) {
      const int j = threadIdx.x;
      for (int t = 0; t < bs; ++t) v += Db[(int64_t)j * 32 + t] * sh[(jb + t) * R + r];
    }
    __syncthreads();
    if (threadIdx.x < bs) sh[(jb + threadIdx.x) * R + r] = v;
    __syncthreads();
    for (int i = threadIdx.x; i < jb; i += SOLVE_T) {
      double acc = 0.0;
      for (int jj = jb; jj < je; ++jj) acc += LT[(int64_t)jj * m + i] * sh[jj * R + r];
      sh[i * R + r] -= acc;
    }
    __syncthreads();
  }
}

template <int R>
__global__ void __launch_bounds__(SOLVE_T) chain_solve_multi_kernel(YsolveDev d, int ninst, double* __restrict__ yo,
                                                                   double* __restrict__ y) {
  static_assert(32 * R <= SOLVE_T, "one thread per (output, column) of a 32x32 inverse product");
  extern __shared__ double sh[];  // [max group size * R], element (i, r) at i * R + r
  __shared__ int s_inst[R];
  __shared__ int s_act[R];
  const int i0 = blockIdx.x * R;
  if (threadIdx.x < R) {
    const int i = i0 + threadIdx.x;
    const bool valid = i < ninst;
    s_inst[threadIdx.x] = valid ? i : i0;  // columns past the end read instance i0 and are never written
    s_act[threadIdx.x] = valid && (d.inst_active == nullptr || d.inst_active[i]);
  }
  __syncthreads();
  int any = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) any |= s_act[r];
  if (!any) return;
  const int NG = d.inst_grp[i0 + 1] - d.inst_grp[i0];
  const int gl0 = d.inst_grp[i0];  // the tile's first instance: its shared-group offsets are everyone's

  // ---- forward through the shared groups NG-1 .. 1
  for (int k = NG - 1; k >= 1; --k) {
    const int gl = gl0 + k;
    const int m = d.grp_len[gl];
    const double* L = d.fac + d.fac_off[gl];
    const double* Dg = d.dinv + d.dinv_off[gl];
    for (int idx = threadIdx.x; idx < m * R; idx += SOLVE_T) {
      const int i = idx / R, r = idx - (idx / R) * R;
      sh[idx] = yo[d.grp_beg[d.inst_grp[s_inst[r]] + k] + i];
    }
    __syncthreads();
    if (k + 1 < NG) {
      const int gn = gl + 1;
      const int cn = d.coup_n[gn], nm = d.grp_len[gn];
      const double* E = d.coup + d.coup_off[gn];
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      for (int idx = warp; idx < cn * R; idx += SOLVE_T / 32) {
        const int a = idx / R, r = idx - (idx / R) * R;
        const double* yn = yo + d.grp_beg[d.inst_grp[s_inst[r]] + k + 1];
        double acc = 0.0;
        for (int rr = lane; rr < nm; rr += 32) acc += E[(int64_t)a * nm + rr] * yn[rr];
        acc = warp_sum(acc);
        if (lane == 0) sh[(m - cn + a) * R + r] -= acc;
      }
      __syncthreads();
    }
    for (int jb = 0; jb < m; jb += 32) {
      const int je = min(jb + 32, m), bs = je - jb;
      const double* Db = Dg + (int64_t)(jb / 32) * 1024;
      const int j = threadIdx.x / R, r = threadIdx.x - (threadIdx.x / R) * R;
      double w = 0.0;
      if (threadIdx.x < 32 * R && j < bs)
        for (int t = 0; t < bs; ++t) w += Db[t * 32 + j] * sh[(jb + t) * R + r];
      __syncthreads();
      if (threadIdx.x < 32 * R && j < bs) sh[(jb + j) * R + r] = w;
      __syncthreads();
      for (int i = je + threadIdx.x; i < m; i += SOLVE_T) {
        double acc[R];
#pragma unroll
        for (int q = 0; q < R; ++q) acc[q] = 0.0;
        for (int t = 0; t < bs; ++t) {
          const double l = L[(int64_t)(jb + t) * m + i];
#pragma unroll
          for (int q = 0; q < R; ++q) acc[q] += l * sh[(jb + t) * R + q];
        }
#pragma unroll
        for (int q = 0; q < R; ++q) sh[i * R + q] -= acc[q];
      }
      __syncthreads();
    }
    for (int idx = threadIdx.x; idx < m * R; idx += SOLVE_T) {
      const int i = idx / R, r = idx - (idx / R) * R;
      if (s_act[r]) yo[d.grp_beg[d.inst_grp[s_inst[r]] + k] + i] = sh[idx];
    }
    __syncthreads();
  }

  // ---- the first clique's group, per column (its factor is per instance)
  for (int r = 0; r < R; ++r) {
    if (!s_act[r]) continue;
    const int g = d.inst_grp[s_inst[r]];
    const int m = d.grp_len[g];
    const int64_t g0 = d.grp_beg[g];
    for (int i = threadIdx.x; i < m; i += SOLVE_T) sh[i * R + r] = yo[g0 + i];
    __syncthreads();
    if (NG > 1) {  // coupling with the shared group 2 (its w is in yo)
      const int cn = d.coup_n[g + 1], nm = d.grp_len[g + 1];
      const double* E = d.coup + d.coup_off[g + 1];
      const double* yn = yo + d.grp_beg[g + 1];
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      for (int a = warp; a < cn; a += SOLVE_T / 32) {
        double acc = 0.0;
        for (int rr = lane; rr < nm; rr += 32) acc += E[(int64_t)a * nm + rr] * yn[rr];
        acc = warp_sum(acc);
        if (lane == 0) sh[(m - cn + a) * R + r] -= acc;
      }
      __syncthreads();
    }
    column_forward<R>(d, g, sh, r, yo, 0);
    // backward for this group right away: it has no previous group
    column_backward<R>(d, g, sh, r);
    for (int i = threadIdx.x; i < m; i += SOLVE_T) {
      yo[g0 + i] = sh[i * R + r];
      y[d.oth_rows[g0 + i]] = sh[i * R + r];
    }
    __syncthreads();
  }

  // ---- backward through the shared groups 1 .. NG-1
  for (int k = 1; k < NG; ++k) {
    const int gl = gl0 + k;
    const int m = d.grp_len[gl];
    const double* LT = d.lt + d.fac_off[gl];
    const double* Dg = d.dinv + d.dinv_off[gl];
    const int cprev = d.coup_n[gl];
    const double* E = d.coup + d.coup_off[gl];
    for (int idx = threadIdx.x; idx < m * R; idx += SOLVE_T) {
      const int i = idx / R, r = idx - (idx / R) * R;
      const int gr = d.inst_grp[s_inst[r]] + k;
      const int64_t pc = d.grp_beg[gr - 1] + d.grp_len[gr - 1] - cprev;
      double w = yo[d.grp_beg[gr] + i];
      for (int c = 0; c < cprev; ++c) w -= E[(int64_t)c * m + i] * yo[pc + c];
      sh[idx] = w;
    }
    __syncthreads();
    const int nb = (m + 31) / 32;
    for (int b = nb - 1; b >= 0; --b) {
      const int jb = b * 32, je = min(jb + 32, m), bs = je - jb;
      const double* Db = Dg + (int64_t)b * 1024;
      const int j = threadIdx.x / R, r = threadIdx.x - (threadIdx.x / R) * R;
      double v = 0.0;
      if (threadIdx.x < 32 * R && j < bs)
        for (int t = 0; t < bs; ++t) v += Db[(int64_t)j * 32 + t] * sh[(jb + t) * R + r];
      __syncthreads();
      if (threadIdx.x < 32 * R && j < bs) sh[(jb + j) * R + r] = v;
      __syncthreads();
      for (int i = threadIdx.x; i < jb; i += SOLVE_T) {
        double acc[R];
#pragma unroll
        for (int q = 0; q < R; ++q) acc[q] = 0.0;
        for (int t = 0; t < bs; ++t) {
          const double l = LT[(int64_t)(jb + t) * m + i];
#pragma unroll
          for (int q = 0; q < R; ++q) acc[q] += l * sh[(jb + t) * R + q];
        }
#pragma unroll
        for (int q = 0; q < R; ++q) sh[i * R + q] -= acc[q];
      }
      __syncthreads();
    }
    for (int idx = threadIdx.x; idx < m * R; idx += SOLVE_T) {
      const int i = idx / R, r = idx - (idx / R) * R;
      if (!s_act[r]) continue;
      const int64_t gb = d.grp_beg[d.inst_grp[s_inst[r]] + k];
      yo[gb + i] = sh[idx];
      y[d.oth_rows[gb + i]] = sh[idx];
    }
    __syncthreads();
  }
}

// star rows: y_alpha = (D + c 1 1^T)^{-1} (r_alpha + c gamma 1),
// gamma = sum_{other rows i} A_{i,rep} y_i / s_rep
__global__ void star_post_kernel(YsolveDev d, const double* __restrict__ r, double* __restrict__ y) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.nclass) return;
  if (d.inst_active && !d.inst_active[d.star_inst[c]]) return;
  const int64_t rep = d.star_rep[c];
  double gam = 0.0;
  for (int64_t e = d.atptr[rep]; e < d.atptr[rep + 1]; ++e) {
    const int32_t row = d.atrow[e];
    if (d.row_kind[row] != STROM_ROW_MOM) gam += d.atval[e] * y[row];
  }
  gam *= d.inv_rep_s[rep];
  const double cc = d.star_c[c];
  double su = 0.0;
  for (int32_t q = d.star_ptr[c]; q < d.star_ptr[c + 1]; ++q) su += (r[d.star_row[q]] + cc * gam) * d.star_inv_s2[q];
  const double corr = cc * su / (1.0 + cc * d.star_d[c]);
  for (int32_t q = d.star_ptr[c]; q < d.star_ptr[c + 1]; ++q) {
    const double is2 = d.star_inv_s2[q];
    y[d.star_row[q]] = (r[d.star_row[q]] + cc * gam) * is2 - is2 * corr;
  }
}

}  // namespace

void ysolve_configure(int max_group) {
  const int bytes = (int)(sizeof(double) * (size_t)max_group * 8);
  if (bytes > 48 * 1024) {
    STROM_CUDA(cudaFuncSetAttribute(chain_solve_multi_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    STROM_CUDA(cudaFuncSetAttribute(chain_solve_multi_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes / 2));
    STROM_CUDA(cudaFuncSetAttribute(chain_solve_multi_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes / 4));
    STROM_CUDA(cudaFuncSetAttribute(chain_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes / 8));
  }
}

void ysolve_factor(const YsolveDev& d, int ngroups, int ninst, double rank_tol, cudaStream_t st,
                   const int32_t* glist, const int32_t* ilist, bool first_only, double* zsave, const double* zuse) {
  if (ngroups == 0 || ninst == 0) return;
  assemble_kernel<<<ngroups, FT, 0, st>>>(d, glist);
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
  chain_factor_kernel<<<ninst, FT, 0, st>>>(d, rank_tol, ilist, first_only ? 1 : 0, zsave, zuse);
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
}

void ysolve_star_pre(const YsolveDev& d, const double* r, double* rho, cudaStream_t st) {
  if (d.nclass == 0) return;
  star_pre_kernel<<<ceil_div(d.nclass, 256), 256, 0, st>>>(d, r, rho);
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
}

void ysolve_star_post(const YsolveDev& d, const double* r, double* y, cudaStream_t st) {
  if (d.nclass == 0) return;
  star_post_kernel<<<ceil_div(d.nclass, 256), 256, 0, st>>>(d, r, y);
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
}

void ysolve_apply(const YsolveDev& d, int ninst, int max_group, const double* r, double* y, double* rho,
                  cudaStream_t st) {
  if (d.nclass > 0) {
    star_pre_kernel<<<ceil_div(d.nclass, 256), 256, 0, st>>>(d, r, rho);
    STROM_CUDA(cudaGetLastError());
    count_launches(1);
  }
  if (d.ndropped > 0 && d.inst_active == nullptr) {
    zero_rows_kernel<<<ceil_div(d.ndropped, 256), 256, 0, st>>>(d.dropped, d.ndropped, y);
    STROM_CUDA(cudaGetLastError());
    count_launches(1);
  }
  other_rhs_kernel<<<ceil_div(d.noth, 256), 256, 0, st>>>(d, r, rho, d.yo);
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
  if (d.tile_r > 1) {
    const size_t smem = sizeof(double) * (size_t)max_group * d.tile_r;
    const int grid = (ninst + d.tile_r - 1) / d.tile_r;
    if (d.tile_r == 2) chain_solve_multi_kernel<2><<<grid, SOLVE_T, smem, st>>>(d, ninst, d.yo, y);
    else if (d.tile_r == 4) chain_solve_multi_kernel<4><<<grid, SOLVE_T, smem, st>>>(d, ninst, d.yo, y);
    else chain_solve_multi_kernel<8><<<grid, SOLVE_T, smem, st>>>(d, ninst, d.yo, y);
  } else {
    chain_solve_kernel<<<ninst, SOLVE_T, sizeof(double) * max_group, st>>>(d, d.yo, y);
  }
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
  if (d.nclass > 0) {
    star_post_kernel<<<ceil_div(d.nclass, 256), 256, 0, st>>>(d, r, y);
    STROM_CUDA(cudaGetLastError());
    count_launches(1);
  }
}

}  // namespace strom
