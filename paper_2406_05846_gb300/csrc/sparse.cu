// Sparse factor of the y-solve (eq. cholesky; Sec. 4, hybrid sparse linear
// system solver, here entirely on the GPU). The structure is described in
// sparse.h: S is the Gram of the rows other than A_mom after the exact star
// elimination of the A_mom rows, its rows in the canonical order of the row
// reduction, and L its pivot-skipping Cholesky factor (block bidiagonal by
// clique). All arithmetic is FP64; every reduction has a fixed order, so a
// result does not depend on what else is in the batch.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "factor.cuh"
#include "sparse.cuh"
#include "sparse.h"

namespace strom {
namespace {

constexpr int SOLVE_T = 256;

// S_ij = sum_p omega_p A_ip A_jp over two sorted CSR rows (global row ids)
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

// entries of S into the column-order values: blockIdx.y = listed instance
__global__ void sp_assemble_kernel(SpDev d, YsolveDev y, const int32_t* __restrict__ ilist, int first_only) {
  const SpInstDev I = d.inst[ilist[blockIdx.y]];
  const SpPatDev P = d.pats[I.pat];
  const int64_t e0 = first_only ? P.ns_tail : 0;
  const int64_t q = e0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P.ns) return;
  const int32_t ri = P.s_ri[q], pj = P.s_rj[q];
  const int64_t dst = P.s_dst[q];
  const double v = sdot(y, I.row_off + ri, I.row_off + P.can_local[pj]);
  if (dst < 0) d.sdiag[(pj < P.n_tail ? I.d_tail : I.d_own) + pj] = v;
  else d.bval[(pj < P.n_tail ? I.b_tail : I.b_own) + dst] = v;
}

// Left-looking Cholesky with pivot skipping, one CTA per listed instance,
// columns in canonical order. Column j starts from S[j:, j]; every k < j
// with L_jk != 0 (the row pattern of j) subtracts L_jk L[j:, k]. Warp w
// accumulates the k's of index w (mod NW) in its own buffer; the buffers are
// added in warp order, so the arithmetic is fixed. The pivot test is the
// row reduction's: row j is kept iff its pivot exceeds rank_tol S_jj;
// otherwise its column becomes zero and 1 / L_jj = 0, which makes its
// solution entries zero in the solves (its row entries are then never used).
template <int NW>
__global__ void __launch_bounds__(NW * 32) sp_factor_kernel(SpDev d, const int32_t* __restrict__ ilist, int first_only,
                                                            double rank_tol) {
  const int inst = ilist[blockIdx.x];
  const SpInstDev I = d.inst[inst];
  __shared__ SpPatDev sPf;
  if (threadIdx.x == 0) sPf = d.pats[I.pat];
  __syncthreads();
  const SpPatDev& P = sPf;
  extern __shared__ double smem[];
  const int LDA = d.max_col + 1;
  double* acc = smem;                                                    // [NW][LDA]
  int32_t* posmap = reinterpret_cast<int32_t*>(smem + (size_t)NW * LDA);  // [max_span + 1]
  __shared__ double s_inv;
  __shared__ int s_keep;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nt = P.n_tail;
  const int j0 = first_only ? nt : 0;
  for (int j = j0; j < P.n; ++j) {
    const int64_t cb = P.bptr[j], ce = P.bptr[j + 1];
    const int len = (int)(ce - cb);
    const double* colj = d.bval + ((j < nt) ? I.b_tail : I.b_own) + cb;  // column j (S values on entry)
    const int64_t db = (j < nt) ? I.d_tail : I.d_own;
    for (int t = tid; t < NW * (len + 1); t += NW * 32) {
      const int w = t / (len + 1), q = t - w * (len + 1);
      double v = 0.0;
      if (w == 0) v = (q == 0) ? d.sdiag[db + j] : colj[q - 1];
      acc[w * LDA + q] = v;
    }
    for (int t = tid; t < len; t += NW * 32) posmap[P.brow[cb + t] - j] = t + 1;
    __syncthreads();
    const int64_t rb = P.fptr[j], re = P.fptr[j + 1];
    double* aw = acc + warp * LDA;
    for (int64_t e = rb + warp; e < re; e += NW) {
      const int k = P.fcol[e];
      const double* colk = d.bval + ((k < nt) ? I.b_tail : I.b_own);  // column k (final values)
      const int64_t eb = P.fmap[e];                                   // (j, k) in column k
      const double ljk = colk[eb];
      if (ljk == 0.0) continue;
      if (lane == 0) aw[0] -= ljk * ljk;
      const int64_t ke = P.bptr[k + 1];
#pragma unroll 4
      for (int64_t e2 = eb + 1 + lane; e2 < ke; e2 += 32) {
        const int q = posmap[P.brow[e2] - j];  // in 1..len: column k's rows below j are rows of column j
        if ((unsigned)(q - 1) < (unsigned)len) aw[q] -= colk[e2] * ljk;
      }
    }
    __syncthreads();
    for (int q = tid; q <= len; q += NW * 32) {
      double c = acc[q];
#pragma unroll
      for (int w = 1; w < NW; ++w) c += acc[w * LDA + q];
      acc[q] = c;
    }
    __syncthreads();
    if (tid == 0) {
      const double piv = acc[0], ref = d.sdiag[db + j];
      const int keep = (ref > 0.0) && (piv > rank_tol * ref);
      s_keep = keep;
      s_inv = keep ? 1.0 / sqrt(piv) : 0.0;
      d.dinv[db + j] = s_inv;
      d.keep[I.row_off + P.can_local[j]] = (uint8_t)keep;
    }
    __syncthreads();
    const double inv = s_inv;
    const int keep = s_keep;
    double* colw = d.bval + ((j < nt) ? I.b_tail : I.b_own) + cb;
    for (int t = tid; t < len; t += NW * 32) colw[t] = keep ? acc[t + 1] * inv : 0.0;
    __syncthreads();
  }
}

// the row-order copy of the factor from the column-order one (blockIdx.y =
// listed instance; first_only: the rows of the first clique's group). The
// row-order values are placed by row: a row of the shared tail at f_tail,
// any other row at f_own, its entries in tail columns copied from the
// owner's column values, so a forward-solve load address never depends on a
// loaded column index.
__global__ void sp_rowcopy_kernel(SpDev d, const int32_t* __restrict__ ilist, int first_only) {
  const SpInstDev I = d.inst[ilist[blockIdx.y]];
  const SpPatDev P = d.pats[I.pat];
  const int64_t e0 = first_only ? P.tail_fwd : 0;
  const int64_t e = e0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= P.fptr[P.n]) return;
  const int j = P.fcol[e];
  const int64_t dst = ((e < P.tail_fwd) ? I.f_tail : I.f_own) + e;  // tail rows hold exactly the first tail_fwd entries
  d.fval[dst] = d.bval[((j < P.n_tail) ? I.b_tail : I.b_own) + P.fmap[e]];
}

// t = r + A rho on the other rows, into the working vector (blockIdx.y = instance)
__global__ void sp_rhs_kernel(SpDev d, YsolveDev y, const double* __restrict__ r, const double* __restrict__ rho) {
  const int inst = blockIdx.y;
  if (d.inst_active && !d.inst_active[inst]) return;
  const SpInstDev I = d.inst[inst];
  __shared__ SpPatDev sPf;
  if (threadIdx.x == 0) sPf = d.pats[I.pat];
  __syncthreads();
  const SpPatDev& P = sPf;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  const int64_t row = I.row_off + P.can_local[p];
  double t = r[row];
  for (int64_t e = y.rowptr[row]; e < y.rowptr[row + 1]; ++e) t += y.val[e] * rho[y.col[e]];
  d.w[I.w_off + p] = t;
}

// Inverse of the dense diagonal part of every substitution block (one warp
// per block, blockIdx.y = listed instance). A dropped row is taken as e_i in
// the block (its row entries are not part of the factor) and its row of the
// inverse is zeroed, so its solution entries come out as 0 in both passes.
// Stored column-major: inverse(row q, column k) at k * 32 + q.
constexpr int BINV_W = 4;  // warps (blocks) per CTA of the block inverse
__global__ void __launch_bounds__(BINV_W * 32) sp_blockinv_kernel(SpDev d, const int32_t* __restrict__ ilist,
                                                                  int first_only) {
  const SpInstDev I = d.inst[ilist[blockIdx.y]];
  const SpPatDev P = d.pats[I.pat];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bidx = blockIdx.x * BINV_W + warp;
  if (bidx >= P.nblk || (first_only && bidx < P.tail_blk)) return;
  __shared__ double Lt[BINV_W][kSpBlock][kSpBlock + 1];
  int lo = 0, hi = P.ngroups;  // group of the block: blk_grp[g] <= bidx < blk_grp[g + 1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (P.blk_grp[mid] <= bidx) lo = mid;
    else hi = mid;
  }
  const int g = lo;
  const int b0 = P.grp_ptr[g] + kSpBlock * (bidx - P.blk_grp[g]);
  const int bs = min(kSpBlock, P.grp_ptr[g + 1] - b0);
  const int nt = P.n_tail;
  double (*L)[kSpBlock + 1] = Lt[warp];
  // lane q builds row q
  {
    const int q = lane;
    for (int c = 0; c < kSpBlock; ++c) L[q][c] = 0.0;
    double dq = 0.0;
    if (q < bs) {
      const int i = b0 + q;
      dq = d.dinv[((i < nt) ? I.d_tail : I.d_own) + i];
      const double* rowv = d.fval + ((i < nt) ? I.f_tail : I.f_own);
      if (dq > 0.0)
        for (int64_t e = P.fsplit[i]; e < P.fptr[i + 1]; ++e) L[q][P.fcol[e] - b0] = rowv[e];
    }
    L[q][q] = (dq > 0.0) ? 1.0 / dq : 1.0;
    L[q][kSpBlock] = (q < bs && dq > 0.0) ? 1.0 : 0.0;  // mask of kept rows
  }
  __syncwarp();
  // lane k: column k of the inverse by forward substitution
  const int k = lane;
  double x[kSpBlock];
#pragma unroll
  for (int q = 0; q < kSpBlock; ++q) {
    double acc = (q == k) ? 1.0 : 0.0;
#pragma unroll
    for (int c = 0; c < q; ++c) acc -= L[q][c] * x[c];
    x[q] = (q >= k) ? acc / L[q][q] : 0.0;
  }
  double* Db = d.dinvb + ((bidx < P.tail_blk) ? I.v_tail : I.v_own) + (int64_t)bidx * (kSpBlock * kSpBlock);
#pragma unroll
  for (int q = 0; q < kSpBlock; ++q) Db[k * kSpBlock + q] = L[q][kSpBlock] * x[q];
}

// Forward and backward substitution for a tile of R instances with the same
// pattern (consecutive instances; R > 1 only when they share the tail).
// Groups are processed in canonical order with two group-sized buffers per
// instance in shared memory: by the block-bidiagonal structure a row reads
// only its own group and the group before it (forward), a column only its
// own group and the group after it (backward). Inside a group the positions
// are taken a block of 32 at a time:
//  forward  (L w = t):   when a group starts, every row subtracts its entries
//                        in the previous group (all rows at once, 8 lanes per
//                        row); then block by block, each row of the block
//                        subtracts its entries in earlier blocks of its group
//                        (8 lanes per row, a fixed 3-step sum), and the block
//                        is solved through the inverse of its diagonal part
//                        (8 lanes per output, a fixed 3-step sum)
//  backward (L^T y = w): the same with the columns' entries in the next group
//                        and in later blocks, and the transposed inverse,
//                        blocks and groups last to first
// The entries a step needs do not depend on the solution, so each step loads
// the next step's first entries (up to 64 of a row), its rows' entry ranges
// two steps ahead, and
// its block inverse while the current step computes: a step waits on shared
// memory and on the FP64 pipe, not on global memory. Two barriers a step.
// entries per lane loaded a step ahead: 8 (64 entries of a row) for one or
// two right-hand sides per CTA, fewer for more (registers); the per-lane
// order of the entries, and so the arithmetic, is the same for every choice
template <int R> struct SpPf { static constexpr int value = R <= 2 ? 8 : R == 4 ? 4 : 2; };
constexpr int SP_MAXG = kSpMaxGroups;

// walks the blocks of a pass in order (forward: first to last, backward: last
// to first); g = group, t = block inside it, b0 / bs = its first position and size
struct BlkIt {
  int g, t, b0, bs, bb;
  __device__ void set(const int* sg, const int* sb, int G) {
    if (g < 0 || g >= G) { bs = 0; b0 = 0; bb = -1; return; }
    b0 = sg[g] + kSpBlock * t;
    bs = min(kSpBlock, sg[g + 1] - b0);
    bb = sb[g] + t;
  }
  __device__ void first(const int* sg, const int* sb, int G, bool fwd) {
    g = fwd ? 0 : G - 1;
    t = fwd ? 0 : sb[G] - sb[G - 1] - 1;
    set(sg, sb, G);
  }
  __device__ void next(const int* sg, const int* sb, int G, bool fwd) {
    if (g < 0 || g >= G) return;
    if (fwd) {
      if (++t == sb[g + 1] - sb[g]) { ++g; t = 0; }
    } else {
      if (--t < 0) { --g; t = (g >= 0) ? sb[g + 1] - sb[g] - 1 : 0; }
    }
    set(sg, sb, G);
  }
};

// one pass of the substitution (FWD: L w = t; otherwise L^T y = w), in place
// in the group buffers; see sp_solve_kernel
template <int R, bool FWD>
__device__ void sp_pass_impl(const SpDev& d, const SpPatDev& P, const SpInstDev* sI, const int* s_act, int i0,
                        const int* sg, const int* sb, double* sh, double (*tb)[kSpBlock], double* __restrict__ yout) {
  constexpr int BS = kSpBlock;
  const int tid = threadIdx.x;
  const int MG = d.max_group;
  const int nt = P.n_tail, G = P.ngroups;
  auto buf = [&](int g, int r) -> double* { return sh + ((size_t)(g & 1) * R + r) * MG; };
  const int q = tid >> 3, l8 = tid & 7;     // gather: row / column q of the block, 8 lanes each
  // block inverse: output ioj, terms 4 ik .. 4 ik + 3 (8 lanes per output,
  // every warp busy: the FP64 pipe of each of the SM's four partitions)
  const int ioj = tid >> 3, ik = tid & 7;
  // entries of row / column p inside its group, in earlier blocks: [segb[p], sege[p])
  const int64_t* segb = FWD ? P.fgrp : P.bsplit;
  const int64_t* sege = FWD ? P.fsplit : P.bgrp;
  // entries in the group processed before this one: [cpb[p], cpe[p])
  const int64_t* cpb = FWD ? P.fptr : P.bgrp;
  const int64_t* cpe = FWD ? P.fgrp : P.bptr + 1;
  const int32_t* idx = FWD ? P.fcol : P.brow;
  // value table of a row (forward: placed by row) / column (backward)
  auto vals = [&](int r, int p) -> const double* {
    const SpInstDev& I = sI[r];
    return FWD ? d.fval + ((p < nt) ? I.f_tail : I.f_own) : d.bval + ((p < nt) ? I.b_tail : I.b_own);
  };
  constexpr int SP_PF = SpPf<R>::value;
  BlkIt itk, it1, it2;
  itk.first(sg, sb, G, FWD);
  it1 = itk; it1.next(sg, sb, G, FWD);
  it2 = it1; it2.next(sg, sb, G, FWD);
  int64_t cur_e = 0, cur_end = 0, nb_e = 0, nb_end = 0, nn_e = 0, nn_end = 0;
  int32_t pf_j[SP_PF];
  double pf_v[SP_PF][R];
  double dv[R][4];
  auto load_range = [&](const BlkIt& it, int64_t& e, int64_t& end) {
    e = 0; end = 0;
    if (q < it.bs) { e = segb[it.b0 + q] + l8; end = sege[it.b0 + q]; }
  };
  auto load_entries = [&](const BlkIt& it, int64_t e, int64_t end) {
    const int p = it.b0 + q;
#pragma unroll
    for (int t = 0; t < SP_PF; ++t) {
      const int64_t ee = e + 8 * t;
      const bool ok = ee < end;
      pf_j[t] = ok ? idx[ee] : -1;
#pragma unroll
      for (int r = 0; r < R; ++r) pf_v[t][r] = ok ? vals(r, p)[ee] : 0.0;
    }
  };
  auto load_inverse = [&](const BlkIt& it) {
    if (it.bs == 0) return;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const SpInstDev& I = sI[r];
      const double* Db = d.dinvb + ((it.bb < P.tail_blk) ? I.v_tail : I.v_own) + (int64_t)it.bb * (BS * BS);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int t = 4 * ik + i;
        dv[r][i] = FWD ? Db[t * BS + ioj] : Db[ioj * BS + t];
      }
    }
  };
  auto flush = [&](int g, int a, int b) {
    for (int t = tid; t < R * (b - a); t += SOLVE_T) {
      const int r = t / (b - a), i = t - r * (b - a);
      if (FWD) {
        if (i0 + r < d.ninst) d.w[sI[r].w_off + a + i] = buf(g, r)[i];
      } else if (s_act[r]) {
        yout[sI[r].row_off + P.can_local[a + i]] = buf(g, r)[i];
      }
    }
  };
  load_range(itk, cur_e, cur_end);
  load_range(it1, nb_e, nb_end);
  load_entries(itk, cur_e, cur_end);
  load_inverse(itk);
  int g = -1, a = 0, b = 0, pa = 0;
#pragma unroll 1
  while (itk.bs > 0) {
    if (itk.g != g) {  // a new group: flush the finished one, load this one's buffer
      if (g >= 0) flush(g, a, b);
      g = itk.g;
      a = sg[g];
      b = sg[g + 1];
      pa = (g > 0) ? sg[g - 1] : 0;
      __syncthreads();  // the buffer being refilled held a group two steps back
      for (int t = tid; t < R * (b - a); t += SOLVE_T) {
        const int r = t / (b - a), i = t - r * (b - a);
        buf(g, r)[i] = d.w[sI[r].w_off + a + i];
      }
      __syncthreads();
      // the coupling with the group processed before (its values are final):
      // every row of this group at once, 8 lanes a row, many loads in flight
      // instead of one block step's rows at a time
      if (g != (FWD ? 0 : G - 1)) {
        const int off_prev = FWD ? pa : b;
        for (int p0 = a; p0 < b; p0 += SOLVE_T / 8) {
          const int p = p0 + q;
          double cacc[R];
#pragma unroll
          for (int r = 0; r < R; ++r) cacc[r] = 0.0;
          if (p < b) {
            const int64_t e1 = cpe[p];
#pragma unroll 4
            for (int64_t e = cpb[p] + l8; e < e1; e += 8) {
              const int j = idx[e] - off_prev;
#pragma unroll
              for (int r = 0; r < R; ++r) cacc[r] += vals(r, p)[e] * buf(g + 1, r)[j];
            }
          }
#pragma unroll
          for (int r = 0; r < R; ++r) {
            double v = cacc[r];
            v += __shfl_xor_sync(0xffffffffu, v, 4);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            if (p < b && l8 == 0) buf(g, r)[p - a] -= v;
          }
        }
        __syncthreads();
      }
    }
    load_range(it2, nn_e, nn_end);
    const int b0 = itk.b0, bs = itk.bs;
    // forward: finished entries are in earlier blocks of this group or in the
    // group before (buf(g + 1)); backward: in later blocks or the group after
    auto val_at = [&](int r, int j) -> double {
      return FWD ? ((j >= a) ? buf(g, r)[j - a] : buf(g + 1, r)[j - pa])
                 : ((j < b) ? buf(g, r)[j - a] : buf(g + 1, r)[j - b]);
    };
    double acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0;
    if (q < bs) {
#pragma unroll
      for (int t = 0; t < SP_PF; ++t) {
        const int j = pf_j[t];
        if (j >= 0) {
#pragma unroll
          for (int r = 0; r < R; ++r) acc[r] += pf_v[t][r] * val_at(r, j);
        }
      }
      const int p = b0 + q;
#pragma unroll 4
      for (int64_t e = cur_e + 8 * SP_PF; e < cur_end; e += 8) {
        const int j = idx[e];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] += vals(r, p)[e] * val_at(r, j);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      double v = acc[r];
      v += __shfl_xor_sync(0xffffffffu, v, 4);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      if (q < bs && l8 == 0) tb[r][q] = buf(g, r)[b0 + q - a] - v;
    }
    // the next step's entries (their range was loaded a step ago)
    load_entries(it1, nb_e, nb_end);
    cur_e = nb_e; cur_end = nb_end;
    nb_e = nn_e; nb_end = nn_end;
    __syncthreads();
    // the block through the inverse of its diagonal part: each output as 8
    // partial sums of 4 terms, added by a fixed shuffle tree (the same
    // arithmetic for every tile size)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      double c = 0.0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int t = 4 * ik + i;
        c += (t < bs) ? dv[r][i] * tb[r][t] : 0.0;
      }
      c += __shfl_xor_sync(0xffffffffu, c, 1);
      c += __shfl_xor_sync(0xffffffffu, c, 2);
      c += __shfl_xor_sync(0xffffffffu, c, 4);
      if (ik == 0 && ioj < bs) buf(g, r)[b0 - a + ioj] = c;
    }
    load_inverse(it1);
    __syncthreads();
    itk = it1;
    it1 = it2;
    it2.next(sg, sb, G, FWD);
  }
  flush(g, a, b);
  __syncthreads();
}

template <int R>
__global__ void __launch_bounds__(SOLVE_T) sp_solve_kernel(SpDev d, double* __restrict__ yout) {
  static_assert(R >= 1 && R <= 8, "tiles of 1 to 8 instances");
  extern __shared__ double sh[];
  const int i0 = blockIdx.x * R;
  const int tid = threadIdx.x;
  __shared__ SpInstDev sI[R];
  __shared__ int s_act[R];
  __shared__ double tb[R][kSpBlock];  // the block's right-hand side after the gather
  __shared__ int sg[SP_MAXG + 1], sb[SP_MAXG + 1];
  __shared__ SpPatDev sP;
  if (tid < R) {
    const int i = min(i0 + tid, d.ninst - 1);
    sI[tid] = d.inst[i];
    s_act[tid] = (i0 + tid < d.ninst) && (d.inst_active == nullptr || d.inst_active[i0 + tid]);
  }
  __syncthreads();
  int any = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) any |= s_act[r];
  if (!any) return;
  if (tid == 0) sP = d.pats[sI[0].pat];
  __syncthreads();
  const SpPatDev& P = sP;  // in shared memory: the kernel's global stores cannot alias it
  for (int t = tid; t <= P.ngroups; t += SOLVE_T) {
    sg[t] = P.grp_ptr[t];
    sb[t] = P.blk_grp[t];
  }
  __syncthreads();
  sp_pass_impl<R, true>(d, P, sI, s_act, i0, sg, sb, sh, tb, yout);
  sp_pass_impl<R, false>(d, P, sI, s_act, i0, sg, sb, sh, tb, yout);
}

size_t factor_smem(const SpDev& d, int nw) {
  return sizeof(double) * (size_t)nw * (d.max_col + 1) + sizeof(int32_t) * (size_t)(d.max_span + 1);
}
size_t solve_smem(const SpDev& d, int r) { return sizeof(double) * 2 * (size_t)r * d.max_group; }

int factor_warps(const SpDev& d) {
  for (int nw : {8, 4, 2, 1})
    if (factor_smem(d, nw) <= 220 * 1024) return nw;
  return 0;
}

}  // namespace

void sparse_configure(const SpDev& d) {
  const int nw = factor_warps(d);
  if (nw == 0)
    throw StatusError(STROM_ERR_INVALID, "sparse factor: a column of L is too long for one CTA's shared memory");
  const int fs = (int)factor_smem(d, nw);
  if (nw == 8) STROM_CUDA(cudaFuncSetAttribute(sp_factor_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, fs));
  if (nw == 4) STROM_CUDA(cudaFuncSetAttribute(sp_factor_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, fs));
  if (nw == 2) STROM_CUDA(cudaFuncSetAttribute(sp_factor_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, fs));
  if (nw == 1) STROM_CUDA(cudaFuncSetAttribute(sp_factor_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, fs));
  const size_t ss = solve_smem(d, d.tile_r);
  if (ss > 200 * 1024)  // the kernel's static tables take about 11 KB more
    throw StatusError(STROM_ERR_INVALID, "sparse factor: two clique groups do not fit one CTA's shared memory");
  const int si = (int)ss;
  switch (d.tile_r) {
    case 1: STROM_CUDA(cudaFuncSetAttribute(sp_solve_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, si)); break;
    case 2: STROM_CUDA(cudaFuncSetAttribute(sp_solve_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, si)); break;
    case 4: STROM_CUDA(cudaFuncSetAttribute(sp_solve_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, si)); break;
    default: STROM_CUDA(cudaFuncSetAttribute(sp_solve_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, si)); break;
  }
}

void sparse_factor(const SpDev& d, const YsolveDev& y, const int32_t* ilist_dev, int nlist, bool first_only,
                   double rank_tol, cudaStream_t st, int64_t max_ns, int64_t max_nnz, int max_blk) {
  if (nlist == 0) return;
  const dim3 ga(ceil_div(std::max<int64_t>(1, max_ns), 256), nlist);
  sp_assemble_kernel<<<ga, 256, 0, st>>>(d, y, ilist_dev, first_only ? 1 : 0);
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
  const int nw = factor_warps(d);
  const size_t fs = factor_smem(d, nw);
  const int fo = first_only ? 1 : 0;
  if (nw == 8) sp_factor_kernel<8><<<nlist, 256, fs, st>>>(d, ilist_dev, fo, rank_tol);
  else if (nw == 4) sp_factor_kernel<4><<<nlist, 128, fs, st>>>(d, ilist_dev, fo, rank_tol);
  else if (nw == 2) sp_factor_kernel<2><<<nlist, 64, fs, st>>>(d, ilist_dev, fo, rank_tol);
  else sp_factor_kernel<1><<<nlist, 32, fs, st>>>(d, ilist_dev, fo, rank_tol);
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
  const dim3 gc(ceil_div(std::max<int64_t>(1, max_nnz), 256), nlist);
  sp_rowcopy_kernel<<<gc, 256, 0, st>>>(d, ilist_dev, fo);
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
  const dim3 gb(ceil_div(std::max(1, max_blk), BINV_W), nlist);
  sp_blockinv_kernel<<<gb, BINV_W * 32, 0, st>>>(d, ilist_dev, fo);
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
}

void sparse_solve(const SpDev& d, const YsolveDev& y, const double* r, const double* rho, double* yout,
                  cudaStream_t st, int max_n) {
  const dim3 gr(ceil_div(max_n, 256), d.ninst);
  sp_rhs_kernel<<<gr, 256, 0, st>>>(d, y, r, rho);
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
  const int R = d.tile_r;
  const int grid = (d.ninst + R - 1) / R;
  const size_t ss = solve_smem(d, R);
  switch (R) {
    case 1: sp_solve_kernel<1><<<grid, SOLVE_T, ss, st>>>(d, yout); break;
    case 2: sp_solve_kernel<2><<<grid, SOLVE_T, ss, st>>>(d, yout); break;
    case 4: sp_solve_kernel<4><<<grid, SOLVE_T, ss, st>>>(d, yout); break;
    default: sp_solve_kernel<8><<<grid, SOLVE_T, ss, st>>>(d, yout); break;
  }
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
}

}  // namespace strom
