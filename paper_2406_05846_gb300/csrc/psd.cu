// PSD cone projection of many small symmetric blocks (Sec. 4, parallel PSD
// cone projection): Pi(X_beta) = Q max(0, W) Q^T from X_beta = Q W Q^T.
//
// One CTA per block. The block is unpacked from svec into shared memory and
// diagonalised by the cyclic two-sided Jacobi method with the round-robin
// (tournament) ordering: in each round the np/2 rotations act on disjoint
// index pairs, so all of them are applied at once. Every 2x2 sub-block
// A[{p1,q1},{p2,q2}] is owned by one thread, which applies J1^T (.) J2 in
// registers, so a round needs one barrier after the rotation parameters and
// one after the update. The 2x2 symmetric Schur rotation is the one of
// Golub & Van Loan (Matrix Computations, Sec. 8.5). Sweeps stop when the sum
// of squares of the off-diagonal entries met during a sweep is below
// tol^2 ||A||_F^2. The recombination W = V diag(sqrt(max(lam, 0))),
// Pi = W W^T writes svec output directly, optionally fused with the ADMM
// update S = (Pi(X_b) - X_b) / sigma (eq. solve-S).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace strom {
namespace {

template <typename T> __device__ __forceinline__ T dsqrt_(T x);
template <> __device__ __forceinline__ double dsqrt_<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float dsqrt_<float>(float x) { return __fsqrt_rn(x); }
// 1 / sqrt(x) with correctly rounded sqrt and division: an approximate
// reciprocal square root would make every rotation slightly non-orthogonal
// and the error would grow with the number of rotations applied to V.
template <typename T> __device__ __forceinline__ T drsqrt_(T x);
template <> __device__ __forceinline__ double drsqrt_<double>(double x) { return 1.0 / sqrt(x); }
template <> __device__ __forceinline__ float drsqrt_<float>(float x) { return __fdiv_rn(1.0f, __fsqrt_rn(x)); }

template <int NT>
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < NT / 32; ++i) s += red[i];
  return s;
}

template <typename T> struct Vec2;
template <> struct Vec2<float> {
  using type = float2;
  static __device__ __forceinline__ float2 make(float a, float b) { return make_float2(a, b); }
};
template <> struct Vec2<double> {
  using type = double2;
  static __device__ __forceinline__ double2 make(double a, double b) { return make_double2(a, b); }
};

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int W = 2; };

template <typename T, int NP, int NT, bool VSMEM>
struct JacobiSmem {
  static constexpr int LD = NP + 1;                  // A, row-major, odd stride
  static constexpr int W = Vec<T>::W;
  static constexpr int LDV = NP + W;                 // V^T rows, 16-byte aligned
  static constexpr int H = NP / 2;
  static constexpr size_t a_bytes = ((sizeof(T) * NP * LD + 15) / 16) * 16;
  static constexpr size_t v_bytes = VSMEM ? sizeof(T) * NP * LDV : 0;
  static constexpr size_t rot_bytes = (sizeof(T) * 3 + sizeof(int) * 2) * H;
  static constexpr size_t red_bytes = sizeof(double) * (NT / 32 + 2);
  // T = A V^T of the warm start (FP32 classes with V in shared memory and NP <= 80)
  static constexpr bool WARM = VSMEM && (NP <= 80);
  static constexpr size_t t_bytes = WARM ? ((sizeof(T) * NP * LD + 15) / 16) * 16 : 0;
  static constexpr size_t total = a_bytes + v_bytes + rot_bytes + red_bytes + t_bytes + 64;
  static constexpr int MAXA = (H * (H + 1) / 2 + NT - 1) / NT;     // 2x2 blocks (t1 <= t2) per thread
  static constexpr int MAXV = (H * ((NP + W - 1) / W) + NT - 1) / NT;  // (pair, vector chunk) per thread
};

// One CTA diagonalises one block. A (full, symmetric) lives in shared memory;
// the eigenvector matrix is kept transposed (row k = eigenvector k) so a
// rotation of columns p, q of V is a rotation of two contiguous rows,
// applied with 16-byte vector loads. Only the 2x2 blocks with t1 <= t2 are
// computed; each one also writes its mirror image.
template <typename T, int NP, int NT, bool VSMEM>
__global__ void __launch_bounds__(NT) jacobi_psd_kernel(PsdArgs a, int list_start, double tol, int max_sweeps) {
  using SM = JacobiSmem<T, NP, NT, VSMEM>;
  using VT = typename Vec<T>::type;
  constexpr int LD = SM::LD, LDV = SM::LDV, W = SM::W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  T* V = VSMEM ? reinterpret_cast<T*>(smem_raw + SM::a_bytes)
               : reinterpret_cast<T*>(a.vscratch) + (size_t)blockIdx.x * NP * LDV;
  // rotation of pair t: (s, tau) together, (p, q) together, one load each
  using T2 = typename Vec2<T>::type;
  T2* sSU = reinterpret_cast<T2*>(smem_raw + SM::a_bytes + SM::v_bytes);
  int2* sPQ = reinterpret_cast<int2*>(sSU + SM::H);
  T* sT = reinterpret_cast<T*>(sPQ + SM::H);
  double* red = reinterpret_cast<double*>(smem_raw + SM::a_bytes + SM::v_bytes + SM::rot_bytes + 16);
  red = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(red) + 7) & ~uintptr_t(7));
  T* Tm = reinterpret_cast<T*>(smem_raw + ((SM::a_bytes + SM::v_bytes + SM::rot_bytes + SM::red_bytes + 16 + 15) / 16) * 16);

  const int tid = threadIdx.x;
  const int bid = a.blk_list[list_start + blockIdx.x];
  if (a.blk_active != nullptr && a.blk_active[bid] == 0) return;
  const int n = a.blk_n[bid];
  const int np = n + (n & 1);
  const int half = np / 2;
  // warm start: the eigenvectors of this block from the instance's previous
  // iteration in the same precision (FP32 store / FP64 store)
  bool warm = false;
  if constexpr (SM::WARM) {
    if (sizeof(T) == 4 && a.vstore != nullptr) warm = (a.inst_iter[a.blk_inst[bid]] % a.warm_period) != 0;
    if (sizeof(T) == 8 && a.vstore64 != nullptr) warm = (a.inst_iter64[a.blk_inst[bid]] % a.warm_period) != 0;
  }
  const int64_t off = a.blk_off[bid];
  const double* __restrict__ xb = a.Xb + off;

  // ---- unpack svec -> full symmetric matrix; V^T = I (padding included)
  double fro = 0.0;
  for (int idx = tid; idx < np * np; idx += NT) {
    const int i = idx % np, j = idx / np;
    T v = T(0);
    if (i < n && j < n) {
      const int ii = min(i, j), jj = max(i, j);
      const double x = xb[(int64_t)jj * (jj + 1) / 2 + ii];
      const double e = (ii == jj) ? x : x * 0.70710678118654752440;
      v = (T)e;
      fro += e * e;
    }
    A[i * LD + j] = v;
  }
  if (warm) {
    if constexpr (sizeof(T) == 4) {
      const float* vs = a.vstore + a.vstore_off[bid];
      for (int idx = tid; idx < np * LDV; idx += NT) {
        const int k = idx / LDV, i = idx - (idx / LDV) * LDV;
        V[idx] = (i < np) ? (T)vs[k * np + i] : T(0);
      }
    } else {
      const double* vs = a.vstore64 + a.vstore_off[bid];
      for (int idx = tid; idx < np * LDV; idx += NT) {
        const int k = idx / LDV, i = idx - (idx / LDV) * LDV;
        V[idx] = (i < np) ? (T)vs[k * np + i] : T(0);
      }
    }
  } else {
    for (int idx = tid; idx < np * LDV; idx += NT) {
      const int k = idx / LDV, i = idx - (idx / LDV) * LDV;
      V[idx] = (i == k) ? T(1) : T(0);
    }
  }
  fro = block_sum<NT>(fro, red);   // contains a barrier
  if constexpr (SM::WARM && sizeof(T) == 4 && NP > 40) {
    if (warm && a.reorth) {
      // One Newton-Schulz step towards orthonormal rows,
      // V <- (3 V - (V V^T) V) / 2. The stored FP32 eigenvectors drift from
      // orthogonality over the iterations between cold restarts; on the
      // cart-pole's 78 x 78 blocks that drift leaves the projection an error
      // floor near 1e-5, which the sigma rule answers by shrinking sigma
      // until the iteration diverges. G = V V^T goes to Tm (free until the
      // warm start below), the new rows to registers, then back to V.
      const int h2 = np / 2, nt2 = h2 * h2;
      for (int it = tid; it < nt2; it += NT) {
        const int i0 = 2 * (it / h2), j0 = 2 * (it % h2);
        T g00 = 0, g01 = 0, g10 = 0, g11 = 0;
        for (int k = 0; k < np; ++k) {
          const T a0 = V[i0 * LDV + k], a1 = V[(i0 + 1) * LDV + k];
          const T b0 = V[j0 * LDV + k], b1 = V[(j0 + 1) * LDV + k];
          g00 += a0 * b0; g01 += a0 * b1; g10 += a1 * b0; g11 += a1 * b1;
        }
        Tm[i0 * LD + j0] = g00; Tm[i0 * LD + j0 + 1] = g01;
        Tm[(i0 + 1) * LD + j0] = g10; Tm[(i0 + 1) * LD + j0 + 1] = g11;
      }
      __syncthreads();
      constexpr int MAXT = ((NP / 2) * (NP / 2) + NT - 1) / NT;
      T nv[MAXT][4];
#pragma unroll
      for (int m = 0; m < MAXT; ++m) {
        const int it = tid + m * NT;
        if (it < nt2) {
          const int i0 = 2 * (it / h2), c0 = 2 * (it % h2);
          T s00 = 0, s01 = 0, s10 = 0, s11 = 0;
          for (int k = 0; k < np; ++k) {
            const T g0 = Tm[i0 * LD + k], g1 = Tm[(i0 + 1) * LD + k];
            const T v0 = V[k * LDV + c0], v1 = V[k * LDV + c0 + 1];
            s00 += g0 * v0; s01 += g0 * v1; s10 += g1 * v0; s11 += g1 * v1;
          }
          nv[m][0] = T(1.5) * V[i0 * LDV + c0] - T(0.5) * s00;
          nv[m][1] = T(1.5) * V[i0 * LDV + c0 + 1] - T(0.5) * s01;
          nv[m][2] = T(1.5) * V[(i0 + 1) * LDV + c0] - T(0.5) * s10;
          nv[m][3] = T(1.5) * V[(i0 + 1) * LDV + c0 + 1] - T(0.5) * s11;
        }
      }
      __syncthreads();
#pragma unroll
      for (int m = 0; m < MAXT; ++m) {
        const int it = tid + m * NT;
        if (it < nt2) {
          const int i0 = 2 * (it / h2), c0 = 2 * (it % h2);
          V[i0 * LDV + c0] = nv[m][0]; V[i0 * LDV + c0 + 1] = nv[m][1];
          V[(i0 + 1) * LDV + c0] = nv[m][2]; V[(i0 + 1) * LDV + c0 + 1] = nv[m][3];
        }
      }
      __syncthreads();
    }
  }
  if constexpr (SM::WARM) {
    if (warm) {
      // B = V X V^T in the stored eigenbasis (V^T rows are the eigenvectors):
      // Tm = A V^T, then A = V Tm, each thread a 2x2 tile
      const int nt2 = (np / 2) * (np / 2);
      for (int it = tid; it < nt2; it += NT) {
        const int i0 = 2 * (it / (np / 2)), j0 = 2 * (it % (np / 2));
        T c00 = 0, c01 = 0, c10 = 0, c11 = 0;
        for (int k = 0; k < np; ++k) {
          const T a0 = A[i0 * LD + k], a1 = A[(i0 + 1) * LD + k];
          const T v0 = V[j0 * LDV + k], v1 = V[(j0 + 1) * LDV + k];
          c00 += a0 * v0; c01 += a0 * v1; c10 += a1 * v0; c11 += a1 * v1;
        }
        Tm[i0 * LD + j0] = c00; Tm[i0 * LD + j0 + 1] = c01;
        Tm[(i0 + 1) * LD + j0] = c10; Tm[(i0 + 1) * LD + j0 + 1] = c11;
      }
      __syncthreads();
      for (int it = tid; it < nt2; it += NT) {
        const int i0 = 2 * (it / (np / 2)), j0 = 2 * (it % (np / 2));
        if (j0 < i0) continue;  // upper 2x2 tiles, mirrored below
        T c00 = 0, c01 = 0, c10 = 0, c11 = 0;
        for (int k = 0; k < np; ++k) {
          const T v0 = V[i0 * LDV + k], v1 = V[(i0 + 1) * LDV + k];
          const T t0 = Tm[k * LD + j0], t1 = Tm[k * LD + j0 + 1];
          c00 += v0 * t0; c01 += v0 * t1; c10 += v1 * t0; c11 += v1 * t1;
        }
        if (i0 == j0) {
          const T o = T(0.5) * (c01 + c10);
          A[i0 * LD + i0] = c00; A[(i0 + 1) * LD + i0 + 1] = c11;
          A[i0 * LD + i0 + 1] = o; A[(i0 + 1) * LD + i0] = o;
        } else {
          A[i0 * LD + j0] = c00; A[i0 * LD + j0 + 1] = c01;
          A[(i0 + 1) * LD + j0] = c10; A[(i0 + 1) * LD + j0 + 1] = c11;
          A[j0 * LD + i0] = c00; A[(j0 + 1) * LD + i0] = c01;
          A[j0 * LD + i0 + 1] = c10; A[(j0 + 1) * LD + i0 + 1] = c11;
        }
      }
      __syncthreads();
    }
  }

  // ---- this thread's work items, fixed for all rounds
  const int nAit = half * (half + 1) / 2;
  const int nchunk = (np + W - 1) / W;
  const int nVit = half * nchunk;
  uint32_t itA[SM::MAXA], itV[SM::MAXV];
#pragma unroll
  for (int i = 0; i < SM::MAXA; ++i) {
    const int idx = tid + i * NT;
    uint32_t code = 0xffffffffu;
    if (idx < nAit) {
      int t1 = 0, base = 0;
      while (base + (half - t1) <= idx) { base += half - t1; ++t1; }
      const int t2 = t1 + (idx - base);
      code = ((uint32_t)t1 << 16) | (uint32_t)t2;
    }
    itA[i] = code;
  }
#pragma unroll
  for (int i = 0; i < SM::MAXV; ++i) {
    const int idx = tid + i * NT;
    itV[i] = (idx < nVit) ? (((uint32_t)(idx / nchunk) << 16) | (uint32_t)(idx % nchunk)) : 0xffffffffu;
  }

  // ---- cyclic Jacobi sweeps, round-robin ordering
  const double thr = tol * tol * fro;
  for (int sweep = 0; sweep < max_sweeps && np > 1; ++sweep) {
    double off_sum = 0.0;
    for (int r = 0; r < np - 1; ++r) {
      if (tid < half) {
        const int t = tid;
        const int pa = (t == 0) ? 0 : ((t - 1 + r) % (np - 1)) + 1;
        const int pb = ((np - 2 - t + r) % (np - 1)) + 1;
        const int p = min(pa, pb), q = max(pa, pb);
        const T app = A[p * LD + p], aqq = A[q * LD + q], apq = A[p * LD + q];
        // tangent t, sine s and tau = s / (1 + c) of the 2x2 symmetric Schur rotation
        T tt = T(0), s = T(0), ta = T(0);
        off_sum += (double)apq * (double)apq;
        if (apq != T(0)) {
          const T tau = (aqq - app) / (T(2) * apq);
          const T at = fabs(tau);
          if (at > T(1e15)) tt = T(0.5) / tau;  // 1 + tau^2 would lose tau's size
          else tt = (tau >= T(0) ? T(1) : T(-1)) / (at + dsqrt_<T>(T(1) + tau * tau));
          const T c = drsqrt_<T>(T(1) + tt * tt);
          s = tt * c;
          ta = s / (T(1) + c);
        }
        sPQ[t] = make_int2(p, q);
        sT[t] = tt;
        sSU[t] = Vec2<T>::make(s, ta);
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < SM::MAXA; ++i) {
        const uint32_t code = itA[i];
        if (code == 0xffffffffu) continue;
        const int t1 = (int)(code >> 16), t2 = (int)(code & 0xffffu);
        const int2 pq1 = sPQ[t1], pq2 = sPQ[t2];
        const int p1 = pq1.x, q1 = pq1.y, p2 = pq2.x, q2 = pq2.y;
        const T x00 = A[p1 * LD + p2], x01 = A[p1 * LD + q2];
        const T x10 = A[q1 * LD + p2], x11 = A[q1 * LD + q2];
        if (t1 == t2) {
          // annihilated pair: a_pp - t a_pq, a_qq + t a_pq, a_pq = 0
          const T tt = sT[t1];
          A[p1 * LD + p1] = x00 - tt * x01;
          A[q1 * LD + q1] = x11 + tt * x01;
          A[p1 * LD + q1] = T(0);
          A[q1 * LD + p1] = T(0);
        } else {
          // J1^T X J2 written as corrections x - s (y + tau x) (Rutishauser):
          // no rounding bias from c ~ 1 when the rotation is small
          const T2 su1 = sSU[t1], su2 = sSU[t2];
          const T s1 = su1.x, u1 = su1.y, s2 = su2.x, u2 = su2.y;
          const T r00 = x00 - s1 * (x10 + u1 * x00), r10 = x10 + s1 * (x00 - u1 * x10);
          const T r01 = x01 - s1 * (x11 + u1 * x01), r11 = x11 + s1 * (x01 - u1 * x11);
          const T y00 = r00 - s2 * (r01 + u2 * r00);
          const T y01 = r01 + s2 * (r00 - u2 * r01);
          const T y10 = r10 - s2 * (r11 + u2 * r10);
          const T y11 = r11 + s2 * (r10 - u2 * r11);
          A[p1 * LD + p2] = y00; A[p1 * LD + q2] = y01;
          A[q1 * LD + p2] = y10; A[q1 * LD + q2] = y11;
          A[p2 * LD + p1] = y00; A[q2 * LD + p1] = y01;
          A[p2 * LD + q1] = y10; A[q2 * LD + q1] = y11;
        }
      }
#pragma unroll
      for (int i = 0; i < SM::MAXV; ++i) {
        const uint32_t code = itV[i];
        if (code == 0xffffffffu) continue;
        const int t = (int)(code >> 16), c = (int)(code & 0xffffu);
        const int2 pq = sPQ[t];
        const int p = pq.x, q = pq.y;
        const T2 su = sSU[t];
        const T s = su.x, u = su.y;
        VT* vp = reinterpret_cast<VT*>(V + p * LDV) + c;
        VT* vq = reinterpret_cast<VT*>(V + q * LDV) + c;
        VT a4 = *vp, b4 = *vq;
        T* ae = reinterpret_cast<T*>(&a4);
        T* be = reinterpret_cast<T*>(&b4);
#pragma unroll
        for (int e = 0; e < W; ++e) {
          const T x = ae[e], y = be[e];
          ae[e] = x - s * (y + u * x);
          be[e] = y + s * (x - u * y);
        }
        *vp = a4;
        *vq = b4;
      }
      __syncthreads();
    }
    off_sum = block_sum<NT>(off_sum, red);
    if (off_sum <= thr) break;
  }

  if constexpr (SM::WARM) {
    if (sizeof(T) == 4 && a.vstore != nullptr) {
      float* vs = a.vstore + a.vstore_off[bid];
      for (int idx = tid; idx < np * np; idx += NT) {
        const int k = idx / np, i = idx - (idx / np) * np;
        vs[idx] = (float)V[k * LDV + i];
      }
    }
    if (sizeof(T) == 8 && a.vstore64 != nullptr) {
      double* vs = a.vstore64 + a.vstore_off[bid];
      for (int idx = tid; idx < np * np; idx += NT) {
        const int k = idx / np, i = idx - (idx / np) * np;
        vs[idx] = (double)V[k * LDV + i];
      }
    }
    // the recombination below scales V in place: every thread must have
    // copied its share of the eigenvectors out first
    __syncthreads();
  }

  // ---- eigen outputs (ascending eigenvalues, top eigenvector)
  if (a.lam != nullptr || a.topvec != nullptr) {
    const int64_t lo = a.lam_off[bid];
    if (a.lam != nullptr) {
      for (int i = tid; i < n; i += NT) {
        const T li = A[i * LD + i];
        int rank = 0;
        for (int j = 0; j < n; ++j) {
          const T lj = A[j * LD + j];
          rank += (lj < li) || (lj == li && j < i);
        }
        a.lam[lo + rank] = (double)li;
      }
    }
    if (a.topvec != nullptr) {
      __shared__ int s_arg;
      if (tid == 0) {
        int best = 0;
        for (int j = 1; j < n; ++j) if (A[j * LD + j] > A[best * LD + best]) best = j;
        s_arg = best;
      }
      __syncthreads();
      const int kk = s_arg;
      for (int i = tid; i < n; i += NT) a.topvec[lo + i] = (double)V[kk * LDV + i];
    }
    __syncthreads();
  }
  if (a.out == nullptr) return;

  // ---- recombination Pi = W^T W with W = diag(sqrt(max(lam, 0))) V^T
  for (int idx = tid; idx < np * LDV; idx += NT) {
    const int k = idx / LDV;
    const T lk = (k < n) ? A[k * LD + k] : T(0);
    V[idx] = (lk > T(0)) ? V[idx] * dsqrt_<T>(lk) : T(0);
  }
  __syncthreads();
  const int nt = n * (n + 1) / 2;
  const double inv_sigma = (a.blk_inv_sigma != nullptr) ? a.blk_inv_sigma[bid] : 0.0;
  double* __restrict__ out = a.out + off;
  for (int idx = tid; idx < nt; idx += NT) {
    int j = (int)((sqrt(8.0 * idx + 1.0) - 1.0) * 0.5);
    while ((j + 1) * (j + 2) / 2 <= idx) ++j;
    while (j * (j + 1) / 2 > idx) --j;
    const int i = idx - j * (j + 1) / 2;
    T acc = T(0);
    for (int k = 0; k < n; ++k) acc += V[k * LDV + i] * V[k * LDV + j];
    double x = (double)acc;
    if (i != j) x *= 1.41421356237309504880;
    if (a.blk_inv_sigma != nullptr) x = (x - xb[idx]) * inv_sigma;
    out[idx] = x;
  }
}

template <typename T, int NP, int NT, bool VSMEM>
void set_attr() {
  using SM = JacobiSmem<T, NP, NT, VSMEM>;
  STROM_CUDA(cudaFuncSetAttribute(jacobi_psd_kernel<T, NP, NT, VSMEM>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::total));
}

template <typename T, int NP, int NT, bool VSMEM>
void launch_class(const PsdArgs& a, int start, int count, double tol, int sweeps, cudaStream_t st) {
  if (count == 0) return;
  using SM = JacobiSmem<T, NP, NT, VSMEM>;
  jacobi_psd_kernel<T, NP, NT, VSMEM><<<count, NT, SM::total, st>>>(a, start, tol, sweeps);
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
}

}  // namespace

namespace {

// Launch shapes per size class: the block size of a class is fixed by its
// shared-memory layout (NP); the thread count is a free choice (more threads:
// fewer 2x2 updates each, fewer CTAs per SM). The first entry is the default.
constexpr int kThr64[4][3] = {{64, 32, 0}, {128, 64, 256}, {256, 128, 512}, {512, 256, 0}};
constexpr int kThr32[4][3] = {{64, 32, 0}, {128, 64, 256}, {256, 128, 512}, {512, 256, 0}};

template <typename T, int NP, bool VSMEM, int NT0, int NT1, int NT2>
void set_attrs() {
  set_attr<T, NP, NT0, VSMEM>();
  set_attr<T, NP, NT1, VSMEM>();
  if constexpr (NT2 > 0) set_attr<T, NP, NT2, VSMEM>();
}

template <typename T, int NP, bool VSMEM, int NT0, int NT1, int NT2>
void launch_sel(int threads, const PsdArgs& a, int start, int count, double tol, int sweeps, cudaStream_t st) {
  if (threads == NT1) launch_class<T, NP, NT1, VSMEM>(a, start, count, tol, sweeps, st);
  else if (NT2 > 0 && threads == NT2) launch_class<T, NP, (NT2 > 0 ? NT2 : NT0), VSMEM>(a, start, count, tol, sweeps, st);
  else launch_class<T, NP, NT0, VSMEM>(a, start, count, tol, sweeps, st);
}

__global__ void fill_test_kernel(double* x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t h = (uint64_t)i * 0x9E3779B97F4A7C15ull;
    h ^= h >> 31;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 29;
    x[i] = (double)(h >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

}  // namespace

int psd_threads_candidates(int precision, int k, int* out) {
  const int(*t)[3] = precision == STROM_PREC_FP64 ? kThr64 : kThr32;
  int c = 0;
  for (int j = 0; j < 3; ++j)
    if (t[k][j] > 0) out[c++] = t[k][j];
  return c;
}

void psd_fill_test_input(double* x, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  fill_test_kernel<<<(int)std::min<int64_t>(4096, (n + 255) / 256), 256, 0, st>>>(x, n);
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
}

// The shared-memory attributes are per device: each device is configured once,
// under a lock so that host threads calling at the same time do not race.
void psd_configure() {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static bool done[kMaxDev] = {};
  int dev = 0;
  STROM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev) throw StatusError(STROM_ERR_INVALID, "psd_configure: device index out of range");
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return;
  set_attrs<double, 16, true, 64, 32, 0>();
  set_attrs<double, 40, true, 128, 64, 256>();
  set_attrs<double, 80, true, 256, 128, 512>();
  set_attrs<double, 160, false, 512, 256, 0>();
  set_attrs<float, 16, true, 64, 32, 0>();
  set_attrs<float, 40, true, 128, 64, 256>();
  set_attrs<float, 80, true, 256, 128, 512>();
  set_attrs<float, 160, true, 512, 256, 0>();
  done[dev] = true;
}

void psd_launch(const PsdArgs& a, const PsdClasses& c, int precision, cudaStream_t st) {
  psd_configure();
  if (precision == STROM_PREC_FP64) {
    const double tol = 1e-14;
    const int sw = 30;
    const int* th = c.threads[0];
    launch_sel<double, 16, true, 64, 32, 0>(th[0], a, c.start[0], c.count[0], tol, sw, st);
    launch_sel<double, 40, true, 128, 64, 256>(th[1], a, c.start[1], c.count[1], tol, sw, st);
    launch_sel<double, 80, true, 256, 128, 512>(th[2], a, c.start[2], c.count[2], tol, sw, st);
    launch_sel<double, 160, false, 512, 256, 0>(th[3], a, c.start[3], c.count[3], tol, sw, st);
  } else {
    const double tol = 2e-6;
    const int sw = 20;
    const int* th = c.threads[1];
    launch_sel<float, 16, true, 64, 32, 0>(th[0], a, c.start[0], c.count[0], tol, sw, st);
    launch_sel<float, 40, true, 128, 64, 256>(th[1], a, c.start[1], c.count[1], tol, sw, st);
    launch_sel<float, 80, true, 256, 128, 512>(th[2], a, c.start[2], c.count[2], tol, sw, st);
    launch_sel<float, 160, true, 512, 256, 0>(th[3], a, c.start[3], c.count[3], tol, sw, st);
  }
}

}  // namespace strom

// ---------------------------------------------------------------------------
// C ABI: PSD projection plans
// ---------------------------------------------------------------------------
struct strom_psd_plan {
  int nblk = 0;
  int precision = STROM_PREC_FP64;
  strom::PsdClasses cls;
  strom::DevBuf<int64_t> off, lam_off;
  strom::DevBuf<int32_t> n, list;
  strom::DevBuf<double> vscratch;
};

namespace strom {
int class_of(int n) { return n <= 16 ? 0 : n <= 40 ? 1 : n <= 80 ? 2 : 3; }

void build_classes(const int32_t* blk_n, int nblk, std::vector<int32_t>& list, PsdClasses& c) {
  std::vector<std::vector<int32_t>> per(4);
  for (int i = 0; i < nblk; ++i) per[class_of(blk_n[i])].push_back(i);
  list.clear();
  for (int k = 0; k < 4; ++k) {
    c.start[k] = (int)list.size();
    c.count[k] = (int)per[k].size();
    for (int b : per[k]) { list.push_back(b); c.max_n[k] = std::max(c.max_n[k], blk_n[b]); }
  }
}
}  // namespace strom

extern "C" int strom_psd_plan_create(const int64_t* blk_off, const int32_t* blk_n, int32_t nblk, int32_t precision,
                                     strom_psd_plan** out) {
  try {
    if (!out || nblk < 0 || (nblk > 0 && (!blk_off || !blk_n)))
      throw strom::StatusError(STROM_ERR_INVALID, "strom_psd_plan_create: bad arguments");
    if (precision != STROM_PREC_FP64 && precision != STROM_PREC_FP32)
      throw strom::StatusError(STROM_ERR_INVALID, "strom_psd_plan_create: precision must be FP64 or FP32");
    for (int i = 0; i < nblk; ++i)
      if (blk_n[i] < 1 || blk_n[i] > 160 || blk_off[i] < 0)
        throw strom::StatusError(STROM_ERR_INVALID, "strom_psd_plan_create: block size must be in 1..160");
    auto* p = new strom_psd_plan();
    p->nblk = nblk;
    p->precision = precision;
    std::vector<int32_t> list;
    strom::build_classes(blk_n, nblk, list, p->cls);
    std::vector<int64_t> lo(nblk);
    int64_t acc = 0;
    for (int i = 0; i < nblk; ++i) { lo[i] = acc; acc += blk_n[i]; }
    p->off.upload(blk_off, nblk);
    p->n.upload(blk_n, nblk);
    p->list.upload(list.data(), list.size());
    p->lam_off.upload(lo.data(), nblk);
    if (precision == STROM_PREC_FP64 && p->cls.count[3] > 0) p->vscratch.alloc((size_t)p->cls.count[3] * strom::kVScratchPerBlock);
    STROM_CUDA(cudaDeviceSynchronize());
    *out = p;
    return STROM_OK;
  } catch (const strom::StatusError& e) {
    strom::set_error(e.what());
    return e.status;
  } catch (const std::exception& e) {
    strom::set_error(e.what());
    return STROM_ERR_CUDA;
  }
}

extern "C" void strom_psd_plan_destroy(strom_psd_plan* p) { delete p; }

extern "C" int strom_psd_execute(strom_psd_plan* p, const double* Xb_dev, double* P_dev, double* lam_dev, void* stream) {
  try {
    if (!p || !Xb_dev || (!P_dev && !lam_dev) || (P_dev != nullptr && P_dev == Xb_dev))
      throw strom::StatusError(STROM_ERR_INVALID, "strom_psd_execute: bad arguments");
    strom::PsdArgs a{};
    a.Xb = Xb_dev;
    a.out = P_dev;
    a.blk_off = p->off.p;
    a.blk_n = p->n.p;
    a.blk_list = p->list.p;
    a.lam = lam_dev;
    a.lam_off = p->lam_off.p;
    a.vscratch = p->vscratch.p;
    strom::psd_launch(a, p->cls, p->precision, (cudaStream_t)stream);
    return STROM_OK;
  } catch (const strom::StatusError& e) {
    strom::set_error(e.what());
    return e.status;
  } catch (const std::exception& e) {
    strom::set_error(e.what());
    return STROM_ERR_CUDA;
  }
}

extern "C" int strom_kernel_psd_project(const double* Xb_dev, const int64_t* blk_off, const int32_t* blk_n,
                                        int32_t nblk, int32_t precision, double* P_dev, void* stream) {
  strom_psd_plan* p = nullptr;
  int st = strom_psd_plan_create(blk_off, blk_n, nblk, precision, &p);
  if (st != STROM_OK) return st;
  st = strom_psd_execute(p, Xb_dev, P_dev, nullptr, stream);
  if (st == STROM_OK) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) { strom::set_error(cudaGetErrorString(e)); st = STROM_ERR_CUDA; }
  }
  strom_psd_plan_destroy(p);
  return st;
}
