// End-of-solve certificate (host part; eigenvalues come from the GPU):
//  * rank-1 test lambda_2 / lambda_1 of every M_k (Theorem 1 iii);
//  * extraction: top eigenvector of M_k normalised by its first entry, its
//    degree-1 entries give z_bar(I_k) (Sec. 2.2, extraction heuristic);
//  * local step: controls clipped to [-R, R], each clique's equalities solved
//    for its new state by Gauss-Newton (the paper uses fmincon here);
//  * valid lower bound <b,y> + sum_beta R_beta min(0, lambda_min((C-A^T y)_beta))
//    (eq. valid-lowerbound) and xi (eq. suboptimality-gap), with R_beta from
//    the theorem of App. C: s(n, kappa) max(1,R)^(2 kappa) for moment blocks,
//    gmax s(n, kappa - d_g) max(1,R)^(2(kappa - d_g)) for localizing blocks,
//    gmax = sum_t |c_t| max(1,R)^deg(t) (an upper bound of max g on the box).
#include <algorithm>
#include <cmath>
#include <stdexcept>
#include <string>
#include <vector>

#include "internal.h"

namespace strom {
void solver_eig_blocks(strom_solver* s, int inst, bool use_Z, std::vector<double>& lam, std::vector<double>& topvec);
void solver_eig_all(strom_solver* s, bool use_Z, std::vector<double>& lam, std::vector<double>& topvec,
                    std::vector<int64_t>& lam_off, std::vector<double>& stats);
int solver_inst_blocks(const strom_solver* s, int inst, std::vector<int32_t>& n, std::vector<int8_t>& kind,
                       std::vector<int32_t>& clique, int64_t* first_blk);
int solver_blocks_of(const strom_solver* s, int inst, std::vector<int32_t>& n, std::vector<int8_t>& kind,
                     std::vector<int32_t>& clique, std::vector<int64_t>& lam_off, double* by);

namespace {

double ipow(double x, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

double peval(const Poly& p, int nv, const double* z) {
  double s = 0.0;
  for (int t = 0; t < p.nterms(); ++t) {
    double v = p.coef[t];
    for (int i = 0; i < nv; ++i) v *= ipow(z[i], p.expo[(size_t)t * nv + i]);
    s += v;
  }
  return s;
}

double pderiv(const Poly& p, int nv, const double* z, int var) {
  double s = 0.0;
  for (int t = 0; t < p.nterms(); ++t) {
    const int e = p.expo[(size_t)t * nv + var];
    if (e == 0) continue;
    double v = p.coef[t] * e;
    for (int i = 0; i < nv; ++i) v *= ipow(z[i], p.expo[(size_t)t * nv + i] - (i == var ? 1 : 0));
    s += v;
  }
  return s;
}

// least-squares step: minimise ||J d + F|| via normal equations with a
// small ridge, Gaussian elimination with partial pivoting
std::vector<double> ls_step(const std::vector<double>& J, const std::vector<double>& F, int rows, int cols) {
  std::vector<double> M((size_t)cols * cols, 0.0), rhs(cols, 0.0);
  for (int a = 0; a < cols; ++a) {
    for (int b = 0; b < cols; ++b) {
      double s = 0.0;
      for (int r = 0; r < rows; ++r) s += J[(size_t)r * cols + a] * J[(size_t)r * cols + b];
      M[(size_t)a * cols + b] = s;
    }
    double s = 0.0;
    for (int r = 0; r < rows; ++r) s -= J[(size_t)r * cols + a] * F[r];
    rhs[a] = s;
  }
  double scale = 0.0;
  for (int a = 0; a < cols; ++a) scale = std::max(scale, M[(size_t)a * cols + a]);
  for (int a = 0; a < cols; ++a) M[(size_t)a * cols + a] += 1e-14 * std::max(scale, 1e-300);
  for (int c = 0; c < cols; ++c) {
    int piv = c;
    for (int r = c + 1; r < cols; ++r)
      if (std::fabs(M[(size_t)r * cols + c]) > std::fabs(M[(size_t)piv * cols + c])) piv = r;
    if (M[(size_t)piv * cols + c] == 0.0) continue;
    if (piv != c) {
      for (int k = 0; k < cols; ++k) std::swap(M[(size_t)c * cols + k], M[(size_t)piv * cols + k]);
      std::swap(rhs[c], rhs[piv]);
    }
    for (int r = c + 1; r < cols; ++r) {
      const double f = M[(size_t)r * cols + c] / M[(size_t)c * cols + c];
      for (int k = c; k < cols; ++k) M[(size_t)r * cols + k] -= f * M[(size_t)c * cols + k];
      rhs[r] -= f * rhs[c];
    }
  }
  std::vector<double> d(cols, 0.0);
  for (int c = cols - 1; c >= 0; --c) {
    double s = rhs[c];
    for (int k = c + 1; k < cols; ++k) s -= M[(size_t)c * cols + k] * d[k];
    d[c] = (M[(size_t)c * cols + c] != 0.0) ? s / M[(size_t)c * cols + c] : 0.0;
  }
  return d;
}

double s_count(int n, int d) {
  double r = 1.0;
  for (int i = 1; i <= d; ++i) r = r * (n + i) / i;
  return r;
}

}  // namespace

std::vector<double> rollout(const Problem& p, const std::vector<double>& zbar) {
  const int dx = p.dx, du = p.du, nv = p.nv();
  std::vector<double> z = zbar;
  for (int k = 0; k < p.N; ++k) {
    const int s0 = k * (dx + du);
    for (int i = 0; i < du; ++i) z[s0 + dx + i] = std::min(p.R, std::max(-p.R, z[s0 + dx + i]));
    std::vector<int> unk;
    if (k == 0)
      for (int i = 0; i < dx; ++i) unk.push_back(i);
    for (int i = dx + du; i < nv; ++i) unk.push_back(i);
    const auto& hs = p.cl[k].h;
    const int rows = (int)hs.size(), cols = (int)unk.size();
    if (rows == 0) continue;
    std::vector<double> zk(z.begin() + s0, z.begin() + s0 + nv);
    for (int itn = 0; itn < 60; ++itn) {
      std::vector<double> F(rows), J((size_t)rows * cols);
      double fmax = 0.0;
      for (int r = 0; r < rows; ++r) {
        F[r] = peval(hs[r], nv, zk.data());
        fmax = std::max(fmax, std::fabs(F[r]));
        for (int c = 0; c < cols; ++c) J[(size_t)r * cols + c] = pderiv(hs[r], nv, zk.data(), unk[c]);
      }
      if (fmax < 1e-14) break;
      auto d = ls_step(J, F, rows, cols);
      for (int c = 0; c < cols; ++c) zk[unk[c]] += d[c];
    }
    for (int i = 0; i < nv; ++i) z[s0 + i] = zk[i];
  }
  return z;
}

// certificate of one instance from the eigen data of its blocks
// (lamX/topX: eigenvalues ascending and top eigenvector of X's blocks,
// lamZ: eigenvalues of Z = C - A^T y; lo[b]: offset of block b in them)
void certify_one(const Problem& p, const std::vector<int32_t>& bn, const std::vector<int8_t>& bk,
                 const std::vector<int32_t>& bc, const int64_t* lo, const double* lamX, const double* topX,
                 const double* lamZ, double by, double rank_tol, double xi_tol, strom_certificate* out,
                 double* zbar_out, double* zhat_out) {
  const int nv = p.nv(), dx = p.dx, du = p.du;
  std::vector<double> zbar(p.nz(), 0.0);
  double max_ratio = 0.0;
  for (size_t b = 0; b < bn.size(); ++b) {
    if (bk[b] != 0) continue;
    const int n = bn[b];
    const double l1 = lamX[lo[b] + n - 1], l2 = lamX[lo[b] + n - 2];
    const double ratio = l1 > 0 ? l2 / l1 : INFINITY;
    max_ratio = std::max(max_ratio, ratio);
    const double v0 = topX[lo[b]];
    const int k = bc[b];
    const int s0 = k * (dx + du);
    for (int t = 0; t < dx + du; ++t) zbar[s0 + t] = topX[lo[b] + 1 + t] / v0;
    if (k == p.N - 1)
      for (int t = dx + du; t < nv; ++t) zbar[s0 + t] = topX[lo[b] + 1 + t] / v0;
  }
  std::vector<double> zhat = rollout(p, zbar);
  double hmax = 0.0, gmin = INFINITY, phat = 0.0;
  for (int k = 0; k < p.N; ++k) {
    const double* zk = zhat.data() + k * (dx + du);
    for (auto& h : p.cl[k].h) hmax = std::max(hmax, std::fabs(peval(h, nv, zk)));
    for (auto& g : p.cl[k].g) gmin = std::min(gmin, peval(g, nv, zk));
    phat += peval(p.cl[k].f, nv, zk);
  }
  const double feas_tol = 1e-9;
  const bool feasible = hmax <= feas_tol && gmin >= -feas_tol;
  const double R = std::max(1.0, p.R);
  const int kappa = p.kappa;
  double lb = by;
  std::vector<int> gi(p.N, 0);
  for (size_t b = 0; b < bn.size(); ++b) {
    const double lmin = lamZ[lo[b]];
    double Rb;
    const int k = bc[b];
    if (bk[b] == 0) {
      Rb = s_count(nv, kappa) * std::pow(R, 2 * kappa);
    } else {
      const Poly& g = p.cl[k].g[gi[k]++];
      const int dg = (g.degree(nv) + 1) / 2;
      double gmax = 0.0;
      for (int t = 0; t < g.nterms(); ++t) {
        int deg = 0;
        for (int v = 0; v < nv; ++v) deg += g.expo[(size_t)t * nv + v];
        gmax += std::fabs(g.coef[t]) * std::pow(R, deg);
      }
      Rb = gmax * s_count(nv, kappa - dg) * std::pow(R, 2 * (kappa - dg));
    }
    lb += Rb * std::min(0.0, lmin);
  }
  out->max_ratio = max_ratio;
  out->lower_bound = lb;
  out->phat = phat;
  out->xi = (phat - lb) / (1.0 + std::fabs(phat) + std::fabs(lb));
  out->hmax = hmax;
  out->gmin = gmin;
  out->feasible = feasible;
  out->rank_one = max_ratio <= rank_tol;
  out->certified = out->rank_one && feasible && out->xi <= xi_tol;
  if (zbar_out) std::copy(zbar.begin(), zbar.end(), zbar_out);
  if (zhat_out) std::copy(zhat.begin(), zhat.end(), zhat_out);
}

}  // namespace strom

using namespace strom;

extern "C" int strom_certify(strom_solver* s, int32_t i, const strom_problem* prob, double rank_tol, double xi_tol,
                             strom_certificate* out, double* zbar_out, double* zhat_out) {
  try {
    if (!s || !prob || !out) {
      set_error("strom_certify: bad arguments");
      return STROM_ERR_INVALID;
    }
    const Problem& p = prob->p;
    std::vector<int32_t> bn, bc;
    std::vector<int8_t> bk;
    std::vector<int64_t> lo;
    double by = 0.0;
    const int N = solver_blocks_of(s, i, bn, bk, bc, lo, &by);
    if (N != p.N || (int)bn.size() == 0) {
      set_error("strom_certify: problem does not match the solver instance");
      return STROM_ERR_INVALID;
    }
    std::vector<double> lamX, topX, lamZ, topZ;
    solver_eig_blocks(s, i, false, lamX, topX);
    solver_eig_blocks(s, i, true, lamZ, topZ);
    certify_one(p, bn, bk, bc, lo.data(), lamX.data(), topX.data(), lamZ.data(), by, rank_tol, xi_tol, out, zbar_out,
                zhat_out);
    return STROM_OK;
  } catch (const std::exception& e) {
    set_error(std::string("strom_certify: ") + e.what());
    return STROM_ERR_CUDA;
  }
}

extern "C" int strom_certify_host(const strom_problem* prob, int32_t nblocks, const int32_t* block_n,
                                  const int8_t* block_kind, const int32_t* block_clique, const double* lamX,
                                  const double* topX, const double* lamZ, double by, double rank_tol, double xi_tol,
                                  strom_certificate* out, double* zbar_out, double* zhat_out) {
  try {
    if (!prob || !out || nblocks < 1 || !block_n || !block_kind || !block_clique || !lamX || !topX || !lamZ)
      throw std::invalid_argument("bad arguments");
    const Problem& p = prob->p;
    const int nv = p.nv();
    const int nmom = (nv + 1) * (nv + 2) / 2;
    std::vector<int> n_mom(p.N, 0), n_loc(p.N, 0);
    std::vector<int64_t> lo(nblocks);
    int64_t acc = 0;
    for (int b = 0; b < nblocks; ++b) {
      const int k = block_clique[b];
      if (k < 0 || k >= p.N || block_n[b] < 1) throw std::invalid_argument("block clique or size out of range");
      if (block_kind[b] == 0) {
        if (block_n[b] != nmom) throw std::invalid_argument("moment block of the wrong size");
        ++n_mom[k];
      } else if (block_kind[b] == 1) {
        ++n_loc[k];
      } else {
        throw std::invalid_argument("block kind must be 0 (moment) or 1 (localizing)");
      }
      lo[b] = acc;
      acc += block_n[b];
    }
    for (int k = 0; k < p.N; ++k)
      if (n_mom[k] != 1 || n_loc[k] != (int)p.cl[k].g.size())
        throw std::invalid_argument("blocks do not match the problem's cliques");
    std::vector<int32_t> bn(block_n, block_n + nblocks), bc(block_clique, block_clique + nblocks);
    std::vector<int8_t> bk(block_kind, block_kind + nblocks);
    certify_one(p, bn, bk, bc, lo.data(), lamX, topX, lamZ, by, rank_tol, xi_tol, out, zbar_out, zhat_out);
    return STROM_OK;
  } catch (const std::exception& e) {
    set_error(std::string("strom_certify_host: ") + e.what());
    return STROM_ERR_INVALID;
  }
}

extern "C" int strom_certify_batch(strom_solver* s, const strom_problem* const* problems, double rank_tol,
                                   double xi_tol, strom_certificate* out) {
  try {
    if (!s || !problems || !out) {
      set_error("strom_certify_batch: bad arguments");
      return STROM_ERR_INVALID;
    }
    const int count = strom_solver_count(s);
    for (int i = 0; i < count; ++i)
      if (!problems[i]) {
        set_error("strom_certify_batch: null problem");
        return STROM_ERR_INVALID;
      }
    std::vector<double> lamX, topX, lamZ, topZ, stats;
    std::vector<int64_t> lo;
    solver_eig_all(s, false, lamX, topX, lo, stats);
    solver_eig_all(s, true, lamZ, topZ, lo, stats);
    for (int i = 0; i < count; ++i) {
      const Problem& p = problems[i]->p;
      std::vector<int32_t> bn, bc;
      std::vector<int8_t> bk;
      int64_t b0 = 0;
      const int N = solver_inst_blocks(s, i, bn, bk, bc, &b0);
      if (N != p.N) {
        set_error("strom_certify_batch: problem does not match the solver instance");
        return STROM_ERR_INVALID;
      }
      certify_one(p, bn, bk, bc, lo.data() + b0, lamX.data(), topX.data(), lamZ.data(), stats[8 * (size_t)i + 4],
                  rank_tol, xi_tol, &out[i], nullptr, nullptr);
    }
    return STROM_OK;
  } catch (const std::exception& e) {
    set_error(std::string("strom_certify_batch: ") + e.what());
    return STROM_ERR_CUDA;
  }
}
