// Rank tests of one moment matrix (host): the flat-extension condition that
// generalises the rank-1 test of Theorem 1 (iii) (Sec. 2.2), and the
// partial rank-1 test on the monomials of a subset of the clique variables
// (the paper's car back-in: auxiliary variables make M_k rank > 1 while the
// submatrix of the trajectory variables stays rank 1).
#include <algorithm>
#include <cmath>
#include <limits>
#include <numeric>
#include <string>
#include <vector>

#include "internal.h"

namespace {

// Symmetric eigendecomposition by the cyclic-by-row Jacobi method with the
// stable 2x2 symmetric Schur rotation (Golub & Van Loan, Matrix
// Computations, Sec. 8.5). A: n x n row-major, destroyed. On return w holds
// the eigenvalues ascending and column j of V (row-major n x n) the
// eigenvector of w[j].
void sym_eig(std::vector<double>& A, int n, std::vector<double>& w, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  double fro = 0.0;
  for (double a : A) fro += a * a;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += 2.0 * A[(size_t)p * n + q] * A[(size_t)p * n + q];
    if (off <= 1e-30 * fro) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double tau = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        // A <- J^T A J with J the rotation in the (p, q) plane
        for (int k = 0; k < n; ++k) {
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  std::vector<int> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return A[(size_t)a * n + a] < A[(size_t)b * n + b]; });
  std::vector<double> V2((size_t)n * n);
  w.resize(n);
  for (int j = 0; j < n; ++j) {
    w[j] = A[(size_t)ord[j] * n + ord[j]];
    for (int i = 0; i < n; ++i) V2[(size_t)i * n + j] = V[(size_t)i * n + ord[j]];
  }
  V.swap(V2);
}

int numerical_rank(const std::vector<double>& w, double tol) {
  const double top = w.empty() ? 0.0 : std::max(w.back(), 0.0);
  if (!(top > 0.0)) return 0;
  int r = 0;
  for (double x : w) r += x > tol * top;
  return r;
}

std::vector<double> principal(const double* M, int n, const std::vector<int>& idx) {
  const int m = (int)idx.size();
  std::vector<double> S((size_t)m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) S[(size_t)i * m + j] = M[(size_t)idx[j] * n + idx[i]];  // column-major input
  return S;
}

}  // namespace

extern "C" int strom_moment_rank_test(const double* M, int32_t nv, const uint8_t* vars, double tol,
                                      strom_rank_test* out, double* zbar) {
  if (!M || !out || nv < 1 || nv > 21 || !(tol > 0.0) || !std::isfinite(tol)) {
    strom::set_error("strom_moment_rank_test: bad arguments");
    return STROM_ERR_INVALID;
  }
  try {
    const auto basis = strom::monomial_basis(nv, 2);
    const int n = (int)basis.size();
    double amax = 0.0;
    for (int64_t e = 0; e < (int64_t)n * n; ++e) {
      if (!std::isfinite(M[e])) {
        strom::set_error("strom_moment_rank_test: non-finite entry");
        return STROM_ERR_INVALID;
      }
      amax = std::max(amax, std::fabs(M[e]));
    }
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j)
        if (std::fabs(M[(size_t)j * n + i] - M[(size_t)i * n + j]) > 1e-12 * amax) {
          strom::set_error("strom_moment_rank_test: M is not symmetric");
          return STROM_ERR_INVALID;
        }
    std::vector<int> all(n), low, sub;
    std::iota(all.begin(), all.end(), 0);
    for (int i = 0; i < n; ++i) {
      int deg = 0;
      bool inside = true;
      for (int t = 0; t < nv; ++t) {
        deg += basis[i][t];
        if (basis[i][t] && vars && !vars[t]) inside = false;
      }
      if (deg <= 1) low.push_back(i);
      if (inside) sub.push_back(i);
    }
    std::vector<double> w, V;
    auto A = principal(M, n, all);
    sym_eig(A, n, w, V);
    out->n = n;
    out->rank = numerical_rank(w, tol);
    out->lambda_max = w.back();
    auto L = principal(M, n, low);
    std::vector<double> wl, Vl;
    sym_eig(L, (int)low.size(), wl, Vl);
    out->rank_low = numerical_rank(wl, tol);
    out->flat = out->rank == out->rank_low;
    const int ns = (int)sub.size();
    auto B = principal(M, n, sub);
    std::vector<double> ws, Vs;
    sym_eig(B, ns, ws, Vs);
    out->n_sub = ns;
    const double top = ws.back();
    out->ratio_sub = top > 0.0 ? (ns > 1 ? ws[ns - 2] / top : 0.0) : std::numeric_limits<double>::infinity();
    if (zbar) {
      for (int t = 0; t < nv; ++t) zbar[t] = std::numeric_limits<double>::quiet_NaN();
      const double lead = Vs[(size_t)0 * ns + (ns - 1)];  // the constant monomial is sub[0]
      for (int j = 0; j < ns; ++j) {
        const auto& e = basis[sub[j]];
        int deg = 0, var = -1;
        for (int t = 0; t < nv; ++t)
          if (e[t]) { deg += e[t]; var = t; }
        if (deg == 1) zbar[var] = Vs[(size_t)j * ns + (ns - 1)] / lead;
      }
    }
    return STROM_OK;
  } catch (const std::exception& e) {
    strom::set_error(std::string("strom_moment_rank_test: ") + e.what());
    return STROM_ERR_INVALID;
  }
}
