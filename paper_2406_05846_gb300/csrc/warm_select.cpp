// Neighbour selection for data-driven warm starts (Sec. 5, inverted pendulum
// with kNN warm starts): the d + 1 stored keys nearest to a query span a
// simplex; inside it the query's barycentric coordinates weight the stored
// states, elsewhere the weights fall back to inverse distances.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "internal.h"

namespace {

// Solves M x = r (d x d, column-major) by Gaussian elimination with partial
// pivoting. Returns false when a pivot falls below tol.
bool solve_small(std::vector<double> M, std::vector<double> r, int d, double tol, std::vector<double>& x) {
  for (int c = 0; c < d; ++c) {
    int p = c;
    for (int i = c + 1; i < d; ++i)
      if (std::fabs(M[c * d + i]) > std::fabs(M[c * d + p])) p = i;
    if (!(std::fabs(M[c * d + p]) > tol)) return false;
    if (p != c) {
      for (int j = 0; j < d; ++j) std::swap(M[j * d + c], M[j * d + p]);
      std::swap(r[c], r[p]);
    }
    for (int i = c + 1; i < d; ++i) {
      const double f = M[c * d + i] / M[c * d + c];
      for (int j = c; j < d; ++j) M[j * d + i] -= f * M[j * d + c];
      r[i] -= f * r[c];
    }
  }
  x.assign(d, 0.0);
  for (int c = d - 1; c >= 0; --c) {
    double acc = r[c];
    for (int j = c + 1; j < d; ++j) acc -= M[j * d + c] * x[j];
    x[c] = acc / M[c * d + c];
  }
  return true;
}

}  // namespace

namespace strom {

int warm_select(const double* keys, int n, int d, const double* key, int32_t* idx, double* wt) {
  if (n <= 0) return 0;
  std::vector<double> d2(n);
  for (int j = 0; j < n; ++j) {
    double acc = 0.0;
    for (int t = 0; t < d; ++t) {
      const double e = key[t] - keys[(int64_t)j * d + t];
      acc += e * e;
    }
    d2[j] = acc;
  }
  const int K = std::min(d + 1, n);
  std::vector<int> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  std::partial_sort(ord.begin(), ord.begin() + K, ord.end(),
                    [&](int a, int b) { return d2[a] < d2[b] || (d2[a] == d2[b] && a < b); });
  for (int j = 0; j < K; ++j) idx[j] = ord[j];
  if (d2[ord[0]] == 0.0) {
    wt[0] = 1.0;
    return 1;
  }
  if (K == d + 1) {
    // key = k_0 + sum_c lambda_c (k_c - k_0): barycentric coordinates
    std::vector<double> M((size_t)d * d), r(d), lam;
    double scale = 0.0;
    for (int c = 0; c < d; ++c)
      for (int t = 0; t < d; ++t) {
        M[(size_t)c * d + t] = keys[(int64_t)ord[c + 1] * d + t] - keys[(int64_t)ord[0] * d + t];
        scale = std::max(scale, std::fabs(M[(size_t)c * d + t]));
      }
    for (int t = 0; t < d; ++t) r[t] = key[t] - keys[(int64_t)ord[0] * d + t];
    if (solve_small(M, r, d, 1e-12 * scale, lam)) {
      double l0 = 1.0;
      for (double l : lam) l0 -= l;
      bool inside = l0 >= -1e-12;
      for (double l : lam) inside = inside && l >= -1e-12;
      if (inside) {
        wt[0] = std::max(0.0, l0);
        for (int c = 0; c < d; ++c) wt[c + 1] = std::max(0.0, lam[c]);
        double s = 0.0;
        for (int j = 0; j < K; ++j) s += wt[j];
        for (int j = 0; j < K; ++j) wt[j] /= s;
        return K;
      }
    }
  }
  double s = 0.0;
  for (int j = 0; j < K; ++j) {
    wt[j] = 1.0 / std::sqrt(d2[ord[j]]);
    s += wt[j];
  }
  for (int j = 0; j < K; ++j) wt[j] /= s;
  return K;
}

}  // namespace strom

extern "C" int strom_warm_select(const double* keys, int32_t n, int32_t key_dim, const double* key, int32_t* idx,
                                 double* wt, int32_t* k) {
  if (n < 0 || key_dim < 1 || key_dim > STROM_WARM_MAX_KEY || (n > 0 && !keys) || !key || !idx || !wt || !k) {
    strom::set_error("strom_warm_select: bad arguments");
    return STROM_ERR_INVALID;
  }
  for (int64_t e = 0; e < (int64_t)n * key_dim; ++e)
    if (!std::isfinite(keys[e])) {
      strom::set_error("strom_warm_select: non-finite stored key");
      return STROM_ERR_INVALID;
    }
  for (int t = 0; t < key_dim; ++t)
    if (!std::isfinite(key[t])) {
      strom::set_error("strom_warm_select: non-finite key");
      return STROM_ERR_INVALID;
    }
  *k = strom::warm_select(keys, n, key_dim, key, idx, wt);
  return STROM_OK;
}
