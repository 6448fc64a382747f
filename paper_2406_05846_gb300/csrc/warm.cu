// Data-driven warm starts (Sec. 5, inverted pendulum with kNN warm starts):
// a device-resident store of solved states (X, S, sigma) keyed by instance
// parameters, and the convex combination of the neighbours of a new key as
// the starting point of Algorithm 1.
#include <cuda_runtime.h>

#include <cmath>
#include <memory>

#include "solver_impl.cuh"
#include "warm.cuh"

namespace {

constexpr int kMaxNb = STROM_WARM_MAX_KEY + 1;

struct Combo {
  int k;
  double w[kMaxNb];
  const double* src[kMaxNb];  // X of each neighbour; its S follows after nsvec entries
};

// X[e] = sum_j w_j X_j[e], S[e] = sum_j w_j S_j[e], j in neighbour order.
// Streams (k + 1) x 2 x nsvec doubles; grid-stride over the svec entries.
__global__ void __launch_bounds__(256) warm_combine_kernel(Combo c, int64_t nsvec, double* __restrict__ X,
                                                           double* __restrict__ S) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nsvec; e += (int64_t)gridDim.x * blockDim.x) {
    double x = 0.0, s = 0.0;
    for (int j = 0; j < c.k; ++j) {
      x = fma(c.w[j], __ldg(c.src[j] + e), x);
      s = fma(c.w[j], __ldg(c.src[j] + nsvec + e), s);
    }
    X[e] = x;
    S[e] = s;
  }
}

template <typename F>
int guard(F&& f) {
  try {
    return f();
  } catch (const StatusError& e) {
    set_error(e.what());
    return e.status;
  } catch (const CudaError& e) {
    set_error(e.what());
    return STROM_ERR_CUDA;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return STROM_ERR_OOM;
  } catch (const std::exception& e) {
    set_error(e.what());
    return STROM_ERR_INVALID;
  }
}

void check_key(const strom_warm* w, const double* key, const char* who) {
  if (!key) throw StatusError(STROM_ERR_INVALID, std::string(who) + ": null key");
  for (int t = 0; t < w->d; ++t)
    if (!std::isfinite(key[t])) throw StatusError(STROM_ERR_INVALID, std::string(who) + ": non-finite key");
}

int grid_for(int64_t n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  const int64_t want = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, 8LL * sms));
}

}  // namespace

bool strom::warm_apply(const strom_warm* w, const double* key, double* X_dev, double* S_dev, double* sigma,
                       cudaStream_t st) {
  int32_t idx[kMaxNb];
  double wt[kMaxNb];
  const int k = warm_select(w->keys.data(), w->n, w->d, key, idx, wt);
  if (k == 0) return false;
  Combo c{};
  c.k = k;
  double lsg = 0.0;
  for (int j = 0; j < k; ++j) {
    c.w[j] = wt[j];
    c.src[j] = w->XS.p + (int64_t)idx[j] * 2 * w->nsvec;
    lsg += wt[j] * std::log(w->sigma[idx[j]]);
  }
  warm_combine_kernel<<<grid_for(w->nsvec), 256, 0, st>>>(c, w->nsvec, X_dev, S_dev);
  STROM_CUDA(cudaGetLastError());
  count_launches(1);
  *sigma = std::exp(lsg);
  return true;
}

int strom::warm_append(strom_warm* w, const double* key, const double* X_dev, const double* S_dev, double sigma,
                       cudaStream_t st) {
  if (w->n >= w->cap) return -1;
  double* dst = w->XS.p + (int64_t)w->n * 2 * w->nsvec;
  STROM_CUDA(cudaMemcpyAsync(dst, X_dev, sizeof(double) * w->nsvec, cudaMemcpyDeviceToDevice, st));
  STROM_CUDA(cudaMemcpyAsync(dst + w->nsvec, S_dev, sizeof(double) * w->nsvec, cudaMemcpyDeviceToDevice, st));
  // the entry is complete before any other stream (strom_warm_get, another
  // solver's warm start) can read it
  STROM_CUDA(cudaStreamSynchronize(st));
  w->keys.insert(w->keys.end(), key, key + w->d);
  w->sigma.push_back(sigma);
  return w->n++;
}

extern "C" int strom_warm_create(int32_t key_dim, int64_t nsvec, int32_t capacity, strom_warm** out) {
  return guard([&]() -> int {
    if (!out || key_dim < 1 || key_dim > STROM_WARM_MAX_KEY || nsvec < 1 || capacity < 1)
      throw StatusError(STROM_ERR_INVALID, "strom_warm_create: bad arguments");
    std::unique_ptr<strom_warm> w(new strom_warm());
    w->d = key_dim;
    w->nsvec = nsvec;
    w->cap = capacity;
    STROM_CUDA(cudaGetDevice(&w->device));
    w->XS.alloc((size_t)capacity * 2 * nsvec);
    w->keys.reserve((size_t)capacity * key_dim);
    *out = w.release();
    return STROM_OK;
  });
}

extern "C" void strom_warm_destroy(strom_warm* w) { delete w; }

extern "C" int32_t strom_warm_count(const strom_warm* w) { return w ? w->n : -1; }

extern "C" int strom_warm_add(strom_warm* w, const double* key, const double* X, const double* S, double sigma,
                              int32_t* index) {
  return guard([&]() -> int {
    if (!w || !X || !S || !(sigma > 0) || !std::isfinite(sigma))
      throw StatusError(STROM_ERR_INVALID, "strom_warm_add: bad arguments");
    check_key(w, key, "strom_warm_add");
    if (w->n >= w->cap) throw StatusError(STROM_ERR_INVALID, "strom_warm_add: the store is full");
    double* dst = w->XS.p + (int64_t)w->n * 2 * w->nsvec;
    copy_h2d(dst, X, sizeof(double) * w->nsvec, 0);
    copy_h2d(dst + w->nsvec, S, sizeof(double) * w->nsvec, 0);
    STROM_CUDA(cudaStreamSynchronize(0));
    w->keys.insert(w->keys.end(), key, key + w->d);
    w->sigma.push_back(sigma);
    if (index) *index = w->n;
    w->n++;
    return STROM_OK;
  });
}

extern "C" int strom_warm_add_from_solver(strom_warm* w, const strom_solver* s, int32_t i, const double* key,
                                          int32_t* index) {
  return guard([&]() -> int {
    if (!w || !s || i < 0 || i >= s->ninst) throw StatusError(STROM_ERR_INVALID, "strom_warm_add_from_solver: bad arguments");
    check_key(w, key, "strom_warm_add_from_solver");
    const int64_t so = s->svec_off[i], n = s->svec_off[i + 1] - so;
    if (n != w->nsvec) throw StatusError(STROM_ERR_INVALID, "strom_warm_add_from_solver: svec length differs from the store's");
    if (w->n >= w->cap) throw StatusError(STROM_ERR_INVALID, "strom_warm_add_from_solver: the store is full");
    double sg = 0.0;
    copy_d2h(&sg, s->sigma.p + i, sizeof(double), s->stream);
    STROM_CUDA(cudaStreamSynchronize(s->stream));
    const int at = warm_append(w, key, s->X.p + so, s->S.p + so, sg, s->stream);
    STROM_CUDA(cudaStreamSynchronize(s->stream));
    if (index) *index = at;
    return STROM_OK;
  });
}

extern "C" int strom_warm_query(const strom_warm* w, const double* key, int32_t* idx, double* wt, int32_t* k) {
  return guard([&]() -> int {
    if (!w || !idx || !wt || !k) throw StatusError(STROM_ERR_INVALID, "strom_warm_query: bad arguments");
    check_key(w, key, "strom_warm_query");
    *k = warm_select(w->keys.data(), w->n, w->d, key, idx, wt);
    return STROM_OK;
  });
}

extern "C" int strom_warm_get(const strom_warm* w, int32_t j, double* key, double* X, double* S, double* sigma) {
  return guard([&]() -> int {
    if (!w || j < 0 || j >= w->n) throw StatusError(STROM_ERR_INVALID, "strom_warm_get: bad entry");
    const double* src = w->XS.p + (int64_t)j * 2 * w->nsvec;
    if (X) copy_d2h(X, src, sizeof(double) * w->nsvec, 0);
    if (S) copy_d2h(S, src + w->nsvec, sizeof(double) * w->nsvec, 0);
    STROM_CUDA(cudaStreamSynchronize(0));
    if (key) for (int t = 0; t < w->d; ++t) key[t] = w->keys[(size_t)j * w->d + t];
    if (sigma) *sigma = w->sigma[j];
    return STROM_OK;
  });
}

extern "C" int strom_solver_warm_start(strom_solver* s, int32_t i, const strom_warm* w, const double* key) {
  return guard([&]() -> int {
    if (!s || !w || i < 0 || i >= s->ninst) throw StatusError(STROM_ERR_INVALID, "strom_solver_warm_start: bad arguments");
    check_key(w, key, "strom_solver_warm_start");
    const int64_t so = s->svec_off[i], n = s->svec_off[i + 1] - so;
    if (n != w->nsvec) throw StatusError(STROM_ERR_INVALID, "strom_solver_warm_start: svec length differs from the store's");
    reset_instances(s, {i});
    double sg = 0.0;
    if (warm_apply(w, key, s->X.p + so, s->S.p + so, &sg, s->stream)) {
      copy_h2d(s->sigma.p + i, &sg, sizeof(double), s->stream);
      STROM_CUDA(cudaStreamSynchronize(s->stream));
    }
    return STROM_OK;
  });
}
