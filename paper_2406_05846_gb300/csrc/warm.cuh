// Store of solved states for data-driven warm starts (warm.cu), shared with
// the serving loop (serve.cu).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"

struct strom_warm {
  int d = 0;                 // key dimension
  int64_t nsvec = 0;         // svec length of every stored state
  int cap = 0, n = 0;        // capacity, entries stored
  int device = 0;
  std::vector<double> keys;  // [n * d]
  std::vector<double> sigma; // [n]
  strom::DevBuf<double> XS;  // [cap][2][nsvec]: X then S of each entry
};

namespace strom {
// Writes the warm start for key into X_dev, S_dev (nsvec each) on stream st
// and returns its sigma; returns false (nothing written) when the store is
// empty.
bool warm_apply(const strom_warm* w, const double* key, double* X_dev, double* S_dev, double* sigma,
                cudaStream_t st);
// Appends (key, X_dev, S_dev, sigma) by device-to-device copies; returns the
// index, or -1 when the store is full.
int warm_append(strom_warm* w, const double* key, const double* X_dev, const double* S_dev, double sigma,
                cudaStream_t st);
}  // namespace strom
