// Device/host helpers shared by the CUDA translation units of libstrom.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <stdexcept>
#include <string>

#include "internal.h"

#define STROM_CUDA(call)                                                                   \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      throw strom::CudaError(std::string(#call) + ": " + cudaGetErrorString(e_));          \
  } while (0)

namespace strom {

struct CudaError : std::runtime_error {
  using std::runtime_error::runtime_error;
};
struct StatusError : std::runtime_error {
  int status;
  StatusError(int s, const std::string& m) : std::runtime_error(m), status(s) {}
};

// Device bytes allocated through DevBuf by the calling host thread while a
// tally is attached (strom_batch_slot_bytes measures a solver's footprint
// with it): live bytes and their peak.
struct AllocTally {
  int64_t live = 0, peak = 0;
};
inline thread_local AllocTally* g_alloc_tally = nullptr;

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) {
      cudaFree(p);
      if (g_alloc_tally) g_alloc_tally->live -= (int64_t)(n * sizeof(T));
    }
    p = nullptr;
    n = 0;
  }
  void alloc(size_t count) {
    release();
    if (count == 0) return;
    cudaError_t e = cudaMalloc((void**)&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      throw StatusError(STROM_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    n = count;
    if (g_alloc_tally) {
      g_alloc_tally->live += (int64_t)(count * sizeof(T));
      if (g_alloc_tally->live > g_alloc_tally->peak) g_alloc_tally->peak = g_alloc_tally->live;
    }
  }
  void upload(const T* h, size_t count, cudaStream_t st = 0) {
    alloc(count);
    if (count) STROM_CUDA(cudaMemcpyAsync(p, h, count * sizeof(T), cudaMemcpyHostToDevice, st));
    count_h2d(count * sizeof(T));
  }
  void zero(cudaStream_t st = 0) {
    if (n) STROM_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), st));
  }
};

// NVTX range over a host-side phase (set-up, factorisation, iterations,
// certificate, admission, retirement), visible to a profiler's timeline;
// without a profiler attached it costs a null check
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// host <-> device copies that are counted by strom_transfer_bytes()
inline void copy_h2d(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (!bytes) return;
  STROM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
  count_h2d(bytes);
}
inline void copy_d2h(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (!bytes) return;
  STROM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st));
  count_d2h(bytes);
}

// ---------------------------------------------------------------------------
// PSD projection launcher (psd.cu)
// ---------------------------------------------------------------------------
struct PsdClasses {
  // block ids grouped by size class; classes: n <= 16, <= 40, <= 80, <= 160
  int count[4] = {0, 0, 0, 0};
  int start[4] = {0, 0, 0, 0};
  int max_n[4] = {0, 0, 0, 0};
  // threads per CTA of each class's launch, [0] FP64 / [1] FP32; 0 = the
  // default shape (psd_threads_candidates lists the others)
  int threads[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
};

// launch shapes (threads per CTA) of size class k in one precision; the first
// is the default. Returns how many (at most 3).
int psd_threads_candidates(int precision, int k, int* out);
// a deterministic symmetric test input (svec entries in [-1, 1] from a hash
// of the index), for timing the eigensolver's launch shapes
void psd_fill_test_input(double* x, int64_t n, cudaStream_t st);

// doubles of global scratch per FP64 block of the n <= 160 class (V^T, 160 x 162)
constexpr size_t kVScratchPerBlock = 160 * 162;

struct PsdArgs {
  const double* Xb;            // svec input
  double* out;                 // svec output
  const int64_t* blk_off;      // [nblk]
  const int32_t* blk_n;        // [nblk]
  const int32_t* blk_list;     // block ids sorted by class
  const double* blk_inv_sigma; // [nblk] or null: out = (Pi(Xb) - Xb) * inv_sigma
  const uint8_t* blk_active;   // [nblk] or null: skip inactive blocks
  double* lam;                 // optional eigenvalues (ascending) at lam_off[b]
  const int64_t* lam_off;
  double* topvec;              // optional eigenvector of the largest eigenvalue at lam_off[b]
  double* vscratch;            // FP64 V storage for the n <= 160 class: [count * 160 * 160]
  // warm start of the FP32 eigensolver across ADMM iterations (nullable):
  // the eigenvectors of block b are kept in vstore + vstore_off[b]; a block
  // whose instance is at an iteration not divisible by warm_period starts its
  // sweeps from B = V X_b V^T with those eigenvectors instead of from X_b
  float* vstore;
  const int64_t* vstore_off;
  const int32_t* blk_inst;
  const int32_t* inst_iter;
  int warm_period;
  int reorth;   // 1: re-orthonormalise the stored FP32 eigenvectors of blocks of 41..80 rows (warm starts)
  // the same for the FP64 eigensolver (the polish): eigenvectors in vstore64,
  // inst_iter64 counts an instance's consecutive FP64 iterations
  double* vstore64;
  const int32_t* inst_iter64;
};

// precision: STROM_PREC_FP64 or STROM_PREC_FP32
void psd_launch(const PsdArgs& a, const PsdClasses& c, int precision, cudaStream_t st);
void psd_configure();  // one-time function attributes (large shared memory)

}  // namespace strom
