// PSD projection for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside another
// framework's memory pool that forbids foreign allocations, real-time loops
// that must not allocate after start-up, or processes whose device memory is
// fully reserved up front. strom_kernel_psd_project_noalloc gives them the
// PSD projection with no device (or host heap) allocation: the block table
// and the FP64 eigenvector scratch live in one file-scope static __device__
// array, g_noalloc, which every GPU that loads the library holds until the
// process exits (about 4.37 MB).
//
// Host code never names g_noalloc as if it were a device address (in host
// code the name is only a host-side stand-in). Its device address is taken
// once per device with cudaGetSymbolAddress, on the first call made with that
// device current, and cached; make that first call before any stream capture.
// Under CUDA's lazy module loading the device code of this file and of the
// projection kernels, and with it g_noalloc itself, is loaded into device
// memory on first use; the set-up therefore also forces the loading of every
// kernel the entry point launches. A call with nblk = 0 does only this
// set-up, so a caller that must not allocate later makes it at start-up.
// Every call reuses the same array, which keeps the previous call's contents:
// calls that overlap on the GPU (different streams, or different host threads
// on one device) race and must be serialised by the caller.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "common.cuh"

namespace strom {
namespace {

constexpr int kNoAllocMaxBlocks = 65536;  // blocks per call
constexpr int kNoAllocMaxVBlocks = 16;    // FP64 blocks with 80 < n <= 160 per launch (more are chunked)
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
  int64_t off[kNoAllocMaxBlocks];
  int32_t n[kNoAllocMaxBlocks];
  int32_t list[kNoAllocMaxBlocks];
  int32_t fill[4];
  int32_t cls[8];  // counts, then starts
  double vs[kNoAllocMaxVBlocks * kVScratchPerBlock];
};

static __device__ __align__(256) NoAllocScratch g_noalloc;

std::mutex g_mu;
NoAllocScratch* g_addr[kMaxDevices] = {};

__device__ __forceinline__ int size_class(int n) { return n <= 16 ? 0 : n <= 40 ? 1 : n <= 80 ? 2 : 3; }

// counting sort of the blocks by size class (order inside a class does not
// matter: every block is projected independently)
__global__ void __launch_bounds__(1024) classify_kernel(NoAllocScratch* sc, int nblk) {
  __shared__ int cnt[4], start[4];
  if (threadIdx.x < 4) cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) atomicAdd(&cnt[size_class(sc->n[i])], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int c = 0; c < 4; ++c) {
      start[c] = acc;
      sc->cls[c] = cnt[c];
      sc->cls[4 + c] = acc;
      sc->fill[c] = 0;
      acc += cnt[c];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
    const int c = size_class(sc->n[i]);
    sc->list[start[c] + atomicAdd(&sc->fill[c], 1)] = i;
  }
}

// set-up of the current device, once: the device address of g_noalloc, the
// projection kernels' attributes, and the loading of classify_kernel (the
// attribute queries load each kernel's module under lazy loading)
NoAllocScratch* scratch_for_current_device() {
  int dev = 0;
  STROM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) throw StatusError(STROM_ERR_INVALID, "device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    STROM_CUDA(cudaGetSymbolAddress(&p, g_noalloc));
    psd_configure();
    cudaFuncAttributes fa;
    STROM_CUDA(cudaFuncGetAttributes(&fa, classify_kernel));
    g_addr[dev] = static_cast<NoAllocScratch*>(p);
  }
  return g_addr[dev];
}

}  // namespace
}  // namespace strom

extern "C" int strom_kernel_psd_project_noalloc(const double* Xb_dev, const int64_t* blk_off, const int32_t* blk_n,
                                                int32_t nblk, int32_t precision, double* P_dev, void* stream) {
  using namespace strom;
  try {
    if (nblk < 0 || (nblk > 0 && (!Xb_dev || !P_dev || Xb_dev == P_dev || !blk_off || !blk_n)))
      throw StatusError(STROM_ERR_INVALID, "strom_kernel_psd_project_noalloc: bad arguments");
    if (nblk > kNoAllocMaxBlocks)
      throw StatusError(STROM_ERR_INVALID,
                        "strom_kernel_psd_project_noalloc: at most 65536 blocks per call (static scratch size)");
    if (precision != STROM_PREC_FP64 && precision != STROM_PREC_FP32)
      throw StatusError(STROM_ERR_INVALID, "strom_kernel_psd_project_noalloc: precision must be FP64 or FP32");
    for (int i = 0; i < nblk; ++i)
      if (blk_n[i] < 1 || blk_n[i] > 160 || blk_off[i] < 0)
        throw StatusError(STROM_ERR_INVALID, "strom_kernel_psd_project_noalloc: block size must be in 1..160");
    NoAllocScratch* sc = scratch_for_current_device();
    if (nblk == 0) return STROM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    STROM_CUDA(cudaMemcpyAsync(sc->off, blk_off, sizeof(int64_t) * nblk, cudaMemcpyHostToDevice, st));
    STROM_CUDA(cudaMemcpyAsync(sc->n, blk_n, sizeof(int32_t) * nblk, cudaMemcpyHostToDevice, st));
    classify_kernel<<<1, 1024, 0, st>>>(sc, nblk);
    STROM_CUDA(cudaGetLastError());
    count_launches(1);
    int32_t cls[8];
    STROM_CUDA(cudaMemcpyAsync(cls, sc->cls, sizeof(cls), cudaMemcpyDeviceToHost, st));
    STROM_CUDA(cudaStreamSynchronize(st));
    PsdArgs a{};
    a.Xb = Xb_dev;
    a.out = P_dev;
    a.blk_off = sc->off;
    a.blk_n = sc->n;
    a.blk_list = sc->list;
    a.lam_off = nullptr;  // no eigenvalue output: the kernels read lam_off only with lam or topvec
    a.vscratch = sc->vs;
    // FP64 blocks of the largest class keep V in the static scratch: run them
    // in chunks of at most kNoAllocMaxVBlocks, in stream order
    PsdClasses c{};
    for (int k = 0; k < 4; ++k) { c.count[k] = cls[k]; c.start[k] = cls[4 + k]; }
    if (precision == STROM_PREC_FP64 && c.count[3] > kNoAllocMaxVBlocks) {
      PsdClasses small = c;
      small.count[3] = 0;
      psd_launch(a, small, precision, st);
      for (int done = 0; done < c.count[3]; done += kNoAllocMaxVBlocks) {
        PsdClasses chunk{};
        chunk.start[3] = c.start[3] + done;
        chunk.count[3] = std::min(kNoAllocMaxVBlocks, c.count[3] - done);
        psd_launch(a, chunk, precision, st);
      }
    } else {
      psd_launch(a, c, precision, st);
    }
    STROM_CUDA(cudaStreamSynchronize(st));
    return STROM_OK;
  } catch (const StatusError& e) {
    set_error(e.what());
    return e.status;
  } catch (const std::exception& e) {
    set_error(e.what());
    return STROM_ERR_CUDA;
  }
}
