// dl_correlate_noalloc: the correlation product A = Y^T D without any device
// allocation, for callers that cannot call cudaMalloc.
//
// Who needs it: code whose device memory is entirely reserved by another
// allocator (a framework's caching pool or a fixed arena, where a cudaMalloc
// would fail or fragment the pool), and code on a latency-critical path where
// the implicit device synchronisation of an allocation is not acceptable.
// Such callers own Y, D and A but cannot give the library a workspace.
//
// The tensor-core path needs the TF32 head/tail split of D as scratch.  Here
// that scratch is a file-scope __device__ array of fixed size, present on every
// GPU that loads the library until the process exits.  Host code cannot use
// the array's name as a device address (in host code it names a host-side
// stand-in), so the device address is queried once per device with
// cudaGetSymbolAddress, with that device current, and passed to the kernels.
#include "../../include/dl_gb300.h"
#include "dl_internal.cuh"

#include <cuda_runtime.h>
#include <mutex>
#include <stdint.h>

namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kScratchFloats = 2u * DL_NOALLOC_MAX_N * DL_NOALLOC_MAX_P;  // D_hi, D_lo

// Scratch shared by every call on a device: D_hi | D_lo | error word.
static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats + 64];

std::mutex g_setup_mutex;
float* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (first call per
// device queries it; later calls reuse it).  nullptr on failure.
float* scratch_for_current_device(int* dev_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  *dev_out = dev;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_scratch_ptr[dev] = (float*)p;
  }
  return g_scratch_ptr[dev];
}

}  // namespace

extern "C" int dl_correlate_noalloc(const float* Y, int64_t m, const float* D, int p, int n,
                                    float* A, void* stream) {
  // sizes beyond the fixed scratch are rejected
  if (!Y || !D || !A || m < 0 || p < 1 || p > DL_NOALLOC_MAX_P || n < 1 || n > DL_NOALLOC_MAX_N)
    return DL_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (m == 0) return DL_OK;
  const bool tc = dlk::corr_tc_supported(Y, p, n, n) && dlk::corr_tc_supported(D, p, n, n) &&
                  ((uintptr_t)A % 16) == 0;
  if (!tc) {
    // p not a multiple of 4, n not a multiple of 16 or an operand (A included) off a
    // 16-byte boundary: the FP32 CUDA-core GEMM, which needs no scratch
    return dlk::gemm_nt_simt(Y, m, D, n, p, A, n, st) == cudaSuccess ? DL_OK : DL_ECUDA;
  }
  int dev = 0;
  float* scratch = scratch_for_current_device(&dev);
  if (!scratch) return DL_ECUDA;
  float* dhi = scratch;
  float* dlo = scratch + (size_t)DL_NOALLOC_MAX_N * DL_NOALLOC_MAX_P;
  int* err = (int*)(scratch + kScratchFloats);
  // the error word keeps the previous call's value: clear it
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return DL_ECUDA;
  if (dlk::split_tf32(D, (int64_t)n * p, dhi, dlo, st) != cudaSuccess) return DL_ECUDA;
  if (dlk::corr_tf32x3(Y, m, dhi, dlo, n, p, A, n, err, st) != cudaSuccess) return DL_ECUDA;
  return DL_OK;
}

extern "C" int dl_correlate_noalloc_status(void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  float* scratch = scratch_for_current_device(&dev);
  if (!scratch) return DL_ECUDA;
  int* err = (int*)(scratch + kScratchFloats);
  int h = 0;  // a host int: the copy below allocates nothing on the device
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return DL_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return DL_ECUDA;
  if (h && cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return DL_ECUDA;
  if (h & dlk::ERR_NONFINITE) return DL_ENUMERIC;
  if (h & dlk::ERR_TIMEOUT) return DL_ETIMEOUT;
  return DL_OK;
}
