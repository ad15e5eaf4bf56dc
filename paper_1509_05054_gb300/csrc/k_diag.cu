// Failure-path diagnostic of the bounded waits.  Every mbarrier wait of the
// tensor-core kernels gives up after a fixed span of the GPU's global timer,
// flags ERR_TIMEOUT in the device error word and lets the kernel return, so a
// lost arrival ends as an error status instead of a hang.  This kernel runs
// exactly that path on purpose: one thread waits on phase 0 of an mbarrier that
// nothing arrives at.
#include "dl_internal.cuh"
#include "tc_ptx.cuh"

namespace dlk {
namespace {

__global__ void wait_timeout_kernel(int* err) {
  __shared__ __align__(8) uint64_t bar;
  tc::mbar_init(&bar, 1);
  if (!tc::mbar_wait(&bar, 0)) atomicOr(err, ERR_TIMEOUT);
}

// FP32 throughput probe: every thread runs 8 independent FMA chains of float2
// pairs (packed FFMA2 when PACKED, else 16 scalar FFMA chains), `iters` times.
// Enough warps and independent chains keep the FMA pipe busy, so the rate it
// reaches is the SM's FP32 multiply-add peak at the running clock.  The
// result is stored only under a condition the chains never meet, which keeps
// them live without memory traffic.
template <bool PACKED>
__global__ void __launch_bounds__(256) ffma_probe_kernel(int64_t iters, float* out) {
  const float t = 1e-3f * (float)(threadIdx.x & 63);
  float2 a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = make_float2(t + (float)k, t - (float)k);
  const float2 b = make_float2(0.9999999f, 0.9999999f), c = make_float2(1e-7f, -1e-7f);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if constexpr (PACKED) {
        a[k] = __ffma2_rn(a[k], b, c);
      } else {
        a[k].x = fmaf(a[k].x, b.x, c.x);
        a[k].y = fmaf(a[k].y, b.y, c.y);
      }
    }
  }
  float sum = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) sum += a[k].x + a[k].y;
  if (sum == -1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

}  // namespace

cudaError_t ffma_probe(int packed, int64_t iters, float* out, double* flops, cudaStream_t st) {
  const unsigned blocks = (unsigned)(num_sms() * 4);
  constexpr int threads = 256;
  *flops = (double)blocks * threads * (double)iters * 16.0 * 2.0;
  if (packed)
    ffma_probe_kernel<true><<<blocks, threads, 0, st>>>(iters, out);
  else
    ffma_probe_kernel<false><<<blocks, threads, 0, st>>>(iters, out);
  return cudaGetLastError();
}

cudaError_t bounded_wait_check(int* err, cudaStream_t st) {
  wait_timeout_kernel<<<1, 1, 0, st>>>(err);
  return cudaGetLastError();
}

}  // namespace dlk
