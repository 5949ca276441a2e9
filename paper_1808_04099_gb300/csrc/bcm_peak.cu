// bcm_peak.cu -- measured fused multiply-add rates of the device (FP64 and FP32), the
// denominators of the ALU-bound rooflines of the FP64 kernels.  No counterpart in the
// paper: the step's FP64 passes run on a part whose FP64 rate is a small fraction of
// its FP32 rate, so their bound is min(HBM bandwidth, FMA rate x arithmetic intensity),
// and the FMA rate is measured here rather than taken from a data sheet.
//
// Every thread runs eight independent FMA chains v = v a + b (a just below one, so the
// chains converge instead of overflowing); the sum of the chains goes to a device sink
// only when it equals an impossible value, which keeps the chains live without a store
// per iteration.  Two FLOPs per FMA.
#include <cuda_runtime.h>

#include "../../include/bcm.h"

namespace bcm {
bcm_status grid_fail(bcm_status st, const char* msg);
}

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

static __device__ double g_fma_sink[2];

template <class T>
__global__ __launch_bounds__(kThreads) void k_fma_chains(int iters, T a, T b) {
  T v[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) v[q] = T(threadIdx.x + q + 1) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) v[q] = fma(v[q], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += v[q];
  if (s == T(-12345.0)) g_fma_sink[sizeof(T) == 8 ? 0 : 1] = double(s);
}

template <class T>
cudaError_t time_chains(int blocks, int iters, cudaStream_t s, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  cudaEventRecord(e0, s);
  k_fma_chains<T><<<blocks, kThreads, 0, s>>>(iters, T(0.999999), T(1e-6));
  e = cudaGetLastError();
  cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace

extern "C" bcm_status bcm_measure_fma_rate(int fp64, double* flops_per_s) {
  if (!flops_per_s) return bcm::grid_fail(BCM_E_INVALID, "flops_per_s is NULL");
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return bcm::grid_fail(BCM_E_CUDA, "no current CUDA device");
  const int blocks = nsm * 8;  // eight blocks of 256 threads per SM: 64 warps
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
    return bcm::grid_fail(BCM_E_CUDA, "stream creation failed");
  // calibrate the chain length to about 20 ms, then keep the best of three runs
  int iters = 256;
  float ms = 0.f, best = 0.f;
  cudaError_t e = cudaSuccess;
  for (int cal = 0; cal < 12 && e == cudaSuccess; ++cal) {
    e = fp64 ? time_chains<double>(blocks, iters, s, &ms) : time_chains<float>(blocks, iters, s, &ms);
    if (e != cudaSuccess || ms >= 10.f) break;
    iters *= 4;
  }
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    e = fp64 ? time_chains<double>(blocks, iters, s, &ms) : time_chains<float>(blocks, iters, s, &ms);
    if (e == cudaSuccess && (best == 0.f || ms < best)) best = ms;
  }
  cudaStreamDestroy(s);
  if (e != cudaSuccess) return bcm::grid_fail(BCM_E_CUDA, cudaGetErrorString(e));
  const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
  *flops_per_s = flops / (best * 1e-3);
  return BCM_OK;
}
