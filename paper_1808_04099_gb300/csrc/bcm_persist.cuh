// bcm_persist.cuh -- pieces shared by the persistent (cooperative) PCG kernels:
// the bounded grid barrier, sums of the rotating dot-product slots, and the
// co-resident grid size of a launch.
#pragma once

#include <cuda_runtime.h>

#include "bcm_internal.cuh"

namespace bcm {

constexpr int kMaxPersistentSims = 256;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch.  bar: [0] generation, [32 (1+s)] stripe
// counters, [32 (1+kTickets)] top counter (one 128-byte line each).  Thread 0 of each
// block reads the generation once at the start of the kernel (init) and counts the
// barriers it passes, so arriving costs no read of the generation: the generation
// moves only when every block has arrived, hence never twice while one block waits.
// sync() returns false (and sets *err) when the wait exceeded limit_ns or another
// block reported an error.
struct GridBarrier {
  unsigned int* bar;
  int* err;
  unsigned long long limit_ns;
  unsigned int gen;  // generation this block waits to see change (thread 0)

  __device__ __forceinline__ void init(unsigned int* b, int* e, unsigned long long limit) {
    bar = b;
    err = e;
    limit_ns = limit;
    gen = threadIdx.x == 0 ? *(volatile unsigned int*)b : 0u;
  }

  __device__ __forceinline__ bool sync() {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
      volatile unsigned int* g = bar;
      __threadfence();  // this block's writes before its arrival
      const unsigned int nblk = gridDim.x;
      const unsigned int stripe = blockIdx.x % kTickets;
      const unsigned int in_stripe = (nblk - stripe + kTickets - 1) / kTickets;
      const unsigned int t = atomicAdd(&bar[32 * (1 + stripe)], 1u);
      bool released = false;
      if (t == in_stripe - 1) {
        bar[32 * (1 + stripe)] = 0u;
        __threadfence();
        const unsigned int stripes = nblk < (unsigned)kTickets ? nblk : (unsigned)kTickets;
        const unsigned int u = atomicAdd(&bar[32 * (1 + kTickets)], 1u);
        if (u == stripes - 1) {
          bar[32 * (1 + kTickets)] = 0u;
          __threadfence();
          atomicAdd(&bar[0], 1u);
          released = true;
        }
      }
      int good = 1;
      if (!released) {
        const unsigned long long t0 = global_ns();
        while (*g == gen) {
          if (*(volatile int*)err) {
            good = 0;
            break;
          }
          if (global_ns() - t0 > limit_ns) {
            atomicExch(err, 1);
            good = 0;
            break;
          }
          __nanosleep(32);
        }
      }
      gen += 1;
      __threadfence();
      ok = good;
    }
    __syncthreads();
    return ok != 0;
  }
};

__device__ __forceinline__ double slot_sum(SimState& st, int idx) {
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kStripes; ++q) s += ld_acc(&st.acc[q][idx]);
  return s;
}

// Dynamic shared memory beyond the default limit (48 KB minus the kernel's static
// shared memory) needs the kernel's opt-in.
template <class K>
inline cudaError_t allow_dynamic_smem(K kern, size_t dyn) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  if (fa.sharedSizeBytes + dyn > 48 * 1024)
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  return cudaSuccess;
}

template <int B>
constexpr int pcg_threads() { return B == 16 ? 256 : (B == 8 ? 128 : 64); }

// Largest co-resident grid for one kernel configuration.
template <class K>
inline int max_coresident(K kern, int nt, size_t smem, int* out) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, nt, smem);
  if (e != cudaSuccess) return (int)e;
  *out = per * nsm;
  return 0;
}

}  // namespace bcm
