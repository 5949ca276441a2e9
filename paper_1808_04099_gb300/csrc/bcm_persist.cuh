// bcm_persist.cuh -- pieces shared by the persistent (cooperative) PCG kernels:
// the bounded grid barrier, sums of the rotating dot-product slots, and the
// co-resident grid size of a launch.
#pragma once

#include <cuda_runtime.h>

#include "bcm_internal.cuh"

namespace bcm {

constexpr int kMaxPersistentSims = 256;

// Condition of a conditional graph node, set from a kernel inside that node's graph or
// body (a zero handle: no graph loop, nothing to set).
__device__ __forceinline__ void set_cond(unsigned long long handle, unsigned int v) {
  if (handle) cudaGraphSetConditional((cudaGraphConditionalHandle)handle, v);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch: one arrival counter, bar[32] (a 128-byte
// line of its own), zeroed before every launch (launch_pcg).  A block arrives with a
// release reduction that returns nothing (thread 0, after the block barrier) and waits,
// reading the counter with acquire loads, until it reaches gridDim.x times the number
// of barriers it has passed, so the release costs one round trip after the last
// arrival and no full fence is needed on either side.
// sync() returns false (and sets *err) when the wait exceeded limit_ns or another
// block reported an error.
struct GridBarrier {
  unsigned int* count;
  int* err;
  unsigned long long limit_ns;
  unsigned int passed;  // barriers this block has passed (thread 0)

  __device__ __forceinline__ void init(unsigned int* bar, int* e, unsigned long long limit) {
    count = bar + 32;
    err = e;
    limit_ns = limit;
    passed = 0u;
  }

  __device__ __forceinline__ bool sync() {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
      // arrival with release semantics: the block's writes (ordered before this thread
      // by the block barrier) are visible to every block that acquires the count
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
      passed += 1u;
      const unsigned int target = passed * gridDim.x;
      int good = 1;
      if ((int)(acquire_count() - target) < 0) {
        const unsigned long long t0 = global_ns();
        while ((int)(acquire_count() - target) < 0) {
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
      ok = good;
    }
    __syncthreads();
    return ok != 0;
  }

  // the arrival count, read with acquire semantics (the other blocks' writes before
  // their arrivals are visible to this block after the block barrier that follows)
  __device__ __forceinline__ unsigned int acquire_count() const {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
    return v;
  }
};

__device__ __forceinline__ double slot_sum(SimState& st, int idx) {
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kStripes; ++q) s += ld_acc(&st.acc[q][idx]);
  return s;
}

// The sums of two striped accumulators of one sim, read by one warp in one round trip:
// lanes 0 .. kStripes-1 load the stripes of idx_a, the next kStripes lanes those of
// idx_b; every lane gets both sums (a fixed summation order, the same in every block).
__device__ __forceinline__ void warp_slot_sums(SimState& st, int idx_a, int idx_b, double& a,
                                               double& b) {
  static_assert(2 * kStripes <= 32, "one warp reads both accumulators' stripes");
  const int lane = threadIdx.x & 31;
  double v = 0.0;
  if (lane < 2 * kStripes) v = ld_acc(&st.acc[lane % kStripes][lane < kStripes ? idx_a : idx_b]);
#pragma unroll
  for (int o = 1; o < kStripes; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  a = __shfl_sync(0xffffffffu, v, 0);
  b = __shfl_sync(0xffffffffu, v, kStripes);
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

// Launch with programmatic dependent launch: the kernel may be scheduled while the
// previous kernel on the stream drains, and must pass cudaGridDependencySynchronize()
// before it reads or writes anything that kernel touches (a kernel launched without
// the attribute passes it at once).
template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t stream, Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
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
