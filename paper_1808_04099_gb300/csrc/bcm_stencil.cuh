// bcm_stencil.cuh -- pieces shared by the cell-stencil kernels of the fractional step
// (bcm_kernels.cu, bcm_momentum.cu): the ghost rules of the velocity and pressure
// halos (R8), field accessors, the lagged-convection storage type, and the launch
// helpers (threads per block, z-slab depth, shared-memory opt-in, cube-size dispatch).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "bcm_cube.cuh"
#include "bcm_internal.cuh"
#include "bcm_kernels.h"

namespace bcm {

// ------------------------------------------------------------ small helpers

template <int B>
__device__ __forceinline__ int face_w3_sum(const DevGrid& g, int c, int cell) {
  const int i = cell % B, j = (cell / B) % B, k = cell / (B * B);
  int s3 = 18;
  if (i == 0) s3 += g.w3[6 * c + 0] - 3;
  if (i == B - 1) s3 += g.w3[6 * c + 1] - 3;
  if (j == 0) s3 += g.w3[6 * c + 2] - 3;
  if (j == B - 1) s3 += g.w3[6 * c + 3] - 3;
  if (k == 0) s3 += g.w3[6 * c + 4] - 3;
  if (k == B - 1) s3 += g.w3[6 * c + 5] - 3;
  return s3;
}

// 1 / diag(K) of a cell: Jacobi preconditioner of the PCG (R11).
template <int B>
__device__ __forceinline__ double inv_diag(const DevGrid& g, int c, int cell) {
  return g.sp[g.sim[c]].invdiag[g.lvl[c]][face_w3_sum<B>(g, c, cell)];
}

// Ghost rule that is never used (faces whose values come from the boundary data).
struct KeepBC {
  template <class U>
  __device__ __forceinline__ U operator()(int, int, int, U x) const { return x; }
};

// Pressure-like ghost: Neumann (mirror) except Dirichlet p = 0 at outflow faces.
struct PressureBC {
  const SimParams* sp;
  template <class T>
  __device__ __forceinline__ T operator()(int f, int, int, T p0) const {
    return sp->bc[f] == BC_OUTFLOW ? -p0 : p0;
  }
};

// Velocity ghost rules (R8) for component comp.
template <int B, class T>
struct VelocityBC {
  const DevGrid* g;
  const SimParams* sp;
  const T* ub;
  int c, comp;
  __device__ __forceinline__ T operator()(int f, int a, int b, T u0) const {
    const int bc = sp->bc[f];
    if (bc == BC_SLIP) return (comp == (f >> 1)) ? -u0 : u0;
    if (bc == BC_OUTFLOW) {
      const int sl = g->slot[6 * c + f];
      return T(2) * ub[((size_t)(sl * 3 + comp) * B + b) * B + a] - u0;
    }
    return T(2.0 * face_velocity<B>(*g, c, f, comp, a, b)) - u0;
  }
};

// The same rules for a velocity of t^{n+1} (the iterates of the implicit half of
// Eq. substep1): outflow faces take the face value advanced by the convective update
// u_b^{n+1} = u_b^n - U_c dt (u_b^n - u_0^n) / (h/2) (R8), u_0^n the face cell of u^n.
template <int B, class T>
struct VelocityBCNext {
  const DevGrid* g;
  const SimParams* sp;
  const T* ub;
  const T* un;  // u^n of this component
  int c, comp;
  T coef;       // U_c dt / (h/2) of cube c
  __device__ __forceinline__ T operator()(int f, int a, int b, T u0) const {
    const int bc = sp->bc[f];
    if (bc == BC_SLIP) return (comp == (f >> 1)) ? -u0 : u0;
    if (bc == BC_OUTFLOW) {
      const int sl = g->slot[6 * c + f];
      const T vb = ub[((size_t)(sl * 3 + comp) * B + b) * B + a];
      const int d = f >> 1;
      const T uf = un[(size_t)c * B * B * B + cell_of<B>(d, (f & 1) ? B - 1 : 0, a, b)];
      return T(2) * (vb - coef * (vb - uf)) - u0;
    }
    return T(2.0 * face_velocity<B>(*g, c, f, comp, a, b)) - u0;
  }
};

template <class T>
struct FieldVal {
  const T* f;
  int B3;
  __device__ __forceinline__ T operator()(int c, int cell) const {
    return f[(size_t)c * B3 + cell];
  }
  // cells cell0 .. cell0+3 (cell0 a multiple of 4: one 16-byte access)
  __device__ __forceinline__ void get4(int c, int cell0, T (&v)[4]) const {
    ld4(f + (size_t)c * B3 + cell0, v);
  }
};



// The lagged convection N^{n-1} in its storage type: the state type, or bfloat16
// (round to nearest even) in mixed mode when the grid asks for it.
__device__ __forceinline__ float lag_load(const float* p) { return *p; }
__device__ __forceinline__ double lag_load(const double* p) { return *p; }
__device__ __forceinline__ float lag_load(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void lag_store(float* p, float v) { *p = v; }
__device__ __forceinline__ void lag_store(double* p, double v) { *p = v; }
__device__ __forceinline__ void lag_store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

template <int B>
constexpr int threads_for() { return B == 16 ? 256 : (B == 8 ? 128 : 64); }
// z-slab depth of the three-field kernels (shared memory 3 (KS+2)(B+2)^2 values)
template <int B, class T>
constexpr int slab3() { return B == 16 ? (sizeof(T) == 8 ? 4 : 8) : B; }

template <class K>
inline cudaError_t allow_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define BCM_DISPATCH_B(Bv, ...)                      \
  switch (Bv) {                                      \
    case 4: { constexpr int B = 4; __VA_ARGS__; break; }   \
    case 8: { constexpr int B = 8; __VA_ARGS__; break; }   \
    case 16: { constexpr int B = 16; __VA_ARGS__; break; } \
    default: return cudaErrorInvalidValue;           \
  }

}  // namespace bcm
