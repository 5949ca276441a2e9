// bcm_ib.cu -- Lagrangian-particle immersed boundary (arXiv:1808.04099, section
// "Lagrangian Data Structure"; section "Lagrangian-Eulerian Interaction" with Eqs.
// ddeltai and ddeltap and the smoothed 3-point delta; the forcing sub-step and the
// position update of section "Numerical algorithm"), on single-level grids.
//
// Particles stay in id order (X, F, sim, body, dV).  The paper groups them into one set
// per cube, kept in hash tables keyed by a global particle id, and moves runaway
// particles into the set of the cube they entered; here the sets are rebuilt from the
// positions by a counting sort whenever particles move: a count per cube, one exclusive
// scan and a scatter of the ids (set order within a cube is arbitrary).  The forcing
// walks the particles set by set, so neighbouring threads read neighbouring cells:
//   interpolation  U_q = sum_cells u~ phi(r_x) phi(r_y) phi(r_z)          (Eq. ddeltai)
//   force          F_q = (rho / dt) (U_s(X_q, t^n) - U_q)
//   spreading      u* = u~ + (dt / rho) sum_q F_q phi phi phi dV_q / h^3  (Eq. ddeltap)
// over the 27 cells whose centres lie within 1.5 h of the particle per axis; cells
// outside the domain are left out of both sums.  rho = 1.  Interpolation accumulates in
// FP64 for either state type; spreading adds into u* with atomics.  The force on the
// body, -sum_q F_q dV_q, goes into the sim's drag accumulator.  After the step,
// X^{n+1} = X^n + dt U_s(X^n, t^{n+1}) with the rigid motion of the particle's body.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bcm_internal.cuh"
#include "bcm_kernels.h"

namespace bcm {

namespace {

constexpr int kIbThreads = 128;

// one-dimensional smoothed 3-point delta phi(r) (printed after Eq. ddeltap)
__device__ __forceinline__ double delta3(double r) {
  const double a = fabs(r);
  if (a <= 0.5) return 0.75 - r * r;
  if (a <= 1.5) return 0.5 * (2.25 - 3.0 * a + r * r);
  return 0.0;
}

// The three cells around a particle along each axis: cube coordinate (-1: outside the
// domain), index inside the cube and 1-D delta weight.
struct Stencil {
  int cc[3][3];
  int li[3][3];
  double w[3][3];
};

__device__ __forceinline__ void particle_stencil(const DevGrid& g, const PartDev& P, int B,
                                                 int q, int s, Stencil& st) {
  const SimParams& sp = g.sp[s];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const double xi = (P.X[3 * q + e] - sp.origin[e]) / sp.h0;
    const int ic = (int)floor(xi);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int I = ic + d - 1;
      st.w[e][d] = delta3(I + 0.5 - xi);
      const bool in = I >= 0 && I < sp.extent[e];
      st.cc[e][d] = in ? I / B : -1;
      st.li[e][d] = in ? I - (I / B) * B : 0;
    }
  }
}

// cube at cube coordinates (cx, cy, cz) of sim s, -1 where no cube is
__device__ __forceinline__ int lattice_cube(const PartDev& P, int s, int cx, int cy, int cz) {
  const int* m = P.lat_meta + 4 * s;
  if (cx < 0 || cy < 0 || cz < 0 || cx >= m[1] || cy >= m[2] || cz >= m[3]) return -1;
  return P.lat[m[0] + (cz * m[2] + cy) * m[1] + cx];
}

// Visit the stencil's cells inside the domain: f(cell index, weight).
template <class Fn>
__device__ __forceinline__ void for_stencil(const PartDev& P, int B, int s, const Stencil& st,
                                            Fn&& f) {
  const size_t B3 = (size_t)B * B * B;
  for (int dk = 0; dk < 3; ++dk) {
    if (st.cc[2][dk] < 0) continue;
    for (int dj = 0; dj < 3; ++dj) {
      if (st.cc[1][dj] < 0) continue;
      for (int di = 0; di < 3; ++di) {
        if (st.cc[0][di] < 0) continue;
        const int cube = lattice_cube(P, s, st.cc[0][di], st.cc[1][dj], st.cc[2][dk]);
        if (cube < 0) continue;
        const double w = st.w[0][di] * st.w[1][dj] * st.w[2][dk];
        f((size_t)cube * B3 + ((size_t)st.li[2][dk] * B + st.li[1][dj]) * B + st.li[0][di], w);
      }
    }
  }
}

// velocity of a particle's body at X and time t: vel + omega x (X - (center + vel t))
__device__ __forceinline__ void body_velocity(const SimParams& sp, int b, const double* X,
                                              double t, double* U) {
  if (b < 0 || b >= sp.n_bodies || sp.bodies[b].kind == 0) {
    U[0] = U[1] = U[2] = 0.0;
    return;
  }
  const bcm_body& bd = sp.bodies[b];
  double r[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) r[e] = X[e] - (bd.center[e] + bd.vel[e] * t);
  U[0] = bd.vel[0] + bd.omega[1] * r[2] - bd.omega[2] * r[1];
  U[1] = bd.vel[1] + bd.omega[2] * r[0] - bd.omega[0] * r[2];
  U[2] = bd.vel[2] + bd.omega[0] * r[1] - bd.omega[1] * r[0];
}

// ---- per-cube sets: count, scan, scatter

__global__ __launch_bounds__(kIbThreads) void k_ib_count(DevGrid g, PartDev P, int B) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P.n) return;
  const int s = P.sim[q];
  const SimParams& sp = g.sp[s];
  int cc[3];
  bool in = true;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int I = (int)floor((P.X[3 * q + e] - sp.origin[e]) / sp.h0);
    in = in && I >= 0 && I < sp.extent[e];
    cc[e] = in ? I / B : 0;
  }
  const int cube = in ? lattice_cube(P, s, cc[0], cc[1], cc[2]) : -1;
  P.cube[q] = cube;
  if (cube >= 0) {
    atomicAdd(&P.set_count[cube], 1);
  } else {  // outside every cube: no force, reported to the host
    P.F[3 * q] = P.F[3 * q + 1] = P.F[3 * q + 2] = 0.0;
    atomicOr(P.err, 1);
  }
}

// exclusive scan of the counts into set_start (one block), cursors reset to zero
__global__ __launch_bounds__(1024) void k_ib_scan(PartDev P, int n_cubes) {
  __shared__ int buf[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n_cubes; base += 1024) {
    const int c = base + threadIdx.x;
    const int v = c < n_cubes ? P.set_count[c] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive Hillis-Steele scan
      const int add = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
      __syncthreads();
      buf[threadIdx.x] += add;
      __syncthreads();
    }
    if (c < n_cubes) {
      P.set_start[c] = carry + buf[threadIdx.x] - v;
      P.set_count[c] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 1023) carry += buf[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) P.set_start[n_cubes] = carry;
}

__global__ __launch_bounds__(kIbThreads) void k_ib_scatter(PartDev P) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P.n) return;
  const int cube = P.cube[q];
  if (cube < 0) return;
  P.set_ids[P.set_start[cube] + atomicAdd(&P.set_count[cube], 1)] = q;
}

// ---- forcing sub-step

// Drag: -F dV summed per sim; one atomic per block when its particles share a sim.
__device__ __forceinline__ void add_drag(const DevGrid& g, int s, const double (&fd)[3],
                                         bool active) {
  __shared__ int s_first;
  __shared__ double red[3 * 32];
  if (threadIdx.x == 0) s_first = -1;
  __syncthreads();
  if (active) atomicCAS(&s_first, -1, s);
  __syncthreads();
  const bool same = __syncthreads_and(!active || s == s_first) != 0;
  if (same) {
    double v[3] = {fd[0], fd[1], fd[2]};
    block_sum<kIbThreads, 3>(v, red);
    if (threadIdx.x == 0 && s_first >= 0)
      for (int e = 0; e < 3; ++e) atomicAdd(&g.ss[s_first].drag_acc[e], v[e]);
  } else if (active) {
    for (int e = 0; e < 3; ++e) atomicAdd(&g.ss[s].drag_acc[e], fd[e]);
  }
}

template <class T>
__global__ __launch_bounds__(kIbThreads) void k_ib_force(DevGrid g, PartDev P, int B,
                                                        const T* __restrict__ us,
                                                        const T* __restrict__ vs,
                                                        const T* __restrict__ ws) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = k < P.set_start[g.n_cubes];
  double fd[3] = {0.0, 0.0, 0.0};
  int s = 0;
  if (active) {
    const int q = P.set_ids[k];
    s = P.sim[q];
    const SimParams& sp = g.sp[s];
    Stencil st;
    particle_stencil(g, P, B, q, s, st);
    double U[3] = {0.0, 0.0, 0.0};
    for_stencil(P, B, s, st, [&](size_t cell, double w) {
      U[0] += double(us[cell]) * w;
      U[1] += double(vs[cell]) * w;
      U[2] += double(ws[cell]) * w;
    });
    double Us[3];
    body_velocity(sp, P.body[q], P.X + 3 * q, g.ss[s].step * sp.dt, Us);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const double F = (Us[e] - U[e]) / sp.dt;
      P.F[3 * q + e] = F;
      fd[e] = -F * P.dV[q];
    }
  }
  add_drag(g, s, fd, active);
}

template <class T>
__global__ __launch_bounds__(kIbThreads) void k_ib_spread(DevGrid g, PartDev P, int B,
                                                         T* __restrict__ us, T* __restrict__ vs,
                                                         T* __restrict__ ws) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.set_start[g.n_cubes]) return;
  const int q = P.set_ids[k], s = P.sim[q];
  const SimParams& sp = g.sp[s];
  Stencil st;
  particle_stencil(g, P, B, q, s, st);
  const double c = sp.dt * P.dV[q] / (sp.h0 * sp.h0 * sp.h0);
  const double f0 = c * P.F[3 * q], f1 = c * P.F[3 * q + 1], f2 = c * P.F[3 * q + 2];
  for_stencil(P, B, s, st, [&](size_t cell, double w) {
    atomicAdd(&us[cell], T(f0 * w));
    atomicAdd(&vs[cell], T(f1 * w));
    atomicAdd(&ws[cell], T(f2 * w));
  });
}

// X^{n+1} = X^n + dt U_s(X^n, t^{n+1}) (after the step counter has advanced)
__global__ __launch_bounds__(kIbThreads) void k_ib_move(DevGrid g, PartDev P) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P.n) return;
  const int s = P.sim[q];
  const SimParams& sp = g.sp[s];
  double* X = P.X + 3 * q;
  double Us[3];
  body_velocity(sp, P.body[q], X, g.ss[s].step * sp.dt, Us);
#pragma unroll
  for (int e = 0; e < 3; ++e) X[e] += sp.dt * Us[e];
}

// ---- test paths on FP64 arrays (every particle in a set)

__global__ __launch_bounds__(kIbThreads) void k_ib_interp_test(DevGrid g, PartDev P, int B,
                                                              const double* __restrict__ f,
                                                              double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.set_start[g.n_cubes]) return;
  const int q = P.set_ids[k], s = P.sim[q];
  Stencil st;
  particle_stencil(g, P, B, q, s, st);
  double U = 0.0;
  for_stencil(P, B, s, st, [&](size_t cell, double w) { U += f[cell] * w; });
  out[q] = U;
}

__global__ __launch_bounds__(kIbThreads) void k_ib_spread_test(DevGrid g, PartDev P, int B,
                                                              const double* __restrict__ F,
                                                              double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.set_start[g.n_cubes]) return;
  const int q = P.set_ids[k], s = P.sim[q];
  const SimParams& sp = g.sp[s];
  Stencil st;
  particle_stencil(g, P, B, q, s, st);
  const double c = F[q] * P.dV[q] / (sp.h0 * sp.h0 * sp.h0);
  for_stencil(P, B, s, st, [&](size_t cell, double w) { atomicAdd(&out[cell], c * w); });
}

unsigned int blocks_for(int n) { return (unsigned int)((n + kIbThreads - 1) / kIbThreads); }

}  // namespace

cudaError_t launch_ib_bin(const Ctx& x) {
  const PartDev& P = x.part;
  cudaError_t e = cudaMemsetAsync(P.set_count, 0, sizeof(int) * (size_t)x.g.n_cubes, x.stream);
  if (e != cudaSuccess) return e;
  if (P.n > 0) k_ib_count<<<blocks_for(P.n), kIbThreads, 0, x.stream>>>(x.g, P, x.B);
  k_ib_scan<<<1, 1024, 0, x.stream>>>(P, x.g.n_cubes);
  if (P.n > 0) k_ib_scatter<<<blocks_for(P.n), kIbThreads, 0, x.stream>>>(P);
  return cudaGetLastError();
}

template <class T>
static cudaError_t force_t(const Ctx& x) {
  const PartDev& P = x.part;
  const unsigned int nb = blocks_for(P.n);
  k_ib_force<T><<<nb, kIbThreads, 0, x.stream>>>(x.g, P, x.B, (const T*)x.f.us,
                                                (const T*)x.f.vs, (const T*)x.f.ws);
  k_ib_spread<T><<<nb, kIbThreads, 0, x.stream>>>(x.g, P, x.B, (T*)x.f.us, (T*)x.f.vs,
                                                 (T*)x.f.ws);
  return cudaGetLastError();
}

cudaError_t launch_ib_force(const Ctx& x) {
  if (x.part.n <= 0) return cudaSuccess;
  return x.f64 ? force_t<double>(x) : force_t<float>(x);
}

cudaError_t launch_ib_move(const Ctx& x) {
  if (x.part.n <= 0) return cudaSuccess;
  k_ib_move<<<blocks_for(x.part.n), kIbThreads, 0, x.stream>>>(x.g, x.part);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? launch_ib_bin(x) : e;
}

cudaError_t launch_ib_interpolate(const Ctx& x, const double* f, double* out) {
  if (x.part.n <= 0) return cudaSuccess;
  k_ib_interp_test<<<blocks_for(x.part.n), kIbThreads, 0, x.stream>>>(x.g, x.part, x.B, f, out);
  return cudaGetLastError();
}

cudaError_t launch_ib_spread(const Ctx& x, const double* F, double* out) {
  if (x.part.n <= 0) return cudaSuccess;
  k_ib_spread_test<<<blocks_for(x.part.n), kIbThreads, 0, x.stream>>>(x.g, x.part, x.B, F, out);
  return cudaGetLastError();
}

}  // namespace bcm
