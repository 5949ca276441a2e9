// bcm_momentum.cu -- the momentum sub-step with the IB forcing and the Poisson
// right-hand side (arXiv:1808.04099, section "Numerical algorithm", Eq. substep1 and
// Eq. poisson), three-field z-slab stencils: each block stages its slab of u, v, w with
// the one-cell face halo (same level, 2:1, domain ghosts) in shared memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bcm_cube.cuh"
#include "bcm_internal.cuh"
#include "bcm_kernels.h"
#include "bcm_stencil.cuh"

namespace bcm {

// ===========================================================================
// (a3,a5,a6,a7) momentum sub-step + IB forcing, fused with the halo staging.
//   N_c = (1/h) sum_d [F+ - F-],  F+ = (u_d,i + u_d,i+1)/2 (u_c,i + u_c,i+1)/2
//   L u_c = (1/h^2) sum_d (u_c,i+1 - 2 u_c,i + u_c,i-1)
//   u~ = u + dt [-(3/2 N^n - 1/2 N^{n-1}) + nu L u]      (R3; N^{-1} := N^0)
//   u* = u~ + phi (u_s - u~),  drag -= phi (u_s - u~) V / dt   (R5)
// and the convective outflow face update u_b^{n+1} (R8).
// ===========================================================================
template <int B, int KS, int NT, class T, class TN>
__global__ __launch_bounds__(NT) void k_momentum(
    DevGrid g, const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ w,
    T* __restrict__ us, T* __restrict__ vs, T* __restrict__ ws, TN* __restrict__ nx,
    TN* __restrict__ ny, TN* __restrict__ nz, const T* __restrict__ phi,
    const unsigned char* __restrict__ bid, T* __restrict__ ub) {
  using SL = Slab<B, KS>;
  constexpr int B3 = B * B * B, NSL = B / KS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S0 = reinterpret_cast<T*>(smem_raw);
  T* S1 = S0 + SL::N;
  T* S2 = S1 + SL::N;
  __shared__ double red[3 * 32];
  const int c = blockIdx.x / NSL, z0 = (blockIdx.x % NSL) * KS;
  const int s = g.sim[c];
  const SimParams& sp = g.sp[s];
  {
    VelocityBC<B, T> b0{&g, &sp, ub, c, 0}, b1{&g, &sp, ub, c, 1}, b2{&g, &sp, ub, c, 2};
    stage_slab<B, KS, NT>(S0, g, c, z0, FieldVal<T>{u, B3}, b0);
    stage_slab<B, KS, NT>(S1, g, c, z0, FieldVal<T>{v, B3}, b1);
    stage_slab<B, KS, NT>(S2, g, c, z0, FieldVal<T>{w, B3}, b2);
  }
  __syncthreads();
  const double hd = cell_h<B>(g, c);
  const T h = T(hd), ih = T(1.0 / hd), ih2 = T(1.0 / (hd * hd));
  const T dt = T(sp.dt), nu = T(sp.nu);
  const bool first = g.ss[s].step == 0 || g.ss[s].ab2_restart != 0;
  const bool has_phi = g.near[c] != 0;
  const double t = g.ss[s].step * sp.dt;
  const T* Sf[3] = {S0, S1, S2};
  T* outs[3] = {us, vs, ws};
  TN* Ns[3] = {nx, ny, nz};
  T fsum[3] = {T(0), T(0), T(0)};
  for (int q = threadIdx.x; q < KS * B * B; q += NT) {
    const int kk = q / (B * B), rem = q - kk * B * B, j = rem / B, i = rem - j * B;
    const int k = z0 + kk;
    const size_t gi = (size_t)c * B3 + (k * B + j) * B + i;
    const int o = SL::at(i, j, kk + 1);
    const int off[3] = {1, SL::P, SL::P * SL::P};
    T ph = T(0);
    T usb[3] = {T(0), T(0), T(0)};
    if (has_phi) {
      ph = phi[gi];
      if (ph != T(0)) {
        const bcm_body& bd = sp.bodies[bid[gi]];
        double x[3] = {centre<B>(g, c, 0, i), centre<B>(g, c, 1, j), centre<B>(g, c, 2, k)};
        double r[3];
        for (int e = 0; e < 3; ++e) r[e] = x[e] - (bd.center[e] + bd.vel[e] * t);
        usb[0] = T(bd.vel[0] + bd.omega[1] * r[2] - bd.omega[2] * r[1]);
        usb[1] = T(bd.vel[1] + bd.omega[2] * r[0] - bd.omega[0] * r[2]);
        usb[2] = T(bd.vel[2] + bd.omega[0] * r[1] - bd.omega[1] * r[0]);
      }
    }
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      const T* Sc = Sf[comp];
      const T u0 = Sc[o];
      T N = T(0), L = T(0);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const T* Sd = Sf[d];
        const int e = off[d];
        const T Fp = T(0.5) * (Sd[o] + Sd[o + e]) * (T(0.5) * (u0 + Sc[o + e]));
        const T Fm = T(0.5) * (Sd[o - e] + Sd[o]) * (T(0.5) * (Sc[o - e] + u0));
        N += Fp - Fm;
        L += Sc[o + e] - T(2) * u0 + Sc[o - e];
      }
      N *= ih;
      L *= ih2;
      const T Np = first ? N : T(lag_load(Ns[comp] + gi));
      const T ut = u0 + dt * (-(T(1.5) * N - T(0.5) * Np) + nu * L);
      const T du = ph * (usb[comp] - ut);
      outs[comp][gi] = ut + du;
      lag_store(Ns[comp] + gi, N);
      fsum[comp] += du;
    }
  }
  // convective outflow: u_b^{n+1} = u_b - U_c dt (u_b - u_0) / (h/2), this slab's cells
  for (int f = 0; f < 6; ++f) {
    const int sl = g.slot[6 * c + f];
    if (sl < 0) continue;
    const int d = f >> 1, side = f & 1;
    const T coef = T(sp.uconv * sp.dt / (0.5 * hd));
    if (d == 2) {
      if ((side == 0 && z0 != 0) || (side == 1 && z0 + KS != B)) continue;
      for (int q = threadIdx.x; q < 3 * B * B; q += NT) {
        const int comp = q / (B * B), rem = q - comp * B * B, b = rem / B, a = rem - b * B;
        const T u0 = Sf[comp][SL::at(a, b, side ? KS : 1)];
        T* pb = &ub[((size_t)(sl * 3 + comp) * B + b) * B + a];
        *pb = *pb - coef * (*pb - u0);
      }
    } else {
      for (int q = threadIdx.x; q < 3 * KS * B; q += NT) {
        const int comp = q / (KS * B), rem = q - comp * KS * B, kk = rem / B, t2 = rem - kk * B;
        const int k = z0 + kk, a = t2, b = k;
        const int nrm = side ? B - 1 : 0;
        const int o = d == 0 ? SL::at(nrm, t2, kk + 1) : SL::at(t2, nrm, kk + 1);
        const T u0 = Sf[comp][o];
        T* pb = &ub[((size_t)(sl * 3 + comp) * B + b) * B + a];
        *pb = *pb - coef * (*pb - u0);
      }
    }
  }
  if (has_phi) {  // drag: force of the fluid on the body = -sum f V, f = du/dt
    double vals[3] = {double(fsum[0]), double(fsum[1]), double(fsum[2])};
    block_sum<NT, 3>(vals, red);
    if (threadIdx.x == 0) {
      const double scale = -hd * hd * hd / sp.dt;
      for (int e = 0; e < 3; ++e) atomicAdd(&g.ss[s].drag_acc[e], vals[e] * scale);
    }
  }
}

// ===========================================================================
// (a8) Poisson right-hand side b = (1/dt)(1/h) sum_f A U_f.n  (R2): interior faces
// average the two cells, domain faces take the boundary normal velocity.
// ===========================================================================
template <int B, int KS, int NT, class T>
__global__ __launch_bounds__(NT) void k_rhs(DevGrid g, const T* __restrict__ us,
                                            const T* __restrict__ vs, const T* __restrict__ ws,
                                            const T* __restrict__ ub, double* __restrict__ b) {
  using SL = Slab<B, KS>;
  constexpr int B3 = B * B * B, NSL = B / KS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S0 = reinterpret_cast<T*>(smem_raw);
  T* S1 = S0 + SL::N;
  T* S2 = S1 + SL::N;
  __shared__ double red[32];
  const int c = blockIdx.x / NSL, z0 = (blockIdx.x % NSL) * KS;
  const int s = g.sim[c];
  const SimParams& sp = g.sp[s];
  KeepBC keep;
  stage_slab<B, KS, NT>(S0, g, c, z0, FieldVal<T>{us, B3}, keep);
  stage_slab<B, KS, NT>(S1, g, c, z0, FieldVal<T>{vs, B3}, keep);
  stage_slab<B, KS, NT>(S2, g, c, z0, FieldVal<T>{ws, B3}, keep);
  __syncthreads();
  const T* Sf[3] = {S0, S1, S2};
  const double hd = cell_h<B>(g, c);
  const double scale = 1.0 / (hd * sp.dt);
  int code[6];
  for (int f = 0; f < 6; ++f) code[f] = g.nb[6 * c + f];
  const T* const comps[3] = {us, vs, ws};
  double bsum = 0.0;
  for (int q = threadIdx.x; q < KS * B * B; q += NT) {
    const int kk = q / (B * B), rem = q - kk * B * B, j = rem / B, i = rem - j * B;
    const int k = z0 + kk;
    const int ii[3] = {i, j, k};
    const int o = SL::at(i, j, kk + 1);
    const int off[3] = {1, SL::P, SL::P * SL::P};
    T div = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T* Sd = Sf[d];
      const int e = off[d];
      const int a = ii[tan1(d)], bb = ii[tan2(d)];
      // normal velocity through the low (side 0) and high (side 1) face of the cell
      T U2[2];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int f = 2 * d + side;
        const bool on_face = side ? (ii[d] == B - 1) : (ii[d] == 0);
        const T other = side ? Sd[o + e] : Sd[o - e];
        if (on_face && code[f] == NB_BOUNDARY) {
          const int bc = sp.bc[f];
          U2[side] = bc == BC_SLIP ? T(0)
                     : bc == BC_OUTFLOW ? ub[((size_t)(g.slot[6 * c + f] * 3 + d) * B + bb) * B + a]
                                        : T(face_velocity<B>(g, c, f, d, a, bb));
        } else if (on_face && code[f] == NB_COARSE) {
          // fine cell, coarse neighbour: linear between the two centres (R7), the
          // staged halo holds the coarse cell
          U2[side] = (T(2) * Sd[o] + other) / T(3);
        } else if (on_face && code[f] == NB_FINE) {
          // coarse cell, four fine neighbours: area mean of the four sub-face values
          const T* comp = comps[d];
          auto valg = [&](int cube, int cell) { return comp[(size_t)cube * B3 + cell]; };
          const T m4 = poisson_ghost_21<B, T>(g, c, f, a, bb, NB_FINE, valg);
          U2[side] = (T(2) * m4 + Sd[o]) / T(3);
        } else {
          U2[side] = side ? T(0.5) * (Sd[o] + other) : T(0.5) * (other + Sd[o]);
        }
      }
      const T Um = U2[0], Up = U2[1];
      div = div - Um;
      div = div + Up;
    }
    const double bv = double(div) * scale;
    b[(size_t)c * B3 + (k * B + j) * B + i] = bv;
    bsum += bv;
  }
  double vals[1] = {bsum};
  block_sum<NT, 1>(vals, red);
  if (threadIdx.x == 0 && sp.all_neumann) acc_add(g.ss[s], ACC_BSUM, vals[0]);
  if (last_block(g.counter)) {
    for (int q = threadIdx.x; q < g.n_sims; q += NT) {
      SimState& st = g.ss[q];
      const double bs = acc_take(st, ACC_BSUM);
      st.bmean = g.sp[q].all_neumann ? bs / g.sp[q].n_cells : 0.0;
    }
  }
}

// ===========================================================================
// Launchers
// ===========================================================================

// z-slabs per cube of the three-field kernels: x.slabs_m on 16^3 cubes (1, 2 or 4; 0
// takes the default, 2 in FP32 and 4 in FP64, whose tiles of 3 (KS+2)(B+2)^2 values
// leave room for four blocks per SM), whole cubes below 16^3
template <int B, class T>
inline int stencil_slabs(const Ctx& x) {
  if (B != 16) return 1;
  return x.slabs_m ? x.slabs_m : B / slab3<B, T>();
}

template <class T, class TN, int B, int KS>
static cudaError_t momentum_ks(const Ctx& x) {
  constexpr int NT = threads_for<B>();
  const size_t sm = 3 * sizeof(T) * Slab<B, KS>::N;
  auto kern = k_momentum<B, KS, NT, T, TN>;
  cudaError_t e = allow_smem(kern, sm);
  if (e != cudaSuccess) return e;
  kern<<<x.g.n_cubes * (B / KS), NT, sm, x.stream>>>(
      x.g, (const T*)x.f.u, (const T*)x.f.v, (const T*)x.f.w, (T*)x.f.us, (T*)x.f.vs,
      (T*)x.f.ws, (TN*)x.f.nx, (TN*)x.f.ny, (TN*)x.f.nz, (const T*)x.f.phi, x.f.bid,
      (T*)x.f.ub);
  return cudaGetLastError();
}
template <class T, class TN>
static cudaError_t momentum_t(const Ctx& x) {
  BCM_DISPATCH_B(x.B, {
    if constexpr (B == 16) {
      switch (stencil_slabs<B, T>(x)) {
        case 1: return momentum_ks<T, TN, B, B>(x);
        case 2: return momentum_ks<T, TN, B, B / 2>(x);
        case 4: return momentum_ks<T, TN, B, B / 4>(x);
        default: return cudaErrorInvalidValue;
      }
    } else {
      return momentum_ks<T, TN, B, B>(x);
    }
  });
  return cudaSuccess;
}
cudaError_t launch_momentum(const Ctx& x) {
  if (x.f64) return momentum_t<double, double>(x);
  return x.lag_bf16 ? momentum_t<float, __nv_bfloat16>(x) : momentum_t<float, float>(x);
}

template <class T, int B, int KS>
static cudaError_t rhs_ks(const Ctx& x) {
  constexpr int NT = threads_for<B>();
  const size_t sm = 3 * sizeof(T) * Slab<B, KS>::N;
  auto kern = k_rhs<B, KS, NT, T>;
  cudaError_t e = allow_smem(kern, sm);
  if (e != cudaSuccess) return e;
  kern<<<x.g.n_cubes * (B / KS), NT, sm, x.stream>>>(x.g, (const T*)x.f.us, (const T*)x.f.vs,
                                                    (const T*)x.f.ws, (const T*)x.f.ub, x.f.b);
  return cudaGetLastError();
}
template <class T>
static cudaError_t rhs_t(const Ctx& x) {
  BCM_DISPATCH_B(x.B, {
    if constexpr (B == 16) {
      switch (stencil_slabs<B, T>(x)) {
        case 1: return rhs_ks<T, B, B>(x);
        case 2: return rhs_ks<T, B, B / 2>(x);
        case 4: return rhs_ks<T, B, B / 4>(x);
        default: return cudaErrorInvalidValue;
      }
    } else {
      return rhs_ks<T, B, B>(x);
    }
  });
  return cudaSuccess;
}
cudaError_t launch_rhs(const Ctx& x) { return x.f64 ? rhs_t<double>(x) : rhs_t<float>(x); }

}  // namespace bcm
