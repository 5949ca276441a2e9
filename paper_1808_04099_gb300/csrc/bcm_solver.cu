// bcm_solver.cu -- pressure Poisson solver and projection kernels (arXiv:1808.04099,
// Eq. poisson and the projection step of section "Numerical algorithm").
//
// Jacobi-preconditioned CG (Saad, Alg. 9.1) on K p = -V (b - mean), K = -V A the
// 7-point flux-form operator, fused into two passes per iteration:
//   pass A  p_new = z + beta p_old  (z = r / diag, staged with its face halo),
//           q = K p_new, <p_new, q>   -> alpha = <r,z> / <p,q> per sim
//   pass B  x += alpha p, r -= alpha q, <r, z>, <r, r>  -> beta, convergence
// The PCG passes run one CTA per z-slab of a cube (the slab depth is a launch
// parameter); cube constants are read once into shared memory,
// interior rows move as 16-byte vectors, and the dot products are reduced with warp
// shuffles into FP64 per-sim atomics.  The mixed mode runs the same passes on FP32
// vectors inside an FP64 defect-correction loop (FP64 residual, x += e).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bcm_cube.cuh"
#include "bcm_internal.cuh"
#include "bcm_kernels.h"
#include "bcm_persist.cuh"

namespace bcm {

// ===========================================================================
// residual r = rhs - K x of the FP64 iterate x = p, rhs = -V (b - mean).
// FP64 mode: starts the PCG.  Mixed mode: one defect-correction cycle; r goes to
// FP32 as the inner right-hand side and the inner iterate e is zeroed.
// ===========================================================================
template <int B, int NT, class TV, bool MIXED>
__global__ __launch_bounds__(NT) void k_residual(DevGrid g, const double* __restrict__ b,
                                                 const double* __restrict__ x,
                                                 TV* __restrict__ r, float* __restrict__ e,
                                                 SolveParams prm) {
  using SL = Slab<B, B>;
  constexpr int B3 = B * B * B, BB = B * B;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* S = reinterpret_cast<double*>(smem_raw);
  __shared__ CubeSh<double> cs;
  __shared__ double red[4 * 32];
  const int c = blockIdx.x;
  const int s = g.sim[c];
  SimState& st = g.ss[s];
  const bool skip = MIXED ? (st.outer_done != 0) : false;
  double acc4[4] = {0, 0, 0, 0};  // bb, rr64, rz, rr
  if (!skip) {
    load_cube(cs, g, c);
    __syncthreads();
    const size_t base = (size_t)c * B3;
    auto own4 = [&](int q4, int, int, int, double (&v)[4]) { ld4(x + base + 4 * q4, v); };
    auto nbv = [&](int, int n, int cell) { return x[(size_t)n * B3 + cell]; };
    auto valg = [&](int n, int cell) { return x[(size_t)n * B3 + cell]; };
    stage_pressure_cube<B, NT, double>(S, cs, g, c, own4, nbv, valg);
    const double hd = cell_h<B>(g, c), V = hd * hd * hd, mean = st.bmean;
    float rz32 = 0.f, rr32 = 0.f;
    for (int q4 = threadIdx.x; q4 < B3 / 4; q4 += NT) {
      const int cell = 4 * q4, i0 = cell % B, j = (cell / B) % B, k = cell / BB;
      const int o = SL::at(i0, j, k + 1);
      double bv[4];
      ld4(b + base + cell, bv);
      double rv[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const double rhs = -V * (bv[m] - mean);
        rv[m] = rhs - hd * stencil_sum_w<B>(S, o + m, cs, i0 + m, j, k);
        acc4[0] += rhs * rhs;
      }
      if (MIXED) {
        float r32[4], z0[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          r32[m] = float(rv[m]);
          const float z = r32[m] * float(cs.invtab[s3_of<B>(cs.w3, i0 + m, j, k)]);
          rz32 += r32[m] * z;
          rr32 += r32[m] * r32[m];
          acc4[1] += rv[m] * rv[m];
        }
        st4(reinterpret_cast<float*>(r) + base + cell, r32);
        st4(e + base + cell, z0);
      } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const double z = rv[m] * cs.invtab[s3_of<B>(cs.w3, i0 + m, j, k)];
          acc4[2] += rv[m] * z;
          acc4[3] += rv[m] * rv[m];
        }
        st4(reinterpret_cast<double*>(r) + base + cell, rv);
      }
    }
    if (MIXED) {
      acc4[2] = rz32;
      acc4[3] = rr32;
    }
  }
  block_sum<NT, 4>(acc4, red);
  if (threadIdx.x == 0 && !skip) {
    acc_add(st, ACC_BB, acc4[0]);
    if (MIXED) acc_add(st, ACC_RR64, acc4[1]);
    acc_add(st, ACC_RZ, acc4[2]);
    acc_add(st, ACC_RR, acc4[3]);
  }
  if (last_block(g.counter)) {
    int alive = 0, outer_alive = 0;
    for (int q = threadIdx.x; q < g.n_sims; q += NT) {
      SimState& t = g.ss[q];
      const double bb = acc_take(t, ACC_BB), rr64 = acc_take(t, ACC_RR64);
      const double rz = acc_take(t, ACC_RZ), rr = acc_take(t, ACC_RR);
      if (MIXED && t.outer_done) continue;
      if (MIXED) {
        t.cycles += 1;
        if (t.cycles == 1) {
          t.bb = bb;
          t.tol2 = prm.rtol * prm.rtol * bb;
          t.zero_rhs = (bb == 0.0);
        }
        t.rr64 = rr64;
        const bool ok = t.zero_rhs || rr64 <= t.tol2;
        if (!isfinite(rr64)) t.nonfinite = 1;
        if (ok || t.cycles > prm.max_cycles || t.nonfinite) {
          t.outer_done = 1;
          t.done = 1;
          t.converged = ok;
        } else {
          t.rz = rz;
          t.rr = rr;
          // inner target: the reduction eta = inner_rtol per cycle, or, once the
          // reduction rho still needed (||r|| rho = the outer tolerance) is within 4 eta,
          // rho / 2, so the cycle ends the solve instead of overshooting it or stopping
          // just short of it
          const double in2 = prm.inner_rtol * prm.inner_rtol, need2 = 0.25 * t.tol2 / rr64;
          t.inner_tol2 = (16.0 * need2 >= in2 ? need2 : in2) * rr;
          t.iter = 0;
          t.beta = 0.0;
          t.done = (rr == 0.0);
          // reliable update: after the first cycle the inner CG resumes its previous
          // search direction with the true (FP64) residual in place of its own
          t.cont = (prm.recycle && t.cycles > 1) ? 1 : 0;
          alive |= !t.done;
          outer_alive = 1;
        }
      } else {
        t.bb = bb;
        t.tol2 = prm.rtol * prm.rtol * bb;
        t.zero_rhs = (bb == 0.0);
        t.rz = rz;
        t.rr = rr;
        t.rr64 = rr;
        t.iter = 0;
        t.total_iters = 0;
        t.beta = 0.0;
        t.cont = 0;
        if (!isfinite(rr)) t.nonfinite = 1;
        t.done = t.zero_rhs || rr <= t.tol2 || t.nonfinite;
        t.converged = t.zero_rhs || rr <= t.tol2;
        alive |= !t.done;
      }
    }
    // the persistent PCG's rotating dot-product slots start every solve at zero
    for (int i = threadIdx.x; i < g.n_sims * kStripes; i += NT) {
      SimState& t = g.ss[i / kStripes];
      for (int sl = 0; sl < ACC_NSLOT; ++sl) t.acc[i % kStripes][ACC_SLOT_PQ + sl] = 0.0;
      for (int sl = 0; sl < ACC_FZ_SLOTS; ++sl) t.acc[i % kStripes][ACC_SLOT_FZ + sl] = 0.0;
    }
    alive = __syncthreads_or(alive);
    outer_alive = __syncthreads_or(outer_alive);
    if (threadIdx.x == 0) {
      g.flags[0] = !alive;
      g.flags[1] = MIXED ? !outer_alive : 1;
      set_cond(prm.cond_inner, alive ? 1u : 0u);
      if (MIXED) set_cond(prm.cond_outer, outer_alive ? 1u : 0u);
    }
  }
}

// ===========================================================================
// PCG pass A on a z-slab of KS planes of one cube:
//   p_new = z + beta p_old (z = r / diag), q = K p_new, <p_new, q>.
// ===========================================================================
template <int B, int KS, int NT, class TV>
__global__ __launch_bounds__(NT) void k_cg_a(DevGrid g, const TV* __restrict__ r,
                                             const TV* __restrict__ zv,
                                             TV* __restrict__ p0, TV* __restrict__ p1,
                                             TV* __restrict__ q, SolveParams prm) {
  cudaGridDependencySynchronize();  // (multigrid iteration: launched while the V-cycle drains)
  using SL = Slab<B, KS>;
  constexpr int B3 = B * B * B, BB = B * B, NSL = B / KS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TV* S = reinterpret_cast<TV*>(smem_raw);
  __shared__ CubeSh<TV> cs;
  __shared__ double red[32];
  const int c = blockIdx.x / NSL, z0 = (blockIdx.x - c * NSL) * KS;
  SimState& st = g.ss[g.sim[c]];
  TV pq = TV(0);
  const bool active = !st.done;
  if (active) {
    load_cube(cs, g, c);
    const int it = st.iter;
    const TV* __restrict__ pold = (it & 1) ? p1 : p0;
    TV* __restrict__ pnew = (it & 1) ? p0 : p1;
    const TV beta = TV(st.beta);
    const bool first = (it == 0);
    __syncthreads();
    // z = M^-1 r: the multigrid V-cycle's output, or the Jacobi scaling of r
    auto val4 = [&](int cube, int cell0, int face, TV (&v)[4]) {
      const size_t gi = (size_t)cube * B3 + cell0;
      TV rr[4], pp[4] = {TV(0), TV(0), TV(0), TV(0)};
      if (!first) ld4(pold + gi, pp);
      if (zv) {
        ld4(zv + gi, rr);
#pragma unroll
        for (int m = 0; m < 4; ++m) v[m] = first ? rr[m] : rr[m] + beta * pp[m];
        return;
      }
      ld4(r + gi, rr);
      const int* w3 = face < 0 ? cs.w3 : cs.nbw3[face];
      const int k = cell0 / BB, j = (cell0 / B) % B, i0 = cell0 % B;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const TV z = rr[m] * cs.invtab[s3_of<B>(w3, i0 + m, j, k)];
        v[m] = first ? z : z + beta * pp[m];
      }
    };
    auto val1 = [&](int f, int n, int cell) {
      const int i = cell % B, j = (cell / B) % B, k = cell / BB;
      const size_t gi = (size_t)n * B3 + cell;
      const TV z = zv ? zv[gi] : r[gi] * cs.invtab[s3_of<B>(cs.nbw3[f], i, j, k)];
      return first ? z : z + beta * pold[gi];
    };
    auto valg = [&](int n, int cell) {
      const size_t gi = (size_t)n * B3 + cell;
      const TV z = zv ? zv[gi] : r[gi] * inv_diag_any<B, TV>(g, n, cell);
      return first ? z : z + beta * pold[gi];
    };
    stage_pressure_slab<B, KS, NT, TV>(S, cs, g, c, z0, val4, val1, valg);
    const TV h = TV(cell_h<B>(g, c));
    const size_t base = (size_t)c * B3 + (size_t)z0 * BB;
    TV part = TV(0);
    for (int q4 = threadIdx.x; q4 < KS * BB / 4; q4 += NT) {
      const int cell = 4 * q4, kk = cell / BB, j = (cell / B) % B, i0 = cell % B;
      const int o = SL::at(i0, j, kk + 1);
      TV pc[4], qv[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        pc[m] = S[o + m];
        qv[m] = h * stencil_sum_w<B, TV, KS>(S, o + m, cs, i0 + m, j, z0 + kk);
        part += pc[m] * qv[m];
      }
      st4(pnew + base + cell, pc);
      st4(q + base + cell, qv);
    }
    pq = part;
  }
  const TV pp[1] = {pq};
  double vals[1];
  block_sum_tv<NT, 1, TV>(pp, vals, red);
  if (threadIdx.x == 0 && active) acc_add(st, ACC_PQ, vals[0]);
  if (last_block(g.counter)) {
    for (int qq = threadIdx.x; qq < g.n_sims; qq += NT) {
      SimState& t = g.ss[qq];
      const double pqs = acc_take(t, ACC_PQ);
      if (t.done) continue;
      t.alpha = (pqs != 0.0) ? t.rz / pqs : 0.0;
      if (!isfinite(pqs)) {
        t.nonfinite = 1;
        t.alpha = 0.0;
      }
    }
  }
}

// ===========================================================================
// PCG pass B on a z-slab of KS planes (pointwise):
//   x += alpha p, r -= alpha q, z = r / diag, <r,z>, <r,r>;
// then beta, the convergence test and the loop control (last block).
// ===========================================================================
template <int B, int KS, int NT, class TV, class TX>
__global__ __launch_bounds__(NT) void k_cg_b(DevGrid g, TX* __restrict__ x, TV* __restrict__ r,
                                             const TV* __restrict__ p0,
                                             const TV* __restrict__ p1,
                                             const TV* __restrict__ q, SolveParams prm) {
  constexpr int B3 = B * B * B, BB = B * B, NSL = B / KS;
  constexpr int NQ = KS * BB / 4, M = (NQ + NT - 1) / NT;
  __shared__ int w3s[6];
  __shared__ TV invs[kW3];
  __shared__ double red[2 * 32];
  const int c = blockIdx.x / NSL, z0 = (blockIdx.x - c * NSL) * KS;
  const int s = g.sim[c];
  SimState& st = g.ss[s];
  TV sums[2] = {TV(0), TV(0)};
  const bool active = !st.done && !st.nonfinite;
  if (active) {
    if (threadIdx.x < 6) w3s[threadIdx.x] = g.w3[6 * c + threadIdx.x];
    if (threadIdx.x < kW3) invs[threadIdx.x] = TV(g.sp[s].invdiag[g.lvl[c]][threadIdx.x]);
    const TV* __restrict__ pn = (st.iter & 1) ? p0 : p1;
    const TV alpha = TV(st.alpha);
    const size_t base = (size_t)c * B3 + (size_t)z0 * BB;
    __syncthreads();
    TV rz = TV(0), rr = TV(0);
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int q4 = threadIdx.x + m * NT;
      if (q4 < NQ) {
        const int cell = 4 * q4;
        TV xv[4], pv[4], rv[4], qv[4];
        ld4(x + base + cell, xv);
        ld4(pn + base + cell, pv);
        ld4(r + base + cell, rv);
        ld4(q + base + cell, qv);
        const int kk = cell / BB, j = (cell / B) % B, i0 = cell % B;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          xv[e] = xv[e] + alpha * pv[e];
          rv[e] = rv[e] - alpha * qv[e];
          const TV z = rv[e] * invs[s3_of<B>(w3s, i0 + e, j, z0 + kk)];
          rz += rv[e] * z;
          rr += rv[e] * rv[e];
        }
        st4(x + base + cell, xv);
        st4(r + base + cell, rv);
      }
    }
    sums[0] = rz;
    sums[1] = rr;
  }
  double vals[2];
  block_sum_tv<NT, 2, TV>(sums, vals, red);
  if (threadIdx.x == 0 && active) {
    if (!prm.mg) acc_add(st, ACC_RZ, vals[0]);
    acc_add(st, ACC_RR, vals[1]);
  }
  // with the multigrid preconditioner z = M^-1 r comes from the V-cycle that follows,
  // whose last launch takes the decisions below
  if (!prm.mg && last_block(g.counter)) {
    int alive = 0;
    for (int qq = threadIdx.x; qq < g.n_sims; qq += NT) {
      SimState& t = g.ss[qq];
      const double rz = acc_take(t, ACC_RZ), rr = acc_take(t, ACC_RR);
      if (t.done) continue;
      if (t.nonfinite || !isfinite(rr)) {
        t.nonfinite = 1;
        t.done = 1;
        continue;
      }
      t.beta = (t.rz != 0.0) ? rz / t.rz : 0.0;
      t.rz = rz;
      t.rr = rr;
      t.iter += 1;
      t.total_iters += 1;
      const bool inner = prm.mixed != 0;
      const double tol2 = inner ? t.inner_tol2 : t.tol2;
      const bool ok = rr <= tol2;
      if (!inner) {
        t.rr64 = rr;
        t.converged = ok;
      }
      if (ok || t.iter >= (inner ? prm.inner_max_iter : prm.max_iter)) t.done = 1;
      alive |= !t.done;
    }
    alive = __syncthreads_or(alive);
    if (threadIdx.x == 0) {
      g.flags[0] = !alive;
      set_cond(prm.cond_inner, alive ? 1u : 0u);
    }
  }
  // independent guard on a graph loop: a bounded number of body executions (with the
  // multigrid the V-cycle's decisions keep it)
  if (prm.cond_inner && !prm.mg && blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned int n = atomicAdd(prm.guard, 1u) + 1u;
    if (n >= (unsigned int)prm.guard_limit)
      cudaGraphSetConditional((cudaGraphConditionalHandle)prm.cond_inner, 0u);
  }
}

// Mixed mode: x64 += e32 after an inner solve (sims still correcting).
template <int B, int NT>
__global__ __launch_bounds__(NT) void k_add_correction(DevGrid g, double* __restrict__ x,
                                                       const float* __restrict__ e) {
  constexpr int B3 = B * B * B;
  const int c = blockIdx.x;
  if (g.ss[g.sim[c]].outer_done) return;
  const size_t base = (size_t)c * B3;
  for (int q4 = threadIdx.x; q4 < B3 / 4; q4 += NT) {
    double xv[4];
    float ev[4];
    ld4(x + base + 4 * q4, xv);
    ld4(e + base + 4 * q4, ev);
#pragma unroll
    for (int m = 0; m < 4; ++m) xv[m] += double(ev[m]);
    st4(x + base + 4 * q4, xv);
  }
}

// ===========================================================================
// projection: u = u* - dt * (mean of the two face gradients of p) per axis, the
// FP64 divergence check ||b - A p|| / ||b|| (= ||D U^{n+1}|| / ||D U*||) and max |u|.
// ===========================================================================
template <int B, int NT, class T>
__global__ __launch_bounds__(NT) void k_correct(DevGrid g, double* __restrict__ p,
                                                const double* __restrict__ b,
                                                const T* __restrict__ us,
                                                const T* __restrict__ vs,
                                                const T* __restrict__ ws, T* __restrict__ u,
                                                T* __restrict__ v, T* __restrict__ w) {
  using SL = Slab<B, B>;
  constexpr int B3 = B * B * B, BB = B * B;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* S = reinterpret_cast<double*>(smem_raw);
  __shared__ CubeSh<double> cs;
  __shared__ double red[2 * 32];
  const int c = blockIdx.x;
  const int s = g.sim[c];
  const SimParams& sp = g.sp[s];
  SimState& st = g.ss[s];
  const bool zero = st.zero_rhs != 0;
  load_cube(cs, g, c);
  __syncthreads();
  const size_t base = (size_t)c * B3;
  auto own4 = [&](int q4, int, int, int, double (&vv)[4]) {
    if (zero) {
      vv[0] = vv[1] = vv[2] = vv[3] = 0.0;
    } else {
      ld4(p + base + 4 * q4, vv);
    }
  };
  auto nbv = [&](int, int n, int cell) { return zero ? 0.0 : p[(size_t)n * B3 + cell]; };
  auto valg = [&](int n, int cell) { return zero ? 0.0 : p[(size_t)n * B3 + cell]; };
  stage_pressure_cube<B, NT, double>(S, cs, g, c, own4, nbv, valg);
  const double hd = cell_h<B>(g, c);
  const double ih = 1.0 / hd, ih2 = ih * ih;
  const T cdt = T(0.5 * sp.dt);
  const T* stars[3] = {us, vs, ws};
  T* outs[3] = {u, v, w};
  double dn = 0.0, dd = 0.0;
  float umax = 0.f;
  constexpr int off[3] = {1, SL::P, SL::P * SL::P};
  for (int q4 = threadIdx.x; q4 < B3 / 4; q4 += NT) {
    const int cell = 4 * q4, i0 = cell % B, j = (cell / B) % B, k = cell / BB;
    const int o = SL::at(i0, j, k + 1);
    T sv[3][4];
#pragma unroll
    for (int d = 0; d < 3; ++d) ld4(stars[d] + base + cell, sv[d]);
    double bv[4];
    ld4(b + base + cell, bv);
    float m2[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const double pc = S[o + m];
      double lap = 0.0;
      const int ii[3] = {i0 + m, j, k};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        double dm = pc - S[o + m - off[d]], dp = S[o + m + off[d]] - pc;
        if (cs.has21) {  // 2:1 faces: gradient over the distance 0.75 h_c (R7)
          if (ii[d] == 0) dm *= double(cs.wt[2 * d]);
          if (ii[d] == B - 1) dp *= double(cs.wt[2 * d + 1]);
        }
        lap += dp - dm;
        const T nv = sv[d][m] - cdt * T((dm + dp) * ih);
        sv[d][m] = nv;
        m2[m] += float(nv) * float(nv);
      }
      const double res = bv[m] - lap * ih2;  // b - A p
      dn += res * res;
      dd += bv[m] * bv[m];
      umax = fmaxf(umax, sqrtf(m2[m]));
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) st4(outs[d] + base + cell, sv[d]);
    if (zero) {
      const double z4[4] = {0.0, 0.0, 0.0, 0.0};
      st4(p + base + cell, z4);
    }
  }
  double vals[2] = {dn, dd};
  block_sum<NT, 2>(vals, red);
  float um = umax;
  for (int o2 = 16; o2 > 0; o2 >>= 1) um = fmaxf(um, __shfl_xor_sync(0xffffffffu, um, o2));
  if ((threadIdx.x & 31) == 0)
    atomicMax(&st.umax_bits, (unsigned long long)__double_as_longlong(double(um)));
  if (threadIdx.x == 0) {
    acc_add(st, ACC_DIVN, vals[0]);
    acc_add(st, ACC_DIVD, vals[1]);
  }
}

// y = K x (FP64), test path.
template <int B, int NT>
__global__ __launch_bounds__(NT) void k_apply_poisson(DevGrid g, const double* __restrict__ x,
                                                      double* __restrict__ y) {
  using SL = Slab<B, B>;
  constexpr int B3 = B * B * B, BB = B * B;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* S = reinterpret_cast<double*>(smem_raw);
  __shared__ CubeSh<double> cs;
  const int c = blockIdx.x;
  load_cube(cs, g, c);
  __syncthreads();
  const size_t base = (size_t)c * B3;
  auto own4 = [&](int q4, int, int, int, double (&v)[4]) { ld4(x + base + 4 * q4, v); };
  auto nbv = [&](int, int n, int cell) { return x[(size_t)n * B3 + cell]; };
  auto valg = [&](int n, int cell) { return x[(size_t)n * B3 + cell]; };
  stage_pressure_cube<B, NT, double>(S, cs, g, c, own4, nbv, valg);
  const double h = cell_h<B>(g, c);
  for (int q4 = threadIdx.x; q4 < B3 / 4; q4 += NT) {
    const int cell = 4 * q4, i0 = cell % B, j = (cell / B) % B, k = cell / BB;
    const int o = SL::at(i0, j, k + 1);
    double yv[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) yv[m] = h * stencil_sum_w<B>(S, o + m, cs, i0 + m, j, k);
    st4(y + base + cell, yv);
  }
}

// ===========================================================================
// Launchers
// ===========================================================================

template <int B>
constexpr int threads_for() { return B == 16 ? 256 : (B == 8 ? 128 : 64); }

template <class K>
static cudaError_t allow_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define BCM_DISPATCH_B(Bv, ...)                            \
  switch (Bv) {                                            \
    case 4: { constexpr int B = 4; __VA_ARGS__; break; }   \
    case 8: { constexpr int B = 8; __VA_ARGS__; break; }   \
    case 16: { constexpr int B = 16; __VA_ARGS__; break; } \
    default: return cudaErrorInvalidValue;                 \
  }

cudaError_t launch_residual(const Ctx& x, const SolveParams& prm) {
  BCM_DISPATCH_B(x.B, {
    constexpr int NT = threads_for<B>();
    const size_t sm = sizeof(double) * Slab<B, B>::N;
    if (x.solve64) {
      auto kern = k_residual<B, NT, double, false>;
      cudaError_t e = allow_smem(kern, sm);
      if (e != cudaSuccess) return e;
      kern<<<x.g.n_cubes, NT, sm, x.stream>>>(x.g, x.f.b, x.f.p, (double*)x.f.r, nullptr, prm);
    } else {
      auto kern = k_residual<B, NT, float, true>;
      cudaError_t e = allow_smem(kern, sm);
      if (e != cudaSuccess) return e;
      kern<<<x.g.n_cubes, NT, sm, x.stream>>>(x.g, x.f.b, x.f.p, (float*)x.f.r, x.f.e, prm);
    }
  });
  return cudaGetLastError();
}

// z-slab depth KS = B / ns (ns = slabs per cube: 1, 2 or 4)
#define BCM_DISPATCH_KS(ns, ...)                             \
  switch (ns) {                                              \
    case 1: { constexpr int KS = B; __VA_ARGS__; break; }     \
    case 2: { constexpr int KS = B / 2; __VA_ARGS__; break; } \
    case 4: { constexpr int KS = B / 4; __VA_ARGS__; break; } \
    default: return cudaErrorInvalidValue;                   \
  }

template <class TV>
static cudaError_t cg_a_t(const Ctx& x, const SolveParams& prm) {
  BCM_DISPATCH_B(x.B, {
    BCM_DISPATCH_KS(x.slabs_a, {
      constexpr int NT = threads_for<B>();
      const size_t sm = sizeof(TV) * Slab<B, KS>::N;
      auto ka = k_cg_a<B, KS, NT, TV>;
      cudaError_t e = allow_smem(ka, sm);
      if (e != cudaSuccess) return e;
      const TV* zv = prm.mg ? (const TV*)x.mg.y[0] : nullptr;
      if (prm.mg) {  // after the V-cycle's last launch: start while it drains
        e = launch_pdl(ka, dim3(x.g.n_cubes * (B / KS)), dim3(NT), sm, x.stream, x.g,
                       (const TV*)x.f.r, zv, (TV*)x.f.p0, (TV*)x.f.p1, (TV*)x.f.q, prm);
        if (e != cudaSuccess) return e;
      } else {
        ka<<<x.g.n_cubes * (B / KS), NT, sm, x.stream>>>(x.g, (const TV*)x.f.r, zv,
                                                         (TV*)x.f.p0, (TV*)x.f.p1, (TV*)x.f.q,
                                                         prm);
      }
    });
  });
  return cudaGetLastError();
}
template <class TV, class TX>
static cudaError_t cg_b_t(const Ctx& x, const SolveParams& prm, TX* xv) {
  BCM_DISPATCH_B(x.B, {
    BCM_DISPATCH_KS(x.slabs_b, {
      constexpr int NT = threads_for<B>();
      k_cg_b<B, KS, NT, TV, TX><<<x.g.n_cubes * (B / KS), NT, 0, x.stream>>>(
          x.g, xv, (TV*)x.f.r, (const TV*)x.f.p0, (const TV*)x.f.p1, (const TV*)x.f.q, prm);
    });
  });
  return cudaGetLastError();
}
cudaError_t launch_cg_a(const Ctx& x, const SolveParams& prm) {
  return x.solve64 ? cg_a_t<double>(x, prm) : cg_a_t<float>(x, prm);
}
cudaError_t launch_cg_b(const Ctx& x, const SolveParams& prm) {
  return x.solve64 ? cg_b_t<double, double>(x, prm, x.f.p) : cg_b_t<float, float>(x, prm, x.f.e);
}

cudaError_t launch_add_correction(const Ctx& x) {
  BCM_DISPATCH_B(x.B, {
    constexpr int NT = threads_for<B>();
    k_add_correction<B, NT><<<x.g.n_cubes, NT, 0, x.stream>>>(x.g, x.f.p, x.f.e);
  });
  return cudaGetLastError();
}

template <class T>
static cudaError_t correct_t(const Ctx& x) {
  BCM_DISPATCH_B(x.B, {
    constexpr int NT = threads_for<B>();
    const size_t sm = sizeof(double) * Slab<B, B>::N;
    auto kern = k_correct<B, NT, T>;
    cudaError_t e = allow_smem(kern, sm);
    if (e != cudaSuccess) return e;
    kern<<<x.g.n_cubes, NT, sm, x.stream>>>(x.g, x.f.p, x.f.b, (const T*)x.f.us,
                                            (const T*)x.f.vs, (const T*)x.f.ws, (T*)x.f.u,
                                            (T*)x.f.v, (T*)x.f.w);
  });
  return cudaGetLastError();
}
cudaError_t launch_correct(const Ctx& x) {
  return x.f64 ? correct_t<double>(x) : correct_t<float>(x);
}

cudaError_t launch_apply_poisson(const Ctx& x, const double* in, double* out) {
  BCM_DISPATCH_B(x.B, {
    constexpr int NT = threads_for<B>();
    const size_t sm = sizeof(double) * Slab<B, B>::N;
    auto kern = k_apply_poisson<B, NT>;
    cudaError_t e = allow_smem(kern, sm);
    if (e != cudaSuccess) return e;
    kern<<<x.g.n_cubes, NT, sm, x.stream>>>(x.g, in, out);
  });
  return cudaGetLastError();
}

}  // namespace bcm
