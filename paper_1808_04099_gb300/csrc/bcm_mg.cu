// bcm_mg.cu -- geometric multigrid V-cycle, the preconditioner M^-1 of the pressure PCG
// (Eq. poisson; the paper solves the pressure equation with a multigrid on its cubes).
//
// Grids of one or two levels.  Per-cube levels l = 0 .. L coarsen every cube by two per
// level (B, B/2, ..., 1 cells per edge); a level-l+1 cell covers 2x2x2 cells of level l
// of the same cube.  Above level L (one cell per cube) the eight refined cubes of each
// level-0 position first join into one node, then the nodes of a sim are aggregated by
// their level-0 cube coordinates shifted right by m (m = 1 .. M).  Transfers are
// piecewise constant, restriction sums, and the coarse operators are the Galerkin
// products P^T K P.  For the flux-form K these are again flux-form operators: on
// per-cube level l a face carries 4^l fine faces, coefficient 4^l h of its cube, an
// outflow face twice that on the diagonal, other domain faces nothing, and a 2:1 face
// keeps the form of R7 (a coarse face cell against the four fine cells that touch it,
// weight 4/3 on the coarse side and 2/3 on the fine side, since the 2x2x2 aggregates on
// both sides keep the coarse cell / four fine cells pairing); the aggregate levels keep
// their Galerkin sums as small CSR tables built on the host.  The smoother is damped Jacobi
// S = omega D^-1 (omega = 0.8), one sweep before and one after the coarse correction,
// which is scaled by s = 1.75 (piecewise-constant transfers leave it too weak), so the
// V-cycle is symmetric positive definite and M^-1 suits CG:
//   V_l(r) = x + S (r - K x),  x = S r + s P V_{l+1}(P^T (r - K S r)),
//   V_top(r) = four damped-Jacobi sweeps from zero.
//
// Launches per V-cycle: one per per-cube level on the way down (pre-smoothing with the
// neighbours' values computed on the fly, residual, restriction), one single-block
// launch for the aggregate levels, and one per per-cube level on the way up
// (prolongation of the neighbours on the fly, post-smoothing).  The last launch also
// forms <r, z> per sim and, after PCG pass B, takes the iteration's decisions (beta,
// convergence) that pass B leaves to it.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bcm_cube.cuh"
#include "bcm_internal.cuh"
#include "bcm_kernels.h"
#include "bcm_persist.cuh"

namespace bcm {

template <int BL>
__device__ __forceinline__ int lcell(int i, int j, int k) { return (k * BL + j) * BL + i; }

// Per-sim constants of a level in the vector type: the FP32 path does no FP64
// arithmetic (FP64 runs at a small fraction of the FP32 rate on this GPU).
template <class TV>
__device__ __forceinline__ TV sim_inv(const SimParams& sp, int lvl, int s3);
template <>
__device__ __forceinline__ float sim_inv<float>(const SimParams& sp, int lvl, int s3) {
  return sp.invdiag32[lvl][s3];
}
template <>
__device__ __forceinline__ double sim_inv<double>(const SimParams& sp, int lvl, int s3) {
  return sp.invdiag[lvl][s3];
}
template <class TV>
__device__ __forceinline__ TV sim_h(const SimParams& sp);
template <>
__device__ __forceinline__ float sim_h<float>(const SimParams& sp) { return sp.h032; }
template <>
__device__ __forceinline__ double sim_h<double>(const SimParams& sp) { return sp.h0; }
// cell size of cube c (its refinement level halves the sim's level-0 size)
template <class TV>
__device__ __forceinline__ TV cube_h(const DevGrid& g, const SimParams& sp, int c) {
  return g.lvl[c] ? TV(0.5) * sim_h<TV>(sp) : sim_h<TV>(sp);
}

// The value across face f of cell (i, j, k) of cube c on per-cube level l (BL cells per
// edge) and the weight w of that face in the level's flux-form operator, whose
// coefficient 4^l h the caller carries (R7 on the coarser cells; the Galerkin product of
// the finer level keeps that form): a cell of this cube or of a same-level neighbour
// (w = 1), a domain ghost (w = 1; the cell itself, or minus it at an outflow face), the
// coarse cell across a 2:1 face (w = 2/3), or the mean of the four fine cells across it
// (w = 4/3).  val(cube, i, j, k) is a cell's value, xc this cell's.
template <int BL, class TV, class Val>
__device__ __forceinline__ TV mg_across(const DevGrid& g, int c, int l, int i, int j, int k,
                                        int f, TV xc, const Val& val, TV& w) {
  const int d = f >> 1, side = f & 1;
  int q[3] = {i, j, k};
  q[d] += side ? 1 : -1;
  w = TV(1);
  if (q[d] >= 0 && q[d] < BL) return val(c, q[0], q[1], q[2]);
  const int n = checked_nb(g, g.nb[6 * c + f]);
  if (n >= 0) {
    q[d] = side ? 0 : BL - 1;
    return val(n, q[0], q[1], q[2]);
  }
  if (n == NB_BOUNDARY) return g.sp[g.sim[c]].bc[f] == BC_OUTFLOW ? -xc : xc;
  const int t1 = tan1(d), t2 = tan2(d);
  const int a = t1 == 0 ? i : (t1 == 1 ? j : k), b = t2 == 0 ? i : (t2 == 1 ? j : k);
  int r3[3];
  r3[d] = side ? 0 : BL - 1;  // the cells across lie on the neighbour's facing layer
  if (n == NB_COARSE) {
    w = TV(2.0 / 3.0);
    const int C = g.aux[(6 * c + f) * 4];
    if (!bcm_expect(g, C >= 0 && C < g.n_cubes, CHK_AUX)) return xc;
    // corner coordinates in finest-cell units; a level-l cell spans 2^l level-0 cells
    const int sf = (1 << (g.max_level - g.lvl[c])) << l;
    const int sc = (1 << (g.max_level - g.lvl[C])) << l;
    r3[t1] = (g.ijk[3 * c + t1] + a * sf - g.ijk[3 * C + t1]) / sc;
    r3[t2] = (g.ijk[3 * c + t2] + b * sf - g.ijk[3 * C + t2]) / sc;
    if (!bcm_expect(g, r3[t1] >= 0 && r3[t1] < BL && r3[t2] >= 0 && r3[t2] < BL, CHK_CELL))
      return xc;
    return val(C, r3[0], r3[1], r3[2]);
  }
  w = TV(4.0 / 3.0);  // NB_FINE: the four fine cells that touch this coarse cell's face
  TV sum = TV(0);
#pragma unroll
  for (int bb = 0; bb < 2; ++bb)
#pragma unroll
    for (int aa = 0; aa < 2; ++aa) {
      const int ta = 2 * a + aa, tb = 2 * b + bb, qa = ta / BL, qb = tb / BL;
      const int F = g.aux[(6 * c + f) * 4 + qb * 2 + qa];
      if (!bcm_expect(g, F >= 0 && F < g.n_cubes && qa < 2 && qb < 2, CHK_AUX)) return xc;
      r3[t1] = ta - qa * BL;
      r3[t2] = tb - qb * BL;
      sum += val(F, r3[0], r3[1], r3[2]);
    }
  return TV(0.25) * sum;
}

// omega / diag(K_l) of cell (i, j, k) of cube c on per-cube level l (BL cells per edge):
// diag(K_l) = 4^l diag(K) of a fine cell with the same boundary faces; wscale =
// omega / 4^l.  Neighbouring cubes belong to the same sim, so sp serves them too.
template <int BL, class TV>
__device__ __forceinline__ TV smooth_w(const DevGrid& g, const SimParams& sp, int c, int i, int j,
                                       int k, TV wscale) {
  return wscale * sim_inv<TV>(sp, g.lvl[c], s3_of<BL>(g.w3 + 6 * c, i, j, k));
}

// ---- down: x = S r, rr = r - K x, restriction of rr (P^T: sums)
// One thread per coarse cell (its 2x2x2 fine cells), or per cube on the level with one
// cell per cube (its residual goes to `rc` per cube for the aggregate levels).
template <int BL, class TV>
__device__ __forceinline__ void mg_down_item(const DevGrid& g, int l, TV wscale, TV cscale,
                                             const TV* __restrict__ r, TV* __restrict__ x,
                                             TV* __restrict__ rc, int all, long long t) {
  constexpr int CB = BL > 1 ? BL / 2 : 1, C3 = CB * CB * CB, B3 = BL * BL * BL;
  constexpr int CH = BL > 1 ? 2 : 1;
  const int c = (int)(t / C3), ci = (int)(t - (long long)c * C3);
  const int s = g.sim[c];
  if (!all && g.ss[s].done) return;
  const int I = ci % CB, J = (ci / CB) % CB, Kc = ci / (CB * CB);
  const SimParams& sp = g.sp[s];
  const TV coef = cube_h<TV>(g, sp, c) * cscale;  // 4^l h
  auto sval = [&](int cube, int ci2, int cj2, int ck2) {
    return smooth_w<BL, TV>(g, sp, cube, ci2, cj2, ck2, wscale) *
           r[(size_t)cube * B3 + lcell<BL>(ci2, cj2, ck2)];
  };
  TV sum = TV(0);
#pragma unroll
  for (int dk = 0; dk < CH; ++dk)
#pragma unroll
    for (int dj = 0; dj < CH; ++dj)
#pragma unroll
      for (int di = 0; di < CH; ++di) {
        const int i = CH * I + di, j = CH * J + dj, k = CH * Kc + dk;
        const size_t gi = (size_t)c * B3 + lcell<BL>(i, j, k);
        const TV rv = r[gi];
        const TV xc = smooth_w<BL, TV>(g, sp, c, i, j, k, wscale) * rv;
        TV acc = TV(0);
#pragma unroll
        for (int f = 0; f < 6; ++f) {
          TV w;
          const TV xn = mg_across<BL, TV>(g, c, l, i, j, k, f, xc, sval, w);
          acc += w * (xc - xn);
        }
        x[gi] = xc;
        sum += rv - coef * acc;
      }
  rc[t] = sum;
}

template <int BL, class TV>
__global__ __launch_bounds__(256) void k_mg_down(DevGrid g, int l, TV wscale, TV cscale,
                                                 const TV* __restrict__ r,
                                                 TV* __restrict__ x, TV* __restrict__ rc,
                                                 int all) {
  cudaGridDependencySynchronize();  // launched after the previous level's kernel
  constexpr int CB = BL > 1 ? BL / 2 : 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)g.n_cubes * CB * CB * CB) return;
  mg_down_item<BL, TV>(g, l, wscale, cscale, r, x, rc, all, t);
}

// The same with one thread per fine cell (BL >= 2): the eight children of a coarse cell
// are eight consecutive threads of one warp (child bits in the low three bits of the
// thread index), so the restriction is a three-step shuffle sum.  Threads of finished
// sims and of the tail take part in the shuffles with zeros.
template <int BL, class TV>
__global__ __launch_bounds__(256) void k_mg_down_cell(DevGrid g, int l, TV wscale, TV cscale,
                                                      const TV* __restrict__ r,
                                                      TV* __restrict__ x, TV* __restrict__ rc,
                                                      int all) {
  cudaGridDependencySynchronize();  // launched after the previous level's kernel
  static_assert(BL >= 2, "restriction over 2x2x2 children");
  constexpr int CB = BL / 2, C3 = CB * CB * CB, B3 = BL * BL * BL;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)g.n_cubes * B3;
  const int c = (int)(t / B3), q = (int)(t - (long long)c * B3);
  const int d = q & 7, ci = q >> 3;
  TV val = TV(0);
  if (t < total && (all || !g.ss[g.sim[c]].done)) {
    const int I = ci % CB, J = (ci / CB) % CB, Kc = ci / (CB * CB);
    const int i = 2 * I + (d & 1), j = 2 * J + ((d >> 1) & 1), k = 2 * Kc + (d >> 2);
    const SimParams& sp = g.sp[g.sim[c]];
    const TV coef = cube_h<TV>(g, sp, c) * cscale;
    const size_t gi = (size_t)c * B3 + lcell<BL>(i, j, k);
    const TV rv = r[gi];
    const TV xc = smooth_w<BL, TV>(g, sp, c, i, j, k, wscale) * rv;
    auto sval = [&](int cube, int ci2, int cj2, int ck2) {
      return smooth_w<BL, TV>(g, sp, cube, ci2, cj2, ck2, wscale) *
             r[(size_t)cube * B3 + lcell<BL>(ci2, cj2, ck2)];
    };
    TV acc = TV(0);
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      TV w;
      const TV xn = mg_across<BL, TV>(g, c, l, i, j, k, f, xc, sval, w);
      acc += w * (xc - xn);
    }
    x[gi] = xc;
    val = rv - coef * acc;
  }
  val += __shfl_xor_sync(0xffffffffu, val, 1);
  val += __shfl_xor_sync(0xffffffffu, val, 2);
  val += __shfl_xor_sync(0xffffffffu, val, 4);
  if (d == 0 && t < total && (all || !g.ss[g.sim[c]].done)) rc[(size_t)c * C3 + ci] = val;
}

// ---- up: x~ = x + P y_coarse (on the fly for the cell and its neighbours), then
// y = x~ + S (r - K x~).  One thread per cell.  On the level with one cell per cube the
// coarse values come from aggregate level 0 (FP64, through the cube's parent).
template <int BL, class TV>
__device__ __forceinline__ TV up_value(const TV* __restrict__ x, const TV* __restrict__ yc,
                                       const double* __restrict__ yagg,
                                       const int* __restrict__ agg_parent, int c, int i, int j,
                                       int k) {
  constexpr int B3 = BL * BL * BL;
  const TV xv = x[(size_t)c * B3 + lcell<BL>(i, j, k)];
  if constexpr (BL == 1) {
    return xv + TV(kMgOver * yagg[agg_parent[c]]);
  } else {
    constexpr int CB = BL / 2;
    return xv + TV(kMgOver) * yc[(size_t)c * CB * CB * CB + lcell<CB>(i >> 1, j >> 1, k >> 1)];
  }
}

template <int BL, class TV>
__device__ __forceinline__ TV up_cell(const DevGrid& g, int l, TV wscale, TV cscale,
                                      const TV* __restrict__ r,
                                      const TV* __restrict__ x, const TV* __restrict__ yc,
                                      const double* __restrict__ yagg,
                                      const int* __restrict__ agg_parent, int c, int i, int j,
                                      int k, TV* rv_out) {
  constexpr int B3 = BL * BL * BL;
  const SimParams& sp = g.sp[g.sim[c]];
  const TV coef = cube_h<TV>(g, sp, c) * cscale;
  const TV xc = up_value<BL, TV>(x, yc, yagg, agg_parent, c, i, j, k);
  auto uval = [&](int cube, int ci2, int cj2, int ck2) {
    return up_value<BL, TV>(x, yc, yagg, agg_parent, cube, ci2, cj2, ck2);
  };
  TV acc = TV(0);
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    TV w;
    const TV xn = mg_across<BL, TV>(g, c, l, i, j, k, f, xc, uval, w);
    acc += w * (xc - xn);
  }
  const TV rv = r[(size_t)c * B3 + lcell<BL>(i, j, k)];
  *rv_out = rv;
  return xc + smooth_w<BL, TV>(g, sp, c, i, j, k, wscale) * (rv - coef * acc);
}

template <int BL, class TV>
__device__ __forceinline__ void mg_up_item(const DevGrid& g, int l, TV wscale, TV cscale,
                                           const TV* __restrict__ r, const TV* __restrict__ x,
                                           const TV* __restrict__ yc,
                                           const double* __restrict__ yagg,
                                           const int* __restrict__ agg_parent,
                                           TV* __restrict__ y, int all, long long t) {
  constexpr int B3 = BL * BL * BL;
  const int c = (int)(t / B3), cell = (int)(t - (long long)c * B3);
  if (!all && g.ss[g.sim[c]].done) return;
  const int i = cell % BL, j = (cell / BL) % BL, k = cell / (BL * BL);
  TV rv;
  y[t] = up_cell<BL, TV>(g, l, wscale, cscale, r, x, yc, yagg, agg_parent, c, i, j, k, &rv);
}

template <int BL, class TV>
__global__ __launch_bounds__(256) void k_mg_up(DevGrid g, int l, TV wscale, TV cscale,
                                               const TV* __restrict__ r,
                                               const TV* __restrict__ x,
                                               const TV* __restrict__ yc,
                                               const double* __restrict__ yagg,
                                               const int* __restrict__ agg_parent,
                                               TV* __restrict__ y, int all) {
  cudaGridDependencySynchronize();  // launched after the previous level's kernel
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)g.n_cubes * BL * BL * BL) return;
  mg_up_item<BL, TV>(g, l, wscale, cscale, r, x, yc, yagg, agg_parent, y, all, t);
}

// The last block of the finest up launch: mode 0 (start of a solve) takes <r, z> as
// the PCG's rz; mode 1 (after pass B) forms beta, counts the iteration and tests
// convergence on the <r, r> that pass B accumulated.
__device__ void mg_decide(const DevGrid& g, const SolveParams& prm, int mode, int nt) {
  int alive = 0;
  for (int q = threadIdx.x; q < g.n_sims; q += nt) {
    SimState& t = g.ss[q];
    const double rzs = acc_take(t, ACC_RZ);
    if (mode == 0) {
      if (!t.done) t.rz = rzs;
      alive |= !t.done;
      continue;
    }
    const double rr = acc_take(t, ACC_RR);
    if (t.done) continue;
    if (t.nonfinite || !isfinite(rr) || !isfinite(rzs)) {
      t.nonfinite = 1;
      t.done = 1;
      continue;
    }
    t.beta = (t.rz != 0.0) ? rzs / t.rz : 0.0;
    t.rz = rzs;
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
    if (mode == 1) g.flags[0] = !alive;
    // a captured step: this launch ends the inner loop's body (mode 1) or starts an
    // inner solve (mode 0) and sets the loop's condition; mode 1 also keeps the guard
    // on the number of body executions
    if (prm.cond_inner) {
      unsigned int go = alive ? 1u : 0u;
      if (mode == 1 && atomicAdd(prm.guard, 1u) + 1u >= (unsigned int)prm.guard_limit) go = 0u;
      set_cond(prm.cond_inner, go);
      if (prm.body_count) atomicAdd(prm.body_count + (mode == 1 ? 0 : 1), 1u);
    }
  }
}

// ---- up on the finest level: z = y_0, <r, z> per sim, and the PCG's decisions.
// Blocks of NT = min(256, B^3) threads lie inside one cube, hence one sim.
template <int B, int NT, class TV>
__global__ __launch_bounds__(NT) void k_mg_up0(DevGrid g, const TV* __restrict__ r,
                                              const TV* __restrict__ x,
                                              const TV* __restrict__ yc,
                                              const double* __restrict__ yagg,
                                              const int* __restrict__ agg_parent,
                                              TV* __restrict__ z, SolveParams prm, int mode) {
  cudaGridDependencySynchronize();  // launched after the previous level's kernel
  constexpr int B3 = B * B * B, PER = B3 / NT;
  __shared__ double red[32];
  const int c = blockIdx.x / PER;
  const int s = g.sim[c];
  SimState& st = g.ss[s];
  const bool all = mode == 2;
  const bool active = all || !st.done;
  double rz = 0.0;
  if (active) {
    const int cell = (blockIdx.x - c * PER) * NT + threadIdx.x;
    const int i = cell % B, j = (cell / B) % B, k = cell / (B * B);
    TV rv;
    const TV zv = up_cell<B, TV>(g, 0, TV(kMgOmega), TV(1), r, x, yc, yagg, agg_parent, c, i, j,
                                 k, &rv);
    z[(size_t)c * B3 + cell] = zv;
    rz = double(rv * zv);
  }
  if (all) return;
  double vals[1] = {rz};
  block_sum<NT, 1>(vals, red);
  if (threadIdx.x == 0 && active) acc_add(st, ACC_RZ, vals[0]);
  if (last_block(g.counter)) mg_decide(g, prm, mode, NT);
}

// ---- levels of 8^3 / 16^3 cells per cube, one block per cube with the (B+2)^3 tile of
// the PCG passes: down stages x = S r with the face halo, marches each column for
// rr = r - K x and sums the 2x2x2 children of rr into r_{l+1}; up stages
// x~ = x + s P y_{l+1}, marches for y = x~ + S (r - K x~) and, on the finest level, forms
// <r, z>.  On level l, S = (omega / 4^l) D^-1 and K = 4^l h (sum of differences) with
// the finest level's D: the launch passes wl = omega / 4^l and cl = 4^l.  Same values as
// the per-cell kernels above.
//
// With FB the down launch also does the PCG's pass B (x_pcg += alpha p, r -= alpha q,
// <r, r>): it reads the residual r_in of the iteration and writes the new one to the
// other buffer r_out (blocks read their neighbours' r_in for the halo, so it is not
// updated in place), forming the halo's new residual on the fly.  The buffers swap
// with the parity of the sim's iteration count.
template <class TV>
struct PassB {
  TV* x;                 // PCG iterate
  const TV *p0, *p1, *q; // search directions (by iteration parity), q = K p
  TV *ra, *rb;           // residual: in ra, out rb at even iterations; swapped at odd
};

template <int B, class TV, bool FB>
__global__ __launch_bounds__(B * B) void k_mg_down0_tile(DevGrid g, const TV* __restrict__ r0,
                                                         TV* __restrict__ x,
                                                         TV* __restrict__ r1, int all,
                                                         PassB<TV> pb, TV wl, TV cl, int lsh) {
  cudaGridDependencySynchronize();  // launched after the previous level's kernel
  using SL = Slab<B, B>;
  constexpr int NT = B * B, B3 = B * B * B, BB = B * B, PP = SL::P * SL::P, CB = B / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TV* S = reinterpret_cast<TV*>(smem_raw);
  TV* RR = S + (SL::N + 3) / 4 * 4;
  __shared__ CubeSh<TV> cs;
  __shared__ double red[32];
  const int c = blockIdx.x;
  SimState& st = g.ss[g.sim[c]];
  if (!all && st.done) return;
  load_cube(cs, g, c);
  const TV* __restrict__ r = r0;
  TV* __restrict__ rout = nullptr;
  const TV* __restrict__ pn = nullptr;
  TV alpha = TV(0);
  if constexpr (FB) {
    const int it = st.iter;
    r = (it & 1) ? pb.rb : pb.ra;
    rout = (it & 1) ? pb.ra : pb.rb;
    pn = (it & 1) ? pb.p0 : pb.p1;
    alpha = st.nonfinite ? TV(0) : TV(st.alpha);
  }
  __syncthreads();
  const TV w = wl;
  TV rr2 = TV(0);
  // the iteration's residual of a cell: r (FB: r_in - alpha q)
  auto res = [&](size_t gi) {
    if constexpr (FB) return r[gi] - alpha * pb.q[gi];
    else return r[gi];
  };
  auto val4 = [&](int cube, int cell0, int face, TV (&v)[4]) {
    const size_t gi = (size_t)cube * B3 + cell0;
    TV rr[4];
    ld4(r + gi, rr);
    if constexpr (FB) {
      TV qv[4];
      ld4(pb.q + gi, qv);
#pragma unroll
      for (int m = 0; m < 4; ++m) rr[m] = rr[m] - alpha * qv[m];
      if (face < 0) {  // own cells: pass B
        TV xv[4], pv[4];
        ld4(pb.x + gi, xv);
        ld4(pn + gi, pv);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          xv[m] = xv[m] + alpha * pv[m];
          rr2 += rr[m] * rr[m];
          RR[cell0 + m] = rr[m];
        }
        st4(pb.x + gi, xv);
        st4(rout + gi, rr);
      }
    }
    const int mask = face < 0 ? cs.smask : cs.nbmask[face];
    const int* w3 = face < 0 ? cs.w3 : cs.nbw3[face];
    const int kz = cell0 / BB, j = (cell0 / B) % B, i0 = cell0 % B;
#pragma unroll
    for (int m = 0; m < 4; ++m)
      v[m] = w * rr[m] * (mask == 0 ? cs.invtab[18] : cs.invtab[s3_of<B>(w3, i0 + m, j, kz)]);
  };
  auto val1 = [&](int f, int n, int cell) {
    const TV inv = cs.nbmask[f] == 0
                       ? cs.invtab[18]
                       : cs.invtab[s3_of<B>(cs.nbw3[f], cell % B, (cell / B) % B, cell / BB)];
    return w * res((size_t)n * B3 + cell) * inv;
  };
  auto valg = [&](int n, int cell) {
    return w * res((size_t)n * B3 + cell) * inv_diag_any<B, TV>(g, n, cell);
  };
  stage_pressure_slab<B, B, NT, TV>(S, cs, g, c, 0, val4, val1, valg, lsh);
  const TV h = cube_h<TV>(g, g.sp[g.sim[c]], c) * cl;
  const int i = threadIdx.x % B, j = column_row<B>(threadIdx.x);
  int o = SL::at(i, j, 1);
  TV below = S[o - PP], cur = S[o];
#pragma unroll 4
  for (int kk = 0; kk < B; ++kk) {
    const TV above = S[o + PP];
    TV acc = (cur - S[o - 1]) + (cur - S[o + 1]) + (cur - S[o - SL::P]) +
             (cur - S[o + SL::P]) + (cur - below) + (cur - above);
    if (cs.has21) acc = stencil_sum_w<B, TV, B>(S, o, cs, i, j, kk);
    const int cell = (kk * B + j) * B + i;
    const size_t gi = (size_t)c * B3 + cell;
    x[gi] = cur;
    // FB: RR holds the cell's new residual, stored during the staging
    RR[cell] = (FB ? RR[cell] : r[gi]) - h * acc;
    below = cur;
    cur = above;
    o += PP;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < CB * CB * CB; q += NT) {
    const int I = q % CB, J = (q / CB) % CB, K = q / (CB * CB);
    TV sum = TV(0);
#pragma unroll
    for (int d = 0; d < 8; ++d)
      sum += RR[((2 * K + (d >> 2)) * B + 2 * J + ((d >> 1) & 1)) * B + 2 * I + (d & 1)];
    r1[(size_t)c * CB * CB * CB + q] = sum;
  }
  if constexpr (FB) {
    double vals[1] = {double(rr2)};
    block_sum<NT, 1>(vals, red);
    if (threadIdx.x == 0) acc_add(st, ACC_RR, vals[0]);
  }
}

template <int B, class TV>
__global__ __launch_bounds__(B * B) void k_mg_up0_tile(DevGrid g, const TV* __restrict__ ra,
                                                       const TV* __restrict__ rb,
                                                       const TV* __restrict__ x,
                                                       const TV* __restrict__ y1,
                                                       TV* __restrict__ z, SolveParams prm,
                                                       int mode, TV wl, TV cl, int finest,
                                                       int lsh) {
  cudaGridDependencySynchronize();  // launched after the previous level's kernel
  using SL = Slab<B, B>;
  constexpr int NT = B * B, B3 = B * B * B, BB = B * B, PP = SL::P * SL::P, CB = B / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TV* S = reinterpret_cast<TV*>(smem_raw);
  __shared__ CubeSh<TV> cs;
  __shared__ double red[32];
  const int c = blockIdx.x, s = g.sim[c];
  SimState& st = g.ss[s];
  const bool all = mode == 2;
  const bool active = all || !st.done;
  // after a down launch with pass B (rb set) the new residual is in the buffer that
  // the iteration's parity selects, else in ra
  const TV* __restrict__ r = (mode == 1 && rb && !(st.iter & 1)) ? rb : ra;
  double rz = 0.0;
  if (active) {
    load_cube(cs, g, c);
    __syncthreads();
    auto xt = [&](int cube, int cell) {
      const int i = cell % B, j = (cell / B) % B, k = cell / BB;
      return x[(size_t)cube * B3 + cell] +
             TV(kMgOver) *
                 y1[(size_t)cube * CB * CB * CB + ((k >> 1) * CB + (j >> 1)) * CB + (i >> 1)];
    };
    auto val4 = [&](int cube, int cell0, int, TV (&v)[4]) {
      TV xv[4];
      ld4(x + (size_t)cube * B3 + cell0, xv);
      const int kz = cell0 / BB, j = (cell0 / B) % B, i0 = cell0 % B;
      const size_t pb = (size_t)cube * CB * CB * CB + ((kz >> 1) * CB + (j >> 1)) * CB + (i0 >> 1);
      const TV ya = TV(kMgOver) * y1[pb], yb = TV(kMgOver) * y1[pb + 1];
      v[0] = xv[0] + ya;
      v[1] = xv[1] + ya;
      v[2] = xv[2] + yb;
      v[3] = xv[3] + yb;
    };
    auto val1 = [&](int, int n, int cell) { return xt(n, cell); };
    auto valg = [&](int n, int cell) { return xt(n, cell); };
    stage_pressure_slab<B, B, NT, TV>(S, cs, g, c, 0, val4, val1, valg, lsh);
    const TV h = cube_h<TV>(g, g.sp[s], c) * cl, w = wl;
    const int i = threadIdx.x % B, j = column_row<B>(threadIdx.x);
    int o = SL::at(i, j, 1);
    TV below = S[o - PP], cur = S[o];
    TV part = TV(0);
#pragma unroll 4
    for (int kk = 0; kk < B; ++kk) {
      const TV above = S[o + PP];
      TV acc = (cur - S[o - 1]) + (cur - S[o + 1]) + (cur - S[o - SL::P]) +
               (cur - S[o + SL::P]) + (cur - below) + (cur - above);
      if (cs.has21) acc = stencil_sum_w<B, TV, B>(S, o, cs, i, j, kk);
      const size_t gi = (size_t)c * B3 + (kk * B + j) * B + i;
      const TV inv = cs.smask == 0 ? cs.invtab[18] : cs.invtab[s3_of<B>(cs.w3, i, j, kk)];
      const TV rv = r[gi];
      const TV zv = cur + w * inv * (rv - h * acc);
      z[gi] = zv;
      part += rv * zv;
      below = cur;
      cur = above;
      o += PP;
    }
    rz = double(part);
  }
  if (all || !finest) return;
  double vals[1] = {rz};
  block_sum<NT, 1>(vals, red);
  if (threadIdx.x == 0 && active) acc_add(st, ACC_RZ, vals[0]);
  if (last_block(g.counter)) mg_decide(g, prm, mode, NT);
}

// ---- the aggregate levels, in one block: gather of the cubes' residuals, the V-cycle
// on the CSR levels k = 0 .. M-1 (k = M-1 the top), result y = ax[0].  The work is a
// chain of small dependent steps, so it runs from shared memory: with smem_mode 2 the
// node vectors and the level tables (diagonal, CSR rows, children, parents) are copied
// in first, all copies in flight at once (cp.async); with 1 only the node vectors live
// there; with 0 everything stays in the workspace.
struct TopLevel {
  double *ar, *ax, *at, *inv;
  const double *diag, *val;
  const int *row, *col, *cptr, *cidx, *parent;
  int n;
};

// Shared-memory bytes of the node vectors (3 per node) and of the staged tables: per
// level the inverse diagonal, the diagonal, the CSR values, rows and columns, and above
// level 0 the children and parents; every piece 16-byte aligned.
__host__ __device__ inline size_t top_piece(size_t bytes) { return (bytes + 15) & ~(size_t)15; }
__host__ __device__ inline size_t top_vec_bytes(const MgDev& mg) {
  size_t nodes = 0;
  for (int k = 0; k < mg.M; ++k) nodes += (size_t)mg.n[k];
  return top_piece(3 * 8 * nodes);
}
__host__ __device__ inline size_t top_table_bytes(const MgDev& mg) {
  size_t b = 0;
  for (int k = 0; k < mg.M; ++k) {
    const size_t n = (size_t)mg.n[k], nnz = (size_t)mg.nnz[k], np = k ? (size_t)mg.n[k - 1] : 0;
    b += 2 * top_piece(8 * n) + top_piece(8 * nnz) + top_piece(4 * (n + 1)) + top_piece(4 * nnz);
    if (k) b += top_piece(4 * (n + 1)) + 2 * top_piece(4 * np);
  }
  return b;
}

// asynchronous global -> shared copy of `count` elements of 4 or 8 bytes, by the block
template <int E>
__device__ __forceinline__ void copy_async(void* dst, const void* src, int count) {
  static_assert(E == 4 || E == 8, "element size");
  for (int a = threadIdx.x; a < count; a += blockDim.x) {
    const unsigned int d = (unsigned int)__cvta_generic_to_shared(static_cast<char*>(dst) + (size_t)E * a);
    const char* s = static_cast<const char*>(src) + (size_t)E * a;
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(s), "n"(E) : "memory");
  }
}

template <class TV>
__device__ void mg_top(const MgDev& mg, const TV* __restrict__ rr, int smem_mode, double* sm) {
  __shared__ TopLevel lv[kMgMaxM];
  const int tid = threadIdx.x, NT = blockDim.x;
  const double w = kMgOmega;
  if (tid == 0) {  // layout from the sizes alone (no memory reads)
    int tot = 0;
    for (int k = 0; k < mg.M; ++k) tot += mg.n[k];
    int off = 0;
    unsigned char* base = reinterpret_cast<unsigned char*>(sm);
    size_t o = top_vec_bytes(mg);
    auto take = [&](size_t bytes) {
      unsigned char* p = base + o;
      o += top_piece(bytes);
      return p;
    };
    for (int k = 0; k < mg.M; ++k) {
      TopLevel& L = lv[k];
      const int n = mg.n[k], nnz = mg.nnz[k], np = k ? mg.n[k - 1] : 0;
      L.n = n;
      L.ar = smem_mode ? sm + off : mg.ar[k];
      L.ax = smem_mode ? sm + tot + off : mg.ax[k];
      L.at = smem_mode ? sm + 2 * tot + off : mg.at[k];
      off += n;
      if (smem_mode == 2) {
        L.inv = reinterpret_cast<double*>(take(8 * (size_t)n));
        L.diag = reinterpret_cast<double*>(take(8 * (size_t)n));
        L.val = reinterpret_cast<double*>(take(8 * (size_t)nnz));
        L.row = reinterpret_cast<int*>(take(4 * ((size_t)n + 1)));
        L.col = reinterpret_cast<int*>(take(4 * (size_t)nnz));
        L.cptr = k ? reinterpret_cast<int*>(take(4 * ((size_t)n + 1))) : mg.cptr[k];
        L.cidx = k ? reinterpret_cast<int*>(take(4 * (size_t)np)) : mg.cidx[k];
        L.parent = k ? reinterpret_cast<int*>(take(4 * (size_t)np)) : mg.parent[k];
      } else {
        L.inv = nullptr;
        L.diag = mg.diag[k];
        L.val = mg.val[k];
        L.row = mg.row[k];
        L.col = mg.col[k];
        L.cptr = mg.cptr[k];
        L.cidx = mg.cidx[k];
        L.parent = mg.parent[k];
      }
    }
  }
  __syncthreads();
  if (smem_mode == 2) {
    for (int k = 0; k < mg.M; ++k) {
      const TopLevel& L = lv[k];
      const int n = L.n, nnz = mg.nnz[k], np = k ? mg.n[k - 1] : 0;
      copy_async<8>(const_cast<double*>(L.diag), mg.diag[k], n);
      copy_async<8>(const_cast<double*>(L.val), mg.val[k], nnz);
      copy_async<4>(const_cast<int*>(L.row), mg.row[k], n + 1);
      copy_async<4>(const_cast<int*>(L.col), mg.col[k], nnz);
      if (k) {
        copy_async<4>(const_cast<int*>(L.cptr), mg.cptr[k], n + 1);
        copy_async<4>(const_cast<int*>(L.cidx), mg.cidx[k], np);
        copy_async<4>(const_cast<int*>(L.parent), mg.parent[k], np);
      }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    for (int k = 0; k < mg.M; ++k) {
      const TopLevel& L = lv[k];
      for (int a = tid; a < L.n; a += NT) {
        const double d = L.diag[a];
        L.inv[a] = d > 0.0 ? 1.0 / d : 0.0;
      }
    }
  }
  auto dinv = [&](const TopLevel& L, int a) {
    if (L.inv) return L.inv[a];
    const double d = L.diag[a];
    return d > 0.0 ? 1.0 / d : 0.0;
  };
  // at = ar - K ax on level k
  auto residual = [&](const TopLevel& L) {
    for (int a = tid; a < L.n; a += NT) {
      double kx = L.diag[a] * L.ax[a];
      for (int e = L.row[a]; e < L.row[a + 1]; ++e) kx -= L.val[e] * L.ax[L.col[e]];
      L.at[a] = L.ar[a] - kx;
    }
    __syncthreads();
  };
  for (int a = tid; a < mg.n[0]; a += NT) {  // level 0: sums of the cubes' residuals
    double sum = 0.0;
    for (int e = mg.cptr[0][a]; e < mg.cptr[0][a + 1]; ++e) sum += double(rr[mg.cidx[0][e]]);
    lv[0].ar[a] = sum;
  }
  __syncthreads();
  const int top = mg.M - 1;
  for (int k = 0; k < top; ++k) {
    const TopLevel& L = lv[k];
    for (int a = tid; a < L.n; a += NT) L.ax[a] = w * dinv(L, a) * L.ar[a];
    __syncthreads();
    residual(L);
    const TopLevel& C = lv[k + 1];
    for (int a = tid; a < C.n; a += NT) {
      double sum = 0.0;
      for (int e = C.cptr[a]; e < C.cptr[a + 1]; ++e) sum += L.at[C.cidx[e]];
      C.ar[a] = sum;
    }
    __syncthreads();
  }
  {
    const TopLevel& L = lv[top];
    for (int a = tid; a < L.n; a += NT) L.ax[a] = 0.0;
    __syncthreads();
    for (int sweep = 0; sweep < kMgNuTop; ++sweep) {
      residual(L);
      for (int a = tid; a < L.n; a += NT) L.ax[a] += w * dinv(L, a) * L.at[a];
      __syncthreads();
    }
  }
  for (int k = top - 1; k >= 0; --k) {
    const TopLevel& L = lv[k];
    const TopLevel& C = lv[k + 1];
    for (int a = tid; a < L.n; a += NT) L.ax[a] += kMgOver * C.ax[C.parent[a]];
    __syncthreads();
    residual(L);
    for (int a = tid; a < L.n; a += NT) L.ax[a] += w * dinv(L, a) * L.at[a];
    __syncthreads();
  }
  if (smem_mode) {  // the level-0 result for the up launches
    for (int a = tid; a < mg.n[0]; a += NT) mg.ax[0][a] = lv[0].ax[a];
  }
}

template <class TV>
__global__ __launch_bounds__(1024) void k_mg_top(MgDev mg, const TV* __restrict__ rr,
                                                 int smem_mode) {
  cudaGridDependencySynchronize();  // launched after the previous level's kernel
  extern __shared__ __align__(16) unsigned char smem_raw[];
  mg_top<TV>(mg, rr, smem_mode, reinterpret_cast<double*>(smem_raw));
}

// ---------------------------------------------------------------- launcher

template <int BL, class TV>
static cudaError_t down_t(const Ctx& x, int l, int all) {
  constexpr int CB = BL > 1 ? BL / 2 : 1;
  const TV* r = (const TV*)x.mg.r[l];
  TV* xv = (TV*)x.mg.x[l];
  TV* rc = BL > 1 ? (TV*)x.mg.r[l + 1] : (TV*)x.mg.rr;
  const double c4 = double(1 << (2 * l));
  if constexpr (BL > 1) {  // one thread per fine cell
    const long long n = (long long)x.g.n_cubes * BL * BL * BL;
    return launch_pdl(k_mg_down_cell<BL, TV>, dim3((unsigned)((n + 255) / 256)), dim3(256), 0,
                      x.stream, x.g, l, TV(kMgOmega / c4), TV(c4), r, xv, rc, all);
  } else {
    const long long n = (long long)x.g.n_cubes * CB * CB * CB;
    return launch_pdl(k_mg_down<BL, TV>, dim3((unsigned)((n + 255) / 256)), dim3(256), 0,
                      x.stream, x.g, l, TV(kMgOmega / c4), TV(c4), r, xv, rc, all);
  }
}

template <int BL, class TV>
static cudaError_t up_t(const Ctx& x, int l, int all) {
  const long long n = (long long)x.g.n_cubes * BL * BL * BL;
  const TV* yc = BL > 1 ? (const TV*)x.mg.y[l + 1] : nullptr;
  const double c4 = double(1 << (2 * l));
  return launch_pdl(k_mg_up<BL, TV>, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, x.stream,
                    x.g, l, TV(kMgOmega / c4), TV(c4), (const TV*)x.mg.r[l], (const TV*)x.mg.x[l],
                    yc, (const double*)x.mg.ax[0], (const int*)x.mg.parent[0], (TV*)x.mg.y[l],
                    all);
}

template <class TV>
static cudaError_t level_t(const Ctx& x, int l, bool down, int all) {
  const int BL = x.B >> l;
#define BCM_MG_LEVEL(V) \
  case V: return down ? down_t<V, TV>(x, l, all) : up_t<V, TV>(x, l, all);
  switch (BL) {
    BCM_MG_LEVEL(16)
    BCM_MG_LEVEL(8)
    BCM_MG_LEVEL(4)
    BCM_MG_LEVEL(2)
    BCM_MG_LEVEL(1)
    default: return cudaErrorInvalidValue;
  }
#undef BCM_MG_LEVEL
}

template <int B, class TV>
static cudaError_t up0_t(const Ctx& x, const SolveParams& prm, int mode) {
  constexpr int B3 = B * B * B, NT = B3 < 256 ? B3 : 256;
  const TV* yc = (const TV*)x.mg.y[1];
  return launch_pdl(k_mg_up0<B, NT, TV>, dim3(x.g.n_cubes * (B3 / NT)), dim3(NT), 0, x.stream,
                    x.g, (const TV*)x.mg.r[0], (const TV*)x.mg.x[0], yc,
                    (const double*)x.mg.ax[0], (const int*)x.mg.parent[0], (TV*)x.mg.y[0], prm,
                    mode);
}

template <int B, class TV>
static cudaError_t down0_tile_t(const Ctx& x, int l, int all, bool fb) {
  using SL = Slab<B, B>;
  const size_t sm = sizeof(TV) * ((SL::N + 3) / 4 * 4 + (size_t)B * B * B);
  PassB<TV> pb{};
  if (fb) {
    pb.x = x.solve64 ? (TV*)x.f.p : (TV*)x.f.e;
    pb.p0 = (const TV*)x.f.p0;
    pb.p1 = (const TV*)x.f.p1;
    pb.q = (const TV*)x.f.q;
    pb.ra = (TV*)x.f.r;
    pb.rb = (TV*)x.f.s0;
  }
  const double c4 = double(1 << (2 * l));
  auto kern = fb ? k_mg_down0_tile<B, TV, true> : k_mg_down0_tile<B, TV, false>;
  cudaError_t e = allow_dynamic_smem(kern, sm);
  if (e != cudaSuccess) return e;
  return launch_pdl(kern, dim3(x.g.n_cubes), dim3(B * B), sm, x.stream, x.g,
                    (const TV*)x.mg.r[l], (TV*)x.mg.x[l], (TV*)x.mg.r[l + 1], all, pb,
                    TV(kMgOmega / c4), TV(c4), l);
}

template <int B, class TV>
static cudaError_t up0_tile_t(const Ctx& x, int l, const SolveParams& prm, int mode, bool fb) {
  using SL = Slab<B, B>;
  const size_t sm = sizeof(TV) * SL::N;
  const double c4 = double(1 << (2 * l));
  auto kern = k_mg_up0_tile<B, TV>;
  cudaError_t e = allow_dynamic_smem(kern, sm);
  if (e != cudaSuccess) return e;
  return launch_pdl(kern, dim3(x.g.n_cubes), dim3(B * B), sm, x.stream, x.g,
                    (const TV*)x.mg.r[l], fb ? (const TV*)x.f.s0 : (const TV*)nullptr,
                    (const TV*)x.mg.x[l], (const TV*)x.mg.y[l + 1], (TV*)x.mg.y[l], prm, mode,
                    TV(kMgOmega / c4), TV(c4), l == 0 ? 1 : 0, l);
}

template <class TV>
static cudaError_t vcycle_t(const Ctx& x, const SolveParams& prm, int mode) {
  const int all = mode == 2 ? 1 : 0;
  cudaError_t e;
  // the finest level of 8^3 and 16^3 cubes through the shared-memory tile, which after
  // pass A also does the PCG's pass B; other cube sizes launch pass B first
  const bool tile = x.B == 8 || x.B == 16;
  const bool fb = tile && mode == 1;
  if (mode == 1 && !fb && (e = launch_cg_b(x, prm)) != cudaSuccess) return e;
  e = tile ? (x.B == 16 ? down0_tile_t<16, TV>(x, 0, all, fb) : down0_tile_t<8, TV>(x, 0, all, fb))
           : level_t<TV>(x, 0, true, all);
  if (e != cudaSuccess) return e;
  // levels of 8^3 cells per cube through the tile too, the smaller ones per cell
  for (int l = 1; l <= x.mg.L; ++l)
    if ((e = (x.B >> l) == 8 ? down0_tile_t<8, TV>(x, l, all, false)
                             : level_t<TV>(x, l, true, all)) != cudaSuccess)
      return e;
  {
    // node vectors and, where they fit, the level tables in shared memory
    const size_t vec = top_vec_bytes(x.mg), tables = top_table_bytes(x.mg);
    const int smem_mode = vec + tables <= 200 * 1024 ? 2 : vec <= 160 * 1024 ? 1 : 0;
    const size_t sm = smem_mode == 2 ? vec + tables : smem_mode == 1 ? vec : 0;
    int maxn = 0;
    for (int k = 0; k < x.mg.M; ++k) maxn = x.mg.n[k] > maxn ? x.mg.n[k] : maxn;
    const int nt = maxn < 64 ? 64 : maxn > 1024 ? 1024 : (maxn + 31) / 32 * 32;
    auto kern = k_mg_top<TV>;
    if (smem_mode && (e = allow_dynamic_smem(kern, sm)) != cudaSuccess) return e;
    if ((e = launch_pdl(kern, dim3(1), dim3(nt), sm, x.stream, x.mg, (const TV*)x.mg.rr,
                        smem_mode)) != cudaSuccess)
      return e;
  }
  for (int l = x.mg.L; l >= 1; --l)
    if ((e = (x.B >> l) == 8 ? up0_tile_t<8, TV>(x, l, prm, mode, false)
                             : level_t<TV>(x, l, false, all)) != cudaSuccess)
      return e;
  if (tile)
    return x.B == 16 ? up0_tile_t<16, TV>(x, 0, prm, mode, fb)
                     : up0_tile_t<8, TV>(x, 0, prm, mode, fb);
  switch (x.B) {
    case 4: return up0_t<4, TV>(x, prm, mode);
    case 8: return up0_t<8, TV>(x, prm, mode);
    case 16: return up0_t<16, TV>(x, prm, mode);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_mg_vcycle(const Ctx& x, const SolveParams& prm, int mode) {
  return x.solve64 ? vcycle_t<double>(x, prm, mode) : vcycle_t<float>(x, prm, mode);
}

}  // namespace bcm
