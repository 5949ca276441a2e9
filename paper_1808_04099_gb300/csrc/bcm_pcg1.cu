// bcm_pcg1.cu -- persistent Jacobi-PCG with one pass and one grid barrier per
// iteration (Eq. poisson; the single-reduction CG of Chronopoulos and Gear, 1989,
// with the Jacobi preconditioner M = diag(K)).
//
// The kernel keeps s = K p and w = K z (z = M^-1 r) beside r, p and x, so that
// every dot product of an iteration comes from one sweep:
//   p_k = z_k + beta_k p_{k-1},   s_k = w_k + beta_k s_{k-1},
//   x_{k+1} = x_k + alpha_k p_k,  r_{k+1} = r_k - alpha_k s_k,
//   w_{k+1} = K M^-1 r_{k+1},
//   gamma = <r, z>, delta = <z, w>, eps = <z, s_{k-1}>, <r, r>  (all at k+1),
// with beta_k = gamma_k / gamma_{k-1} and alpha_k = gamma_k / <p_k, s_k>, where
//   <p_k, s_k> = delta_k + 2 beta_k eps_k + beta_k^2 <p_{k-1}, s_{k-1}>
// follows from the symmetry of K alone (no conjugacy assumed), so the iteration is
// Saad's Alg. 9.1 in exact arithmetic also when it resumes a search direction kept
// from an earlier launch (the reliable-update mode of the mixed-precision solver).
//
// A pass stages z_{k+1} = M^-1 (r_k - alpha_k (w_k + beta_k s_{k-1})) on the slab and
// its face halo; the block's own cells also write p_k, s_k, x_{k+1} and r_{k+1}, and
// the stencil of the staged tile gives w_{k+1}.  r, w and s alternate between two
// buffers because neighbouring blocks read the halo of iteration k while a block
// writes iteration k+1; p and x are read and written by their owner only.  The
// first pass of a launch stages z_0 = M^-1 r_0 and forms w_0.
//
// Work distribution, slot rotation and the bounded grid barrier are those of the
// two-pass persistent kernel: dot products go to striped accumulators in three
// rotating slots, every block derives the scalars from the same sums, block 0 clears
// the slot two iterations ahead, and every wait ends in BCM_E_TIMEOUT at worst.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bcm_cube.cuh"
#include "bcm_internal.cuh"
#include "bcm_kernels.h"
#include "bcm_persist.cuh"

namespace bcm {

// z_{k+1} at one cell from the cell's r_k, w_k, s_{k-1} (first: s_k = w_k).  The
// owner of the cell evaluates the same expressions when it writes s_k and r_{k+1}.
template <class TV>
__device__ __forceinline__ TV next_z(TV r, TV w, TV s, TV alpha, TV beta, bool first, TV inv) {
  const TV sn = first ? w : w + beta * s;
  const TV rn = r - alpha * sn;
  return rn * inv;
}

template <int B, int KS, int NT, class TV, class TX>
__global__ __launch_bounds__(NT, 4) void k_pcg1(DevGrid g, TX* __restrict__ x,
                                             TV* __restrict__ r0, TV* __restrict__ r1,
                                             TV* __restrict__ w0, TV* __restrict__ w1,
                                             TV* __restrict__ s0, TV* __restrict__ s1,
                                             TV* __restrict__ pv, SolveParams prm,
                                             unsigned int* bar, int* err) {
  using SL = Slab<B, KS>;
  constexpr int B3 = B * B * B, BB = B * B, NSL = B / KS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TV* S = reinterpret_cast<TV*>(smem_raw);
  __shared__ CubeSh<TV> cs;
  __shared__ int cs_cube;
  __shared__ double red[4 * 32];
  const int nsim = g.n_sims;
  double* s_alpha = reinterpret_cast<double*>(smem_raw + (sizeof(TV) * SL::N + 15) / 16 * 16);
  double* s_beta = s_alpha + nsim;
  double* s_gam = s_beta + nsim;   // gamma of the current direction
  double* s_phi = s_gam + nsim;    // <p, K p> of the current direction
  unsigned char* s_done = reinterpret_cast<unsigned char*>(s_phi + nsim);
  unsigned char* s_first = s_done + nsim;  // no kept direction: p_0 = z_0
  unsigned char* s_soff = s_first + nsim;  // s_k lives in buffer (k + soff) & 1
  const bool inner = prm.mixed != 0;
  const int kmax = inner ? prm.inner_max_iter : prm.max_iter;
  const int N = g.n_cubes * NSL, P = gridDim.x, pb = blockIdx.x;
  const int Lq = N / P, Rq = N % P;
  const int item0 = pb * Lq + min(pb, Rq), nitems = (N + P - pb - 1) / P;
  if (threadIdx.x == 0) cs_cube = -1;
  for (int s = threadIdx.x; s < nsim; s += NT) {
    const SimState& st = g.ss[s];
    const bool keep = st.cont != 0 && st.rz_last != 0.0;
    s_done[s] = st.done ? 1 : 0;
    s_first[s] = keep ? 0 : 1;
    s_gam[s] = keep ? st.rz_last : 0.0;
    s_phi[s] = keep ? st.phi_last : 0.0;
    s_soff[s] = keep ? (unsigned char)((st.s_off + 1) & 1) : 0;
    s_alpha[s] = 0.0;
    s_beta[s] = 0.0;
  }
  __syncthreads();
  GridBarrier gb;
  gb.init(bar, err, prm.barrier_timeout_ns);
  // k = -1: the launch's first pass (w_0 and the dots of iteration 0)
  for (int k = -1;; ++k) {
    if (k >= 0) {
      // ---- decisions for iteration k (identical in every block)
      int alive = 0;
      for (int s = threadIdx.x; s < nsim; s += NT) {
        SimState& st = g.ss[s];
        if (s_done[s]) continue;
        const double gam = slot_sum(st, ACC_SLOT_G + k % 3);
        const double del = slot_sum(st, ACC_SLOT_D + k % 3);
        const double eps = slot_sum(st, ACC_SLOT_E + k % 3);
        const double rr = slot_sum(st, ACC_SLOT_R + k % 3);
        const double tol2 = inner ? st.inner_tol2 : st.tol2;
        const bool bad = !isfinite(rr) || !isfinite(gam) || !isfinite(del) || !isfinite(eps);
        if (bad || rr <= tol2 || k >= kmax) {
          s_done[s] = 1;
          if (blockIdx.x == 0) {  // single writer of the solve's results
            st.iter = k;
            st.total_iters += k;
            st.rr = rr;
            st.done = 1;
            // the last direction: p_{k-1} (p buffer), s_{k-1}; unchanged when k = 0
            st.rz_last = s_gam[s];
            st.phi_last = s_phi[s];
            st.s_off = (k - 1 + s_soff[s]) & 1;
            if (bad) st.nonfinite = 1;
            if (!inner) {
              st.rr64 = rr;
              st.converged = !bad && rr <= tol2;
            }
          }
          continue;
        }
        const bool first = k == 0 && s_first[s];
        const double beta = (first || s_gam[s] == 0.0) ? 0.0 : gam / s_gam[s];
        const double phi = first ? del : del + 2.0 * beta * eps + beta * beta * s_phi[s];
        s_beta[s] = beta;
        s_alpha[s] = (phi != 0.0 && isfinite(phi)) ? gam / phi : 0.0;
        s_gam[s] = gam;
        s_phi[s] = phi;
        alive = 1;
      }
      alive = __syncthreads_or(alive);
      if (!alive) break;
      if (blockIdx.x == 0)  // the slot pass k+1 fills (read at iteration k-1)
        for (int i = threadIdx.x; i < nsim * kStripes; i += NT) {
          SimState& st = g.ss[i / kStripes];
          const int sp = i % kStripes, sl = (k + 2) % 3;
          st.acc[sp][ACC_SLOT_G + sl] = 0.0;
          st.acc[sp][ACC_SLOT_D + sl] = 0.0;
          st.acc[sp][ACC_SLOT_E + sl] = 0.0;
          st.acc[sp][ACC_SLOT_R + sl] = 0.0;
        }
    }
    const bool init = k < 0;
    const int out = (k + 1) % 3;  // slot of this pass's sums
    TV* __restrict__ rin = (k & 1) ? r1 : r0;  // k = -1 reads r_0 from r0 (no writes)
    TV* __restrict__ rout = (k & 1) ? r0 : r1;
    const TV* __restrict__ win = (k & 1) ? w1 : w0;
    TV* __restrict__ wout = init ? w0 : ((k & 1) ? w0 : w1);
    if (init) rin = r0;
    for (int it = 0; it < nitems; ++it) {
      const int item = item0 + it, c = item / NSL, z0 = (item - c * NSL) * KS;
      const int s = g.sim[c];
      if (s_done[s]) continue;
      if (cs_cube != c) {
        __syncthreads();
        load_cube(cs, g, c);
        if (threadIdx.x == 0) cs_cube = c;
        __syncthreads();
      }
      const TV alpha = TV(s_alpha[s]), beta = TV(s_beta[s]);
      const bool first = init || (k == 0 && s_first[s]);
      const int so = s_soff[s];
      // s_{k-1}; the first pass reads the kept direction's s_{-1}
      const TV* __restrict__ sin = (((init ? 0 : k) - 1 + so) & 1) ? s1 : s0;
      TV* __restrict__ sout = ((k + so) & 1) ? s1 : s0;           // s_k
      const bool eps_on = init && !s_first[s];  // first pass: a kept direction exists
      TV ga = TV(0), ep = TV(0), rq = TV(0);
      // one cell's value in the staged tile; own cells also advance the iterate
      auto cellz = [&](TV rv, TV wv, TV sv, TV inv) {
        return init ? rv * inv : next_z(rv, wv, sv, alpha, beta, first, inv);
      };
      auto val4 = [&](int cube, int cell0, int face, TV (&v)[4]) {
        const size_t gi = (size_t)cube * B3 + cell0;
        const int kz = cell0 / BB, j = (cell0 / B) % B, i0 = cell0 % B;
        const int mask = face < 0 ? cs.smask : cs.nbmask[face];
        const int* w3 = face < 0 ? cs.w3 : cs.nbw3[face];
        TV inv[4];
#pragma unroll
        for (int m = 0; m < 4; ++m)
          inv[m] = mask == 0 ? cs.invtab[18] : cs.invtab[s3_of<B>(w3, i0 + m, j, kz)];
        TV rv[4], wv[4] = {TV(0), TV(0), TV(0), TV(0)}, sv[4] = {TV(0), TV(0), TV(0), TV(0)};
        ld4(rin + gi, rv);
        if (!init) ld4(win + gi, wv);
        const bool own = face < 0 && kz >= z0 && kz < z0 + KS;
        if (own) {
          if (init) {
#pragma unroll
            for (int m = 0; m < 4; ++m) {
              const TV z = rv[m] * inv[m];
              v[m] = z;
              ga += rv[m] * z;
              rq += rv[m] * rv[m];
            }
            if (eps_on) {
              ld4(sin + gi, sv);
#pragma unroll
              for (int m = 0; m < 4; ++m) ep += v[m] * sv[m];
            }
            return;
          }
          TV pp[4] = {TV(0), TV(0), TV(0), TV(0)}, xv[4];
          if (!first) {
            ld4(sin + gi, sv);
            ld4(pv + gi, pp);
          }
          ld4(x + gi, xv);
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const TV z = rv[m] * inv[m];
            const TV pn = first ? z : z + beta * pp[m];
            const TV sn = first ? wv[m] : wv[m] + beta * sv[m];
            const TV rn = rv[m] - alpha * sn;
            const TV zn = rn * inv[m];
            xv[m] = xv[m] + alpha * pn;
            pp[m] = pn;
            sv[m] = sn;
            rv[m] = rn;
            v[m] = zn;
            ga += rn * zn;
            ep += zn * sn;
            rq += rn * rn;
          }
          st4(pv + gi, pp);
          st4(sout + gi, sv);
          st4(x + gi, xv);
          st4(rout + gi, rv);
          return;
        }
        if (!init && !first) ld4(sin + gi, sv);
#pragma unroll
        for (int m = 0; m < 4; ++m) v[m] = cellz(rv[m], wv[m], sv[m], inv[m]);
      };
      auto val1 = [&](int f, int n, int cell) {
        const size_t gi = (size_t)n * B3 + cell;
        TV inv;
        if (cs.nbmask[f] == 0) {
          inv = cs.invtab[18];
        } else {
          const int i = cell % B, j = (cell / B) % B, kz = cell / BB;
          inv = cs.invtab[s3_of<B>(cs.nbw3[f], i, j, kz)];
        }
        return cellz(rin[gi], init ? TV(0) : win[gi], (init || first) ? TV(0) : sin[gi], inv);
      };
      auto valg = [&](int n, int cell) {
        const size_t gi = (size_t)n * B3 + cell;
        return cellz(rin[gi], init ? TV(0) : win[gi], (init || first) ? TV(0) : sin[gi],
                     inv_diag_any<B, TV>(g, n, cell));
      };
      stage_pressure_slab<B, KS, NT, TV>(S, cs, g, c, z0, val4, val1, valg);
      // w_{k+1} = K z_{k+1} on the own planes, and <z, w>
      const TV h = TV(cell_h<B>(g, c));
      const size_t base = (size_t)c * B3 + (size_t)z0 * BB;
      TV de = TV(0);
      if (NT == BB) {
        constexpr int PP = SL::P * SL::P;
        const int i = threadIdx.x % B, j = column_row<B>(threadIdx.x);
        int o = SL::at(i, j, 1);
        TV below = S[o - PP], cur = S[o];
#pragma unroll 4
        for (int kk = 0; kk < KS; ++kk) {
          const TV above = S[o + PP];
          TV acc = (cur - S[o - 1]) + (cur - S[o + 1]) + (cur - S[o - SL::P]) +
                   (cur - S[o + SL::P]) + (cur - below) + (cur - above);
          if (cs.has21) acc = stencil_sum_w<B, TV, KS>(S, o, cs, i, j, z0 + kk);
          const TV wv = h * acc;
          wout[base + (size_t)kk * BB + j * B + i] = wv;
          de += cur * wv;
          below = cur;
          cur = above;
          o += PP;
        }
      } else {
        for (int q4 = threadIdx.x; q4 < KS * BB / 4; q4 += NT) {
          const int cell = 4 * q4, kk = cell / BB, j = (cell / B) % B, i0 = cell % B;
          const int o = SL::at(i0, j, kk + 1);
          TV wv[4];
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            wv[m] = h * stencil_sum_w<B, TV, KS>(S, o + m, cs, i0 + m, j, z0 + kk);
            de += S[o + m] * wv[m];
          }
          st4(wout + base + cell, wv);
        }
      }
      const TV pp[4] = {ga, TV(de), ep, rq};
      double vals[4];
      block_sum_tv<NT, 4, TV>(pp, vals, red);
      if (threadIdx.x == 0) {
        acc_add(g.ss[s], ACC_SLOT_G + out, vals[0]);
        acc_add(g.ss[s], ACC_SLOT_D + out, vals[1]);
        acc_add(g.ss[s], ACC_SLOT_E + out, vals[2]);
        acc_add(g.ss[s], ACC_SLOT_R + out, vals[3]);
      }
    }
    if (!gb.sync()) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) g.flags[0] = 1;
}

// ---------------------------------------------------------------- launcher

template <int B, int KS, class TV, class TX>
static cudaError_t pcg1_t(const Ctx& x, const SolveParams& prm, TX* xv) {
  constexpr int NT = pcg_threads<B>();
  // tile (16-byte multiple) + alpha, beta, gamma, phi (FP64), done, first, s_off (bytes)
  const size_t tile = (sizeof(TV) * Slab<B, KS>::N + 15) / 16 * 16;
  const size_t sm = tile + (size_t)x.g.n_sims * (4 * sizeof(double) + 3);
  auto kern = k_pcg1<B, KS, NT, TV, TX>;
  {
    const cudaError_t e = allow_dynamic_smem(kern, sm);
    if (e != cudaSuccess) return e;
  }
  int maxg = 0;
  int rc = max_coresident(kern, NT, sm, &maxg);
  if (rc) return (cudaError_t)rc;
  if (maxg < 1) return cudaErrorCooperativeLaunchTooLarge;
  const int items = x.g.n_cubes * (B / KS);
  const int per = (items + maxg - 1) / maxg;
  const int grid = (items + per - 1) / per;
  DevGrid gg = x.g;
  TX* xp = xv;
  TV* r0 = (TV*)x.f.r;
  TV* r1 = (TV*)x.f.q;
  TV* w0 = (TV*)x.f.p1;
  TV* w1 = (TV*)x.f.w1;
  TV* s0 = (TV*)x.f.s0;
  TV* s1 = (TV*)x.f.s1;
  TV* pp = (TV*)x.f.p0;
  SolveParams pr = prm;
  unsigned int* bar = x.f.bar;
  int* err = x.f.err;
  void* args[] = {&gg, &xp, &r0, &r1, &w0, &w1, &s0, &s1, &pp, &pr, &bar, &err};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(NT), args, sm, x.stream);
}

template <class TV, class TX>
static cudaError_t pcg1_dispatch(const Ctx& x, const SolveParams& prm, TX* xv) {
  switch (x.B) {
    case 4: return pcg1_t<4, 4, TV, TX>(x, prm, xv);
    case 8: return pcg1_t<8, 8, TV, TX>(x, prm, xv);
    case 16:
      if (x.slabs_p == 2) return pcg1_t<16, 8, TV, TX>(x, prm, xv);
      if (x.slabs_p == 4) return pcg1_t<16, 4, TV, TX>(x, prm, xv);
      return pcg1_t<16, 16, TV, TX>(x, prm, xv);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pcg1(const Ctx& x, const SolveParams& prm) {
  if (x.g.n_sims > kMaxPersistentSims) return cudaErrorInvalidValue;
  return x.solve64 ? pcg1_dispatch<double, double>(x, prm, x.f.p)
               : pcg1_dispatch<float, float>(x, prm, x.f.e);
}

}  // namespace bcm
