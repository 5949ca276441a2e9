// bcm_pcg.cu -- persistent Jacobi-PCG solver kernel (Eq. poisson; Saad, Alg. 9.1).
//
// One cooperative launch runs all PCG iterations of a solve on every co-resident block.
// Work items are z-slabs of cubes; block p owns a contiguous run of items by the
// paper's load-balanced linear distribution (Eq. loaddist: L = floor(N/P), R = N mod P,
// n_p = floor((N + P - p - 1) / P)), so Z-ordered neighbours mostly share a block, and
// keeps the constants of its cubes in shared memory for the whole solve.  Each
// iteration is pass A (p = z + beta p, q = K p, <p,q>, and the previous iteration's
// x += alpha p on the own cells while their old p is staged), a grid barrier, pass B
// (r -= alpha q, <r,z>, <r,r>), and a second grid barrier; the last iteration's
// x += alpha p runs at the launch's exit.
//
// The per-sim scalars never need a single writer: the dot products go to striped
// accumulators in three rotating slots (iteration k mod 3), and after each barrier
// every block derives alpha, beta and the convergence decision from the same sums.
// Block 0 clears the slot that iteration k+1 will fill.  A grid barrier counts the
// arrivals on one counter (a reduction that returns nothing) and waits until it reaches
// the grid size times the barriers passed; every wait is bounded by %globaltimer, and a
// timeout sets an error flag and ends the kernel (reported to the host as
// BCM_E_TIMEOUT), so a fault never hangs the GPU.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bcm_cube.cuh"
#include "bcm_internal.cuh"
#include "bcm_kernels.h"
#include "bcm_persist.cuh"

namespace bcm {

constexpr int kCubeCache = 4;  // cubes whose constants a block keeps for the whole solve

template <int B, int KS, int NT, class TV, class TX>
__global__ __launch_bounds__(NT, 4) void k_pcg(DevGrid g, TX* __restrict__ x, TV* __restrict__ r,
                                            TV* __restrict__ p0, TV* __restrict__ p1,
                                            TV* __restrict__ q, SolveParams prm,
                                            unsigned int* bar, int* err) {
  using SL = Slab<B, KS>;
  constexpr int B3 = B * B * B, BB = B * B, NSL = B / KS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TV* S = reinterpret_cast<TV*>(smem_raw);
  __shared__ CubeSh<TV> csa[kCubeCache];  // the block's cubes, or one reloaded per item
  __shared__ int tsim[kCubeCache];        // ... their sims and cell sizes
  __shared__ TV th[kCubeCache];
  __shared__ int cs_cube;
  __shared__ double red[2 * 32];
  const int nsim = g.n_sims;
  // per-sim scalars after the tile (dynamic shared memory, see pcg_smem)
  double* s_alpha = reinterpret_cast<double*>(smem_raw + (sizeof(TV) * SL::N + 15) / 16 * 16);
  double* s_beta = s_alpha + nsim;
  double* s_rz = s_beta + nsim;
  int* s_kdone = reinterpret_cast<int*>(s_rz + nsim);  // iterations this launch ran
  unsigned char* s_done = reinterpret_cast<unsigned char*>(s_kdone + nsim);
  unsigned char* s_first = s_done + nsim;  // restart with p = z at iteration 0
  unsigned char* s_poff = s_first + nsim;  // search-direction buffer offset
  const bool inner = prm.mixed != 0;
  const int kmax = inner ? prm.inner_max_iter : prm.max_iter;
  // my items by the linear load-balanced distribution
  const int N = g.n_cubes * NSL, P = gridDim.x, p = blockIdx.x;
  const int Lq = N / P, Rq = N % P;
  const int item0 = p * Lq + min(p, Rq), nitems = (N + P - p - 1) / P;
  if (threadIdx.x == 0) cs_cube = -1;
  // the state at entry: iteration 0 uses the residual kernel's scalars
  for (int s = threadIdx.x; s < nsim; s += NT) {
    SimState& st = g.ss[s];
    const bool cont = st.cont != 0;
    s_rz[s] = cont ? st.rz_last : st.rz;
    s_done[s] = st.done ? 1 : 0;
    s_kdone[s] = 0;
    s_first[s] = cont ? 0 : 1;
    s_poff[s] = cont ? (unsigned char)(st.p_off & 1) : 0;
  }
  // the block's items span cubes cA .. cB; their constants stay in shared memory
  // when they fit the cache (every grid up to a few cubes per block)
  const int cA = item0 / NSL, cB = (item0 + max(nitems, 1) - 1) / NSL;
  const bool cached = cB - cA < kCubeCache;
  if (cached) {
    for (int c = cA; c <= cB && c < g.n_cubes; ++c) load_cube(csa[c - cA], g, c);
    for (int c = cA + threadIdx.x; c <= cB && c < g.n_cubes; c += NT) {
      tsim[c - cA] = g.sim[c];
      th[c - cA] = TV(cell_h<B>(g, c));
    }
  }
  __syncthreads();
  auto sim_of = [&](int c) { return cached ? tsim[c - cA] : g.sim[c]; };
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  GridBarrier gb;
  gb.init(bar, err, prm.barrier_timeout_ns);
  bool failed = false;
  int k = 0;
  for (;; ++k) {
    // ---- decisions for iteration k (identical in every block): warp w takes sims w,
    // w + NW, ..., its lanes reading the stripes of <r,z> and <r,r> together
    int alive = 0;
    for (int s = warp; s < nsim; s += NW) {
      SimState& st = g.ss[s];
      if (s_done[s]) continue;
      double rz, rr;
      if (k == 0) {
        rz = st.rz;
        rr = st.rr;
      } else {
        warp_slot_sums(st, ACC_SLOT_RZ + k % 3, ACC_SLOT_RR + k % 3, rz, rr);
      }
      if (lane != 0) continue;
      const double tol2 = inner ? st.inner_tol2 : st.tol2;
      const bool bad = !isfinite(rr) || !isfinite(rz);
      if (bad || rr <= tol2 || k >= kmax) {
        s_done[s] = 1;
        s_kdone[s] = k;
        if (blockIdx.x == 0) {  // single writer of the solve's results
          st.iter = k;
          st.total_iters += k;
          st.rr = rr;
          st.done = 1;
          st.rz_last = s_rz[s];               // <r,z> of the last direction's iteration
          st.p_off = (k + s_poff[s]) & 1;     // buffer holding the last direction
          if (bad) st.nonfinite = 1;
          if (!inner) {
            st.rr64 = rr;
            st.converged = !bad && rr <= tol2;
          }
        }
        continue;
      }
      s_beta[s] = ((k == 0 && s_first[s]) || s_rz[s] == 0.0) ? 0.0 : rz / s_rz[s];
      s_rz[s] = rz;
      alive = 1;
    }
    alive = __syncthreads_or(alive);
    if (!alive) break;
    if (blockIdx.x == 0)  // clear the slots iteration k+1 fills (held iteration k-2's sums)
      for (int i = threadIdx.x; i < nsim * kStripes; i += NT) {
        SimState& st = g.ss[i / kStripes];
        const int sp = i % kStripes, sl = (k + 1) % 3;
        st.acc[sp][ACC_SLOT_RZ + sl] = 0.0;
        st.acc[sp][ACC_SLOT_RR + sl] = 0.0;
        st.acc[sp][ACC_SLOT_PQ + sl] = 0.0;
      }
    // ---- pass A over my items; <p, q> summed over the block's items of one sim
    TV part = TV(0);
    int psim = -1;
    auto flush_pq = [&]() {
      const TV pp[1] = {part};
      double vals[1];
      block_sum_tv<NT, 1, TV>(pp, vals, red);
      if (threadIdx.x == 0) acc_add(g.ss[psim], ACC_SLOT_PQ + k % 3, vals[0]);
      part = TV(0);
    };
    for (int it = 0; it < nitems; ++it) {
      const int item = item0 + it, c = item / NSL, z0 = (item - c * NSL) * KS;
      const int s = sim_of(c);
      if (s_done[s]) continue;
      if (psim >= 0) {
        if (psim != s) flush_pq();
        __syncthreads();  // the previous item's stencil has read the tile
      }
      psim = s;
      if (!cached && cs_cube != c) {
        __syncthreads();
        load_cube(csa[0], g, c);
        if (threadIdx.x == 0) cs_cube = c;
        __syncthreads();
      }
      const CubeSh<TV>& cs = csa[cached ? c - cA : 0];
      const TV beta = TV(s_beta[s]);
      const bool first = (k == 0) && s_first[s];
      const int pb = (k + s_poff[s]) & 1;
      const TV* __restrict__ pold = pb ? p1 : p0;
      TV* __restrict__ pnew = pb ? p0 : p1;
      // x += alpha p of the previous iteration, on this item's own cells as their p is
      // staged (pass B leaves it; every later iteration of the sim comes through here)
      const TV alpha_prev = TV(s_alpha[s]);
      auto val4 = [&](int cube, int cell0, int face, TV (&v)[4]) {
        const size_t gi = (size_t)cube * B3 + cell0;
        TV rr4[4], pp[4] = {TV(0), TV(0), TV(0), TV(0)};
        ld4(r + gi, rr4);
        if (!first) ld4(pold + gi, pp);
        if (k > 0 && face < 0 && (unsigned)(cell0 - z0 * BB) < (unsigned)(KS * BB)) {
          TX xv[4];
          ld4(x + gi, xv);
#pragma unroll
          for (int m = 0; m < 4; ++m) xv[m] = xv[m] + alpha_prev * pp[m];
          st4(x + gi, xv);
        }
        const int mask = face < 0 ? cs.smask : cs.nbmask[face];
        if (mask == 0) {  // every face of that cube has the same-level weight
          const TV inv = cs.invtab[18];
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const TV z = rr4[m] * inv;
            v[m] = first ? z : z + beta * pp[m];
          }
        } else {
          const int* w3 = face < 0 ? cs.w3 : cs.nbw3[face];
          const int kz = cell0 / BB, j = (cell0 / B) % B, i0 = cell0 % B;
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const TV z = rr4[m] * cs.invtab[s3_of<B>(w3, i0 + m, j, kz)];
            v[m] = first ? z : z + beta * pp[m];
          }
        }
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
        const TV z = r[gi] * inv;
        return first ? z : z + beta * pold[gi];
      };
      auto valg = [&](int n, int cell) {
        const size_t gi = (size_t)n * B3 + cell;
        const TV z = r[gi] * inv_diag_any<B, TV>(g, n, cell);
        return first ? z : z + beta * pold[gi];
      };
      stage_pressure_slab<B, KS, NT, TV>(S, cs, g, c, z0, val4, val1, valg);
      const TV h = cached ? th[c - cA] : TV(cell_h<B>(g, c));
      const size_t base = (size_t)c * B3 + (size_t)z0 * BB;
      if (NT == BB) {
        // one thread per (i, j) column marching up the slab: the z neighbours roll
        // through registers, each plane costs five shared loads per cell
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
          const TV qv = h * acc;
          const size_t gi = base + (size_t)kk * BB + j * B + i;
          pnew[gi] = cur;
          q[gi] = qv;
          part += cur * qv;
          below = cur;
          cur = above;
          o += PP;
        }
      } else {
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
      }
    }
    if (psim >= 0) flush_pq();
    if (!gb.sync()) {
      failed = true;
      break;
    }
    // ---- alpha per sim from the completed <p, q>
    for (int s = warp; s < nsim; s += NW) {
      if (s_done[s]) continue;
      double pq, pq2;
      warp_slot_sums(g.ss[s], ACC_SLOT_PQ + k % 3, ACC_SLOT_PQ + k % 3, pq, pq2);
      if (lane == 0) s_alpha[s] = (pq != 0.0 && isfinite(pq)) ? s_rz[s] / pq : 0.0;
    }
    __syncthreads();
    // ---- pass B over my items (pointwise); the dots summed per sim as in pass A
    TV rz = TV(0), rr = TV(0);
    psim = -1;
    auto flush_rz = [&]() {
      const TV pp[2] = {rz, rr};
      double vals[2];
      block_sum_tv<NT, 2, TV>(pp, vals, red);
      if (threadIdx.x == 0) {
        acc_add(g.ss[psim], ACC_SLOT_RZ + (k + 1) % 3, vals[0]);
        acc_add(g.ss[psim], ACC_SLOT_RR + (k + 1) % 3, vals[1]);
      }
      rz = TV(0);
      rr = TV(0);
    };
    for (int it = 0; it < nitems; ++it) {
      const int item = item0 + it, c = item / NSL, z0 = (item - c * NSL) * KS;
      const int s = sim_of(c);
      if (s_done[s]) continue;
      if (psim >= 0 && psim != s) flush_rz();
      psim = s;
      if (!cached && cs_cube != c) {
        __syncthreads();
        load_cube(csa[0], g, c);
        if (threadIdx.x == 0) cs_cube = c;
        __syncthreads();
      }
      const CubeSh<TV>& cs = csa[cached ? c - cA : 0];
      const TV alpha = TV(s_alpha[s]);
      const size_t base = (size_t)c * B3 + (size_t)z0 * BB;
      const bool plain = cs.smask == 0;
      auto update = [&](int q4, TV (&rv)[4], const TV (&qv)[4]) {
        const int cell = 4 * q4, kk = cell / BB, j = (cell / B) % B, i0 = cell % B;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          rv[e] = rv[e] - alpha * qv[e];
          const TV inv = plain ? cs.invtab[18] : cs.invtab[s3_of<B>(cs.w3, i0 + e, j, z0 + kk)];
          const TV z = rv[e] * inv;
          rz += rv[e] * z;
          rr += rv[e] * rv[e];
        }
        st4(r + base + cell, rv);
      };
      // FP32: four quads per step, all their loads in flight before any use
      constexpr int NQ = KS * BB / 4, STEP = sizeof(TV) == 4 ? 4 : 1;
      for (int q4 = threadIdx.x; q4 < NQ; q4 += STEP * NT) {
        TV ra[4], qa[4];
        ld4(r + base + 4 * q4, ra);
        ld4(q + base + 4 * q4, qa);
        if (STEP == 4 && q4 + 3 * NT < NQ) {
          TV rb[4], qb[4], rc[4], qc[4], rd[4], qd[4];
          ld4(r + base + 4 * (q4 + NT), rb);
          ld4(q + base + 4 * (q4 + NT), qb);
          ld4(r + base + 4 * (q4 + 2 * NT), rc);
          ld4(q + base + 4 * (q4 + 2 * NT), qc);
          ld4(r + base + 4 * (q4 + 3 * NT), rd);
          ld4(q + base + 4 * (q4 + 3 * NT), qd);
          update(q4, ra, qa);
          update(q4 + NT, rb, qb);
          update(q4 + 2 * NT, rc, qc);
          update(q4 + 3 * NT, rd, qd);
        } else {
          update(q4, ra, qa);
          for (int u = 1; u < STEP && q4 + u * NT < NQ; ++u) {
            TV rb[4], qb[4];
            ld4(r + base + 4 * (q4 + u * NT), rb);
            ld4(q + base + 4 * (q4 + u * NT), qb);
            update(q4 + u * NT, rb, qb);
          }
        }
      }
    }
    if (psim >= 0) flush_rz();
    if (!gb.sync()) {
      failed = true;
      break;
    }
  }
  // the last iteration's x += alpha p, on the block's own cells of sims that ran one in
  // this launch; in mixed mode also the defect correction's x64 += e on the cells of
  // sims still correcting (the same update as k_add_correction; each cell has one
  // owner and no block reads x64 before the residual kernel that follows)
  if (!failed) {
    for (int it = 0; it < nitems; ++it) {
      const int item = item0 + it, c = item / NSL, z0 = (item - c * NSL) * KS;
      const int s = sim_of(c), kd = s_kdone[s];
      bool add64 = false;
      if constexpr (sizeof(TX) == 4) add64 = prm.x64_add && !g.ss[s].outer_done;
      if (kd == 0 && !add64) continue;
      const TV alpha = TV(s_alpha[s]);
      const TV* __restrict__ plast = ((kd - 1 + s_poff[s]) & 1) ? p0 : p1;
      const size_t base = (size_t)c * B3 + (size_t)z0 * BB;
      for (int q4 = threadIdx.x; q4 < KS * BB / 4; q4 += NT) {
        TX ev[4];
        ld4(x + base + 4 * q4, ev);
        if (kd > 0) {
          TV pv[4];
          ld4(plast + base + 4 * q4, pv);
#pragma unroll
          for (int m = 0; m < 4; ++m) ev[m] = ev[m] + alpha * pv[m];
          st4(x + base + 4 * q4, ev);
        }
        if constexpr (sizeof(TX) == 4) {
          if (add64) {
            double xv[4];
            ld4(prm.x64_add + base + 4 * q4, xv);
#pragma unroll
            for (int m = 0; m < 4; ++m) xv[m] += double(ev[m]);
            st4(prm.x64_add + base + 4 * q4, xv);
          }
        }
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) g.flags[0] = 1;
}

// ---------------------------------------------------------------- launcher

template <int B, int KS, class TV, class TX>
static cudaError_t pcg_t(const Ctx& x, const SolveParams& prm, TX* xv) {
  constexpr int NT = pcg_threads<B>();
  // tile (16-byte multiple) + alpha, beta, rz (FP64), iterations run (int), done,
  // first, p_off (bytes)
  const size_t tile = (sizeof(TV) * Slab<B, KS>::N + 15) / 16 * 16;
  const size_t sm = tile + (size_t)x.g.n_sims * (3 * sizeof(double) + sizeof(int) + 3);
  auto kern = k_pcg<B, KS, NT, TV, TX>;
  {
    const cudaError_t e = allow_dynamic_smem(kern, sm);
    if (e != cudaSuccess) return e;
  }
  int maxg = 0;
  int rc = max_coresident(kern, NT, sm, &maxg);
  if (rc) return (cudaError_t)rc;
  if (maxg < 1) return cudaErrorCooperativeLaunchTooLarge;
  // every co-resident block takes part: the linear distribution then puts at most
  // ceil(items / maxg) items on a block and evens out the items per SM
  const int items = x.g.n_cubes * (B / KS);
  const int grid = items < maxg ? items : maxg;
  DevGrid gg = x.g;
  TX* xp = xv;
  TV* rp = (TV*)x.f.r;
  TV* p0 = (TV*)x.f.p0;
  TV* p1 = (TV*)x.f.p1;
  TV* qp = (TV*)x.f.q;
  SolveParams pp = prm;
  unsigned int* bar = x.f.bar;
  int* err = x.f.err;
  void* args[] = {&gg, &xp, &rp, &p0, &p1, &qp, &pp, &bar, &err};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(NT), args, sm, x.stream);
}

template <class TV, class TX>
static cudaError_t pcg_dispatch(const Ctx& x, const SolveParams& prm, TX* xv) {
  // slab depth: whole cubes in FP32; half cubes in FP64 (smaller tiles, more blocks)
  switch (x.B) {
    case 4: return pcg_t<4, 4, TV, TX>(x, prm, xv);
    case 8: return pcg_t<8, 8, TV, TX>(x, prm, xv);
    case 16:
      if (x.slabs_p == 2) return pcg_t<16, 8, TV, TX>(x, prm, xv);
      if (x.slabs_p == 4) return pcg_t<16, 4, TV, TX>(x, prm, xv);
      return pcg_t<16, 16, TV, TX>(x, prm, xv);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pcg(const Ctx& x, const SolveParams& prm, int* form) {
  if (x.g.n_sims > kMaxPersistentSims) return cudaErrorInvalidValue;
  // every launch starts its grid barrier's arrival counter at zero
  {
    const cudaError_t e = cudaMemsetAsync(x.f.bar + 32, 0, 32 * sizeof(unsigned int), x.stream);
    if (e != cudaSuccess) return e;
  }
  if (x.fused) {
    bool launched = false;
    const cudaError_t e = launch_pcg_fused(x, prm, &launched);
    if (e != cudaSuccess || launched) {
      *form = PCG_FUSED;
      return e;
    }
  }
  if (x.single_pass) {
    *form = PCG_SINGLE_PASS;
    return launch_pcg1(x, prm);
  }
  if (x.resident && x.slabs_p == 1) {
    bool launched = false;
    const cudaError_t e = launch_pcg_resident(x, prm, &launched);
    if (e != cudaSuccess || launched) {
      *form = PCG_RESIDENT;
      return e;
    }
  }
  *form = PCG_STREAMING;
  return x.solve64 ? pcg_dispatch<double, double>(x, prm, x.f.p)
               : pcg_dispatch<float, float>(x, prm, x.f.e);
}

}  // namespace bcm
