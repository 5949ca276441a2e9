// bcm_pcg_res.cu -- persistent Jacobi-PCG (Eq. poisson; Saad, Alg. 9.1) whose search
// direction stays in shared memory, for grids that fit one co-resident wave of blocks
// holding up to NC cubes each (FP32 inner solve of the mixed-precision solver).
//
// Block b owns a contiguous run of at most NC cubes (the linear load-balanced
// distribution of Eq. loaddist) for the whole solve, and keeps each cube's search
// direction p in a (B+2)^3 shared tile with its face halo, updated in place.  Thread
// (i, j) works on column (i, j) of every cube.  An iteration is
//   pass A, per cube: the column of r and the face-halo values of the neighbours' r
//           and p in one batch of loads; p = M^-1 r + beta p on the tile; q = K p
//           column by column; <p, q>;
//   grid barrier;
//   pass B, per cube: the columns of x and r in one batch of loads; q = K p again from
//           the unchanged tile (the same arithmetic, so the same values); x += alpha p,
//           r -= alpha q, <r, M^-1 r>, <r, r>; x and r back, and p on the cube's face
//           cells, where the neighbours read their halo;
//   grid barrier.
// Compared with the streaming kernel, q is never stored, p is read from and written to
// global memory only on the cube faces, and every pass has one round trip to memory
// per cube instead of one per few cells.  The dot products, rotating slots, per-sim
// decisions and the bounded grid barrier are those of the streaming kernel, whose
// iterates this kernel reproduces up to the summation order of the dot products.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bcm_cube.cuh"
#include "bcm_internal.cuh"
#include "bcm_kernels.h"
#include "bcm_persist.cuh"

namespace bcm {

constexpr int kResCubes = 2;  // cubes per block

template <int B>
constexpr int res_min_blocks() { return B == 16 ? 4 : 8; }

// 1 / diag(K) of cell (i, j, k) of a cube.
template <int B>
__device__ __forceinline__ float own_inv(const CubeSh<float>& cs, int i, int j, int k) {
  return cs.smask == 0 ? cs.invtab[18] : cs.invtab[s3_of<B>(cs.w3, i, j, k)];
}

// 1 / diag(K) of the cell of same-level neighbour f at face position (a, b).
template <int B>
__device__ __forceinline__ float nb_inv(const CubeSh<float>& cs, int f, int a, int b) {
  if (cs.nbmask[f] == 0) return cs.invtab[18];
  const int d = f >> 1;
  int q3[3];
  q3[d] = (f & 1) ? 0 : B - 1;
  q3[tan1(d)] = a;
  q3[tan2(d)] = b;
  return cs.invtab[s3_of<B>(cs.nbw3[f], q3[0], q3[1], q3[2])];
}

// q = K p of cell (i, j, kk) from the tile, marching up the column: below / cur /
// above roll through registers.  fn(kk, p, q) consumes each cell.
template <int B, class Fn>
__device__ __forceinline__ void march_q(const float* __restrict__ T, const CubeSh<float>& cs,
                                        int i, int j, float h, const Fn& fn) {
  using SL = Slab<B, B>;
  constexpr int PP = SL::P * SL::P;
  int o = SL::at(i, j, 1);
  float below = T[o - PP], cur = T[o];
#pragma unroll
  for (int kk = 0; kk < B; ++kk) {
    const float above = T[o + PP];
    float acc = (cur - T[o - 1]) + (cur - T[o + 1]) + (cur - T[o - SL::P]) +
                (cur - T[o + SL::P]) + (cur - below) + (cur - above);
    if (cs.has21) acc = stencil_sum_w<B, float, B>(T, o, cs, i, j, kk);
    fn(kk, cur, h * acc);
    below = cur;
    cur = above;
    o += PP;
  }
}

template <int B, int NC>
__global__ __launch_bounds__(B * B, res_min_blocks<B>()) void k_pcg_res(
    DevGrid g, float* __restrict__ xg, float* __restrict__ rg, float* __restrict__ pg,
    SolveParams prm, unsigned int* bar, int* err) {
  using SL = Slab<B, B>;
  constexpr int NT = B * B, B3 = B * B * B, BB = B * B, TN = (SL::N + 3) / 4 * 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* T0 = reinterpret_cast<float*>(smem_raw);  // NC tiles of TN floats
  double* s_alpha = reinterpret_cast<double*>(T0 + NC * TN);
  const int nsim = g.n_sims;
  double* s_beta = s_alpha + nsim;
  double* s_rz = s_beta + nsim;
  unsigned char* s_done = reinterpret_cast<unsigned char*>(s_rz + nsim);
  unsigned char* s_first = s_done + nsim;
  __shared__ CubeSh<float> csa[NC];
  __shared__ double red[3 * 32];
  const int tid = threadIdx.x, i = tid % B, j = column_row<B>(tid);
  const bool edge = i == 0 || i == B - 1 || j == 0 || j == B - 1;
  const bool inner = prm.mixed != 0;
  const int kmax = inner ? prm.inner_max_iter : prm.max_iter;
  // my cubes: c0 .. c0 + nc - 1 (the launcher makes nc <= NC)
  const int N = g.n_cubes, P = gridDim.x, pb = blockIdx.x;
  const int c0 = pb * (N / P) + min(pb, N % P), nc = (N + P - pb - 1) / P;
  for (int m = 0; m < nc; ++m) load_cube(csa[m], g, c0 + m);
  for (int q = tid; q < nsim; q += NT) {
    const SimState& st = g.ss[q];
    // a kept direction is resumed only from the p buffer this kernel writes
    const bool keep = st.cont != 0 && st.p_off == 0 && st.rz_last != 0.0;
    s_rz[q] = keep ? st.rz_last : st.rz;
    s_done[q] = st.done ? 1 : 0;
    s_first[q] = keep ? 0 : 1;
    s_alpha[q] = 0.0;
    s_beta[q] = 0.0;
  }
  __syncthreads();
  int active = 0;  // bit m: cube m's sim runs in this launch; its tile holds p
  for (int m = 0; m < nc; ++m) {
    const int c = c0 + m, s = g.sim[c];
    if (s_done[s]) continue;
    active |= 1 << m;
    if (!s_first[s]) {
      float* T = T0 + m * TN;
      const size_t col = (size_t)c * B3 + (size_t)j * B + i;
#pragma unroll
      for (int kk = 0; kk < B; ++kk) T[SL::at(i, j, kk + 1)] = pg[col + (size_t)kk * BB];
    }
  }
  // the last direction of a finished cube to global memory (all cells, once)
  auto flush = [&](int m) {
    if (!(active >> m & 1)) return;
    active &= ~(1 << m);
    const float* T = T0 + m * TN;
    const size_t col = (size_t)(c0 + m) * B3 + (size_t)j * B + i;
#pragma unroll
    for (int kk = 0; kk < B; ++kk) pg[col + (size_t)kk * BB] = T[SL::at(i, j, kk + 1)];
  };
  GridBarrier gb;
  gb.init(bar, err, prm.barrier_timeout_ns);
  for (int k = 0;; ++k) {
    // ---- decisions for iteration k (identical in every block)
    int alive = 0;
    for (int q = tid; q < nsim; q += NT) {
      SimState& st = g.ss[q];
      if (s_done[q]) continue;
      double rz, rrs;
      if (k == 0) {
        rz = st.rz;
        rrs = st.rr;
      } else {
        rz = slot_sum(st, ACC_SLOT_RZ + k % 3);
        rrs = slot_sum(st, ACC_SLOT_RR + k % 3);
      }
      const double tol2 = inner ? st.inner_tol2 : st.tol2;
      const bool bad = !isfinite(rrs) || !isfinite(rz);
      if (bad || rrs <= tol2 || k >= kmax) {
        s_done[q] = 1;
        if (blockIdx.x == 0) {  // single writer of the solve's results
          st.iter = k;
          st.total_iters += k;
          st.rr = rrs;
          st.done = 1;
          // the last direction is in the p buffer; none if no iteration ran
          st.rz_last = (k == 0 && s_first[q]) ? 0.0 : s_rz[q];
          st.p_off = 0;
          if (bad) st.nonfinite = 1;
          if (!inner) {
            st.rr64 = rrs;
            st.converged = !bad && rrs <= tol2;
          }
        }
        continue;
      }
      s_beta[q] = ((k == 0 && s_first[q]) || s_rz[q] == 0.0) ? 0.0 : rz / s_rz[q];
      s_rz[q] = rz;
      alive = 1;
    }
    alive = __syncthreads_or(alive);
    for (int m = 0; m < nc; ++m)
      if (s_done[g.sim[c0 + m]]) {
        if (k > 0) flush(m);
        active &= ~(1 << m);  // done before any iteration: p stays as it was
      }
    if (!alive) break;
    if (blockIdx.x == 0)  // clear the slots iteration k+1 fills (held iteration k-2's sums)
      for (int q = tid; q < nsim * kStripes; q += NT) {
        SimState& st = g.ss[q / kStripes];
        const int sp = q % kStripes, sl = (k + 1) % 3;
        st.acc[sp][ACC_SLOT_RZ + sl] = 0.0;
        st.acc[sp][ACC_SLOT_RR + sl] = 0.0;
        st.acc[sp][ACC_SLOT_PQ + sl] = 0.0;
      }
    // ---- pass A, per cube: p = M^-1 r + beta p on the tile, q = K p, <p, q>
    for (int m = 0; m < nc; ++m) {
      const int c = c0 + m, s = g.sim[c];
      const CubeSh<float>& cs = csa[m];
      float* T = T0 + m * TN;
      const bool run = !s_done[s];
      const float beta = float(s_beta[s]);
      const bool first = k == 0 && s_first[s];
      if (run) {
        const size_t col = (size_t)c * B3 + (size_t)j * B + i;
        // one batch: the own column of r and the same-level neighbours' face r, p
        float rv[B], rh[6], ph[6];
#pragma unroll
        for (int kk = 0; kk < B; ++kk) rv[kk] = rg[col + (size_t)kk * BB];
#pragma unroll
        for (int f = 0; f < 6; ++f) {
          rh[f] = 0.f;
          ph[f] = 0.f;
          const int n = cs.nb[f];
          if (n >= 0) {
            const size_t gi = (size_t)n * B3 + cell_of<B>(f >> 1, (f & 1) ? 0 : B - 1, i, j);
            rh[f] = rg[gi];
            if (!first) ph[f] = pg[gi];
          }
        }
#pragma unroll
        for (int kk = 0; kk < B; ++kk) {
          const int o = SL::at(i, j, kk + 1);
          const float z = rv[kk] * own_inv<B>(cs, i, j, kk);
          T[o] = first ? z : z + beta * T[o];
        }
#pragma unroll
        for (int f = 0; f < 6; ++f) {
          const int n = cs.nb[f];
          if (n >= 0) {
            const float z = rh[f] * nb_inv<B>(cs, f, i, j);
            T[ghost_pos<B>(f, i, j)] = first ? z : z + beta * ph[f];
          } else if (n < NB_BOUNDARY) {
            auto valg = [&](int cn, int cell) {
              const size_t gi = (size_t)cn * B3 + cell;
              const float z = rg[gi] * inv_diag_any<B, float>(g, cn, cell);
              return first ? z : z + beta * pg[gi];
            };
            T[ghost_pos<B>(f, i, j)] = poisson_ghost_21<B, float>(g, c, f, i, j, n, valg);
          }
        }
      }
      __syncthreads();
      if (run) {
        // domain faces: the pressure ghost (mirror, or minus the mirror at outflow)
#pragma unroll
        for (int f = 0; f < 6; ++f)
          if (cs.nb[f] == NB_BOUNDARY) {
            const float mv = T[mirror_pos<B>(f, i, j)];
            T[ghost_pos<B>(f, i, j)] = cs.bc[f] == BC_OUTFLOW ? -mv : mv;
          }
      }
      __syncthreads();
      float pq = 0.f;
      if (run) {
        const float h = float(cell_h<B>(g, c));
        march_q<B>(T, cs, i, j, h, [&](int, float p, float qv) { pq += p * qv; });
      }
      const float pp[1] = {pq};
      double vals[1];
      block_sum_tv<NT, 1, float>(pp, vals, red);
      if (tid == 0 && run) acc_add(g.ss[s], ACC_SLOT_PQ + k % 3, vals[0]);
    }
    if (!gb.sync()) break;
    // ---- pass B, per cube: x += alpha p, r -= alpha q, <r, M^-1 r>, <r, r>
    for (int m = 0; m < nc; ++m) {
      const int c = c0 + m, s = g.sim[c];
      const CubeSh<float>& cs = csa[m];
      const float* T = T0 + m * TN;
      const bool run = !s_done[s];
      float rz = 0.f, rs = 0.f;
      if (run) {
        const double pqs = slot_sum(g.ss[s], ACC_SLOT_PQ + k % 3);
        const float alpha = float((pqs != 0.0 && isfinite(pqs)) ? s_rz[s] / pqs : 0.0);
        const size_t col = (size_t)c * B3 + (size_t)j * B + i;
        float xv[B], rv[B];
#pragma unroll
        for (int kk = 0; kk < B; ++kk) {
          xv[kk] = xg[col + (size_t)kk * BB];
          rv[kk] = rg[col + (size_t)kk * BB];
        }
        const float h = float(cell_h<B>(g, c));
        march_q<B>(T, cs, i, j, h, [&](int kk, float p, float qv) {
          const float xn = xv[kk] + alpha * p;
          const float rn = rv[kk] - alpha * qv;
          rz += rn * (rn * own_inv<B>(cs, i, j, kk));
          rs += rn * rn;
          const size_t gi = col + (size_t)kk * BB;
          xg[gi] = xn;
          rg[gi] = rn;
          if (edge || kk == 0 || kk == B - 1) pg[gi] = p;  // the neighbours' halo
        });
      }
      const float pp[2] = {rz, rs};
      double vals[2];
      block_sum_tv<NT, 2, float>(pp, vals, red);
      if (tid == 0 && run) {
        acc_add(g.ss[s], ACC_SLOT_RZ + (k + 1) % 3, vals[0]);
        acc_add(g.ss[s], ACC_SLOT_RR + (k + 1) % 3, vals[1]);
      }
    }
    if (!gb.sync()) break;
  }
  for (int m = 0; m < nc; ++m) flush(m);  // after a timeout: whatever direction is held
  if (blockIdx.x == 0 && tid == 0) g.flags[0] = 1;
}

// ---------------------------------------------------------------- launcher

template <int B>
static cudaError_t pcg_res_t(const Ctx& x, const SolveParams& prm, bool* launched) {
  constexpr int NT = B * B, NC = kResCubes;
  using SL = Slab<B, B>;
  // NC tiles (floats) + alpha, beta, rz (FP64) + done, first (bytes)
  const size_t sm = sizeof(float) * (size_t)NC * ((SL::N + 3) / 4 * 4) +
                    (size_t)x.g.n_sims * (3 * sizeof(double) + 2);
  auto kern = k_pcg_res<B, NC>;
  {
    const cudaError_t e = allow_dynamic_smem(kern, sm);
    if (e != cudaSuccess) return e;
  }
  // the whole unified L1 as shared memory: four blocks of two 16^3 tiles need ~190 KB
  cudaError_t ec = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        (int)cudaSharedmemCarveoutMaxShared);
  if (ec != cudaSuccess) return ec;
  int maxg = 0;
  int rc = max_coresident(kern, NT, sm, &maxg);
  if (rc) return (cudaError_t)rc;
  if (maxg < 1) return cudaSuccess;
  const int per = (x.g.n_cubes + maxg - 1) / maxg;
  if (per > NC) return cudaSuccess;  // more cubes than one co-resident wave holds
  const int grid = x.g.n_cubes < maxg ? x.g.n_cubes : maxg;
  DevGrid gg = x.g;
  float* xp = x.f.e;
  float* rp = (float*)x.f.r;
  float* pp = (float*)x.f.p0;
  SolveParams pr = prm;
  unsigned int* bar = x.f.bar;
  int* err = x.f.err;
  void* args[] = {&gg, &xp, &rp, &pp, &pr, &bar, &err};
  *launched = true;
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(NT), args, sm, x.stream);
}

// The tile-resident PCG when the grid allows it (FP32 inner solve, 16^3 or 8^3 cubes,
// at most kResCubes cubes per co-resident block); *launched says whether it ran.
cudaError_t launch_pcg_resident(const Ctx& x, const SolveParams& prm, bool* launched) {
  *launched = false;
  if (x.solve64 || x.g.n_sims > kMaxPersistentSims || x.g.n_cubes < 1) return cudaSuccess;
  switch (x.B) {
    case 8: return pcg_res_t<8>(x, prm, launched);
    case 16: return pcg_res_t<16>(x, prm, launched);
    default: return cudaSuccess;
  }
}

}  // namespace bcm
