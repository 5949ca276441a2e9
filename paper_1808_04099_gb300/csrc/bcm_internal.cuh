// bcm_internal.cuh -- device-side data structures and helpers of the BCM library.
//
// Data layout in HBM (all inside the caller's workspace):
//   cell fields   cube-major SoA, B^3 values per cube, x fastest (coalesced rows)
//   cube tables   int32 face adjacency [n_cubes*6], 2:1 partners [n_cubes*24],
//                 sim id, level, corner, face Jacobi weights, outflow slots
//   sim tables    SimParams (read-only) and SimState (solver scalars, accumulators)
// Halos are never stored: every stencil kernel stages its cube (or a z-slab of it)
// plus a one-cell face halo in shared memory, reading the halo straight from the
// neighbouring cubes' interiors (Z-ordered cubes keep those reads L2-resident).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bcm.h"

namespace bcm {

constexpr int kMaxBodies = 4;
constexpr int kModes = 8;
constexpr int kW3 = 37;  // sums of face Jacobi weights in thirds (0..36)

enum { BC_WALL = 0, BC_INFLOW = 1, BC_SLIP = 2, BC_OUTFLOW = 3, BC_PERIODIC = 4 };
enum { NB_BOUNDARY = -1, NB_COARSE = -2, NB_FINE = -3 };

// Per-sim constants (written once at grid creation / set_geometry).
struct SimParams {
  double origin[3];
  double h0;          // level-0 cell size
  double hf;          // finest cell size (corner unit)
  double nu, dt, uconv;
  double bcvel[6][3];
  double modes[kModes];
  double L[3];        // domain lengths
  double invdiag[2][kW3];  // 1 / diag(K) per level and face-weight sum (thirds)
  float invdiag32[2][kW3]; // FP32 copy of invdiag (multigrid levels in FP32)
  float h032;              // FP32 copy of h0
  bcm_body bodies[kMaxBodies];
  int n_bodies, has_modes, moving, all_neumann;
  int extent[3];
  int bc[6];
  int cube_begin, cube_end;
  int n_cells;
  int pad;
};

// Accumulators are striped over kStripes cache lines (block index mod kStripes) so
// that thousands of blocks adding into one sim do not serialise on one address.
constexpr int kStripes = 8;
constexpr int kAccPad = 40;  // doubles per stripe (320 bytes)

// Per-sim mutable state (solver scalars and atomic accumulators).
struct SimState {
  double acc[kStripes][kAccPad];  // atomics: see ACC_* below
  double drag_acc[3];
  double drag[3];
  double drag_sum[3];  // sum of the steps' drag since the last reset (bcm_drag_mean)
  int drag_n;          //   and their number
  double bb;           // ||rhs||^2
  double tol2;         // rtol^2 ||rhs||^2 (outer)
  double rz, rr, alpha, beta;
  double inner_tol2;
  double rr64;         // FP64 residual^2 (mixed) / final rr (FP64 mode)
  double bmean;        // volume mean of b (all-Neumann sims)
  double div_num, div_den;
  unsigned long long umax_bits;
  int iter;            // iterations of the running (inner) CG
  int done;            // running CG finished
  int outer_done;      // mixed: defect correction finished
  int cycles;          // mixed: residual evaluations
  int total_iters;     // CG iterations of this solve (summed over cycles)
  int step;            // steps taken (time = step * dt)
  int zero_rhs;        // b == 0: p = 0
  int converged;
  int nonfinite;
  int cont;            // mixed: the next PCG launch continues the previous Krylov sequence
  double rz_last;      // <r,z> before the last iteration of the previous PCG launch
  int p_off;           // buffer offset of the previous launch's last search direction
  int s_off;           // single-pass PCG: buffer offset of the last A p
  double phi_last;     // single-pass PCG: <p, A p> of the last direction
  double cn_d2prev;    // QUICK + Crank-Nicolson: ||update||^2 of the previous iteration
  int cn_iter;         //   iterations of this step's momentum solve
  int cn_done;         //   that solve has converged (or hit its iteration limit)
  int ab2_restart;     // the next Adams-Bashforth step takes N^{n-1} := N^n
  int fz_par;          // fused PCG: face-array parity written by the last pass
  int fz_valid;        //   the last launch of this solve left r, p and faces to resume from
  double fz_rzpred;    //   the <r,z> its last direction was formed with
};

enum { ACC_PQ = 0, ACC_RZ = 1, ACC_RR = 2, ACC_BSUM = 3, ACC_BB = 4, ACC_RR64 = 5,
       ACC_DIVN = 6, ACC_DIVD = 7,
       // persistent PCG: three rotating slots (iteration mod 3) per dot product
       ACC_SLOT_PQ = 8, ACC_SLOT_RZ = 11, ACC_SLOT_RR = 14,
       // single-pass PCG: <r,u>, <w,u>, <u,s_prev>, <r,r>
       ACC_SLOT_G = 8, ACC_SLOT_D = 11, ACC_SLOT_E = 14, ACC_SLOT_R = 17, ACC_NSLOT = 12,
       // QUICK + Crank-Nicolson iteration: ||u^(k+1) - u^(k)||^2, ||u^(k+1)||^2
       ACC_CN_D = 20, ACC_CN_U = 21,
       // fused single-barrier PCG: three rotating slots of <p,q>, <q,z>, <q,D^-1 q>,
       // <r,r>, <r,z>
       ACC_SLOT_FZ = 24, ACC_FZ_N = 5, ACC_FZ_SLOTS = 15 };

// Device view of the grid tables, passed by value to every kernel.
struct DevGrid {
  int n_cubes, n_sims, max_level, two_level;
  const int* __restrict__ nb;     // [6n] same-level id or NB_* code
  const int* __restrict__ aux;    // [24n] coarse id (slot 0) or 4 fine ids
  const int* __restrict__ sim;    // [n]
  const int* __restrict__ lvl;    // [n]
  const int* __restrict__ ijk;    // [3n]
  const int* __restrict__ w3;     // [6n] Jacobi face weight in thirds (0,2,3,4,6)
  const int* __restrict__ nbw3;   // [36n] w3 of each same-level neighbour (3 elsewhere)
  const int* __restrict__ slot;   // [6n] outflow slot or -1
  const unsigned char* __restrict__ near;  // [n] cube may hold phi != 0
  const SimParams* __restrict__ sp;
  SimState* ss;
  unsigned int* counter;          // last-block tickets
  int* flags;                     // [0] every running CG finished, [1] every defect correction finished
  int* check;                     // checked build: code of the first failed index check
};

// Checked build (compiled with -DBCM_CHECK=1): kernels test the cube, sim and cell
// indexes they take from the grid tables before they use them; a failed test records
// its code in DevGrid::check (the first one wins), the access is skipped (a neighbour
// becomes a domain face), and the host reports BCM_E_BOUNDS.  Shared-memory tiles are
// filled with NaN before staging, so a tile value the stencil reads without it having
// been staged turns the result non-finite.  In the default build both are no-ops.
#ifndef BCM_CHECK
#define BCM_CHECK 0
#endif
enum { CHK_CUBE = 1, CHK_SIM = 2, CHK_NEIGHBOUR = 3, CHK_LEVEL = 4, CHK_AUX = 5, CHK_CELL = 6 };
__device__ __forceinline__ bool bcm_expect(const DevGrid& g, bool ok, int code) {
#if BCM_CHECK
  if (!ok) atomicCAS(g.check, 0, code);
  return ok;
#else
  (void)g;
  (void)code;
  return true;
#endif
}
// A face-table entry n of cube c (same-level id, or NB_* code), checked: an id outside
// the grid, or a 2:1 code on a single-level grid, comes back as NB_BOUNDARY.
__device__ __forceinline__ int checked_nb(const DevGrid& g, int n) {
  const bool ok = (n >= 0 && n < g.n_cubes) || n == NB_BOUNDARY ||
                  (g.max_level > 0 && (n == NB_COARSE || n == NB_FINE));
  return bcm_expect(g, ok, CHK_NEIGHBOUR) ? n : NB_BOUNDARY;
}
// NaN into the n values of a tile before it is staged (checked build only).
template <class T>
__device__ __forceinline__ void poison_tile(T* S, int n) {
#if BCM_CHECK
  for (int i = threadIdx.x; i < n; i += blockDim.x) S[i] = T(__int_as_float(0x7fc00000));
  __syncthreads();
#else
  (void)S;
  (void)n;
#endif
}

__host__ __device__ __forceinline__ int tan1(int d) { return d == 0 ? 1 : 0; }
__host__ __device__ __forceinline__ int tan2(int d) { return d == 2 ? 1 : 2; }

// ---------------------------------------------------------------- geometry

template <int B>
__device__ __forceinline__ double cell_h(const DevGrid& g, int c) {
  return g.sp[g.sim[c]].h0 / double(1 << g.lvl[c]);
}

template <int B>
__device__ __forceinline__ int cell_span(const DevGrid& g, int c) {
  return 1 << (g.max_level - g.lvl[c]);
}

// Physical coordinate of cell index n (halo indices allowed) of cube c along axis e.
template <int B>
__device__ __forceinline__ double centre(const DevGrid& g, int c, int e, int n) {
  const SimParams& p = g.sp[g.sim[c]];
  return p.origin[e] + g.ijk[3 * c + e] * p.hf + (n + 0.5) * cell_h<B>(g, c);
}

// Inflow profile factor 1 + sum a_m sin(k pi s/Ls) sin(l pi t/Lt) on face f of cube c.
template <int B>
__device__ double inflow_profile(const DevGrid& g, int c, int f, int a, int b) {
  const int mk[kModes] = {1, 1, 2, 2, 1, 3, 2, 3};
  const int ml[kModes] = {1, 2, 1, 2, 3, 1, 3, 2};
  const SimParams& p = g.sp[g.sim[c]];
  int d = f >> 1, e1 = tan1(d), e2 = tan2(d);
  double y = centre<B>(g, c, e1, a) - p.origin[e1];
  double z = centre<B>(g, c, e2, b) - p.origin[e2];
  double prof = 1.0;
  for (int m = 0; m < kModes; ++m)
    prof += p.modes[m] * sin(mk[m] * M_PI * y / p.L[e1]) * sin(ml[m] * M_PI * z / p.L[e2]);
  return prof;
}

// Wall / inflow velocity component comp on face f of cube c at tangential (a, b).
template <int B>
__device__ __forceinline__ double face_velocity(const DevGrid& g, int c, int f, int comp, int a,
                                                int b) {
  const SimParams& p = g.sp[g.sim[c]];
  double w = p.bcvel[f][comp];
  if (p.bc[f] == BC_INFLOW && p.has_modes) w *= inflow_profile<B>(g, c, f, a, b);
  return w;
}

// Cell index of (normal index n along d, tangential a, b).
template <int B>
__device__ __forceinline__ int cell_of(int d, int n, int a, int b) {
  int q[3];
  q[d] = n;
  q[tan1(d)] = a;
  q[tan2(d)] = b;
  return (q[2] * B + q[1]) * B + q[0];
}

// ----------------------------------------------------------------- halo value
//
// Value of the ghost cell at distance layer+1 outside face f of cube c, tangential
// (a, b), by the halo rules of the paper ("Building Cube Method"):
//   same level: copy of the neighbour's boundary interior cell;
//   coarse neighbour (this cube fine): the coarse cell covering the ghost (injection);
//   fine neighbours (this cube coarse): mean of the 2x2x2 fine cells it covers;
//   domain face: bc(f, a, b, mirror interior value).
// val(cube, cell) returns the interior value of any cube.
template <int B, class T, class Val, class Bc>
__device__ __forceinline__ T halo_value(const DevGrid& g, int c, int f, int a, int b, int layer,
                                        const Val& val, const Bc& bc) {
  const int d = f >> 1, side = f & 1;
  const int n = checked_nb(g, g.nb[6 * c + f]);
  if (n >= 0) return val(n, cell_of<B>(d, side ? layer : B - 1 - layer, a, b));
  if (n == NB_BOUNDARY)
    return bc(f, a, b, val(c, cell_of<B>(d, side ? B - 1 - layer : layer, a, b)));
  if (n == NB_COARSE) {
    const int C = g.aux[(6 * c + f) * 4];
    if (!bcm_expect(g, C >= 0 && C < g.n_cubes, CHK_AUX)) return T(0);
    const int sf = 1 << (g.max_level - g.lvl[c]), sc = 2 * sf;
    const int A = (g.ijk[3 * c + tan1(d)] + a * sf - g.ijk[3 * C + tan1(d)]) / sc;
    const int Bb = (g.ijk[3 * c + tan2(d)] + b * sf - g.ijk[3 * C + tan2(d)]) / sc;
    if (!bcm_expect(g, A >= 0 && A < B && Bb >= 0 && Bb < B, CHK_CELL)) return T(0);
    return val(C, cell_of<B>(d, side ? 0 : B - 1, A, Bb));
  }
  // NB_FINE
  const int qa = (2 * a) / B, qb = (2 * b) / B;
  const int F = g.aux[(6 * c + f) * 4 + qb * 2 + qa];
  if (!bcm_expect(g, F >= 0 && F < g.n_cubes, CHK_AUX)) return T(0);
  const int fa = 2 * a - qa * B, fb = 2 * b - qb * B;
  T sum = T(0);
  for (int l2 = 0; l2 < 2; ++l2) {
    const int fn = side ? 2 * layer + l2 : B - 1 - 2 * layer - l2;
    for (int bb = 0; bb < 2; ++bb)
      for (int aa = 0; aa < 2; ++aa) sum += val(F, cell_of<B>(d, fn, fa + aa, fb + bb));
  }
  return T(0.125) * sum;
}

// ---------------------------------------------------------------- slab staging
//
// A CTA owns planes [z0, z0+KS) of one cube.  Shared memory holds those planes
// plus one plane below and above, each (B+2)^2 with a one-cell x/y ring.  Edge and
// corner ring cells are never read by the 7-point stencils and stay unset.
template <int B, int KS>
struct Slab {
  static constexpr int P = B + 2;
  static constexpr int N = (KS + 2) * P * P;
  __device__ __forceinline__ static int at(int i, int j, int kk) {
    return (kk * P + (j + 1)) * P + (i + 1);
  }
};

template <int B, int KS, int NT, class T, class Val, class Bc>
__device__ __forceinline__ void stage_slab(T* __restrict__ S, const DevGrid& g, int c, int z0,
                                           const Val& val, const Bc& bc) {
  using SL = Slab<B, KS>;
  constexpr int BB = B * B;
  poison_tile(S, SL::N);
  for (int idx = threadIdx.x; idx < (KS + 2) * BB; idx += NT) {
    const int kk = idx / BB, rem = idx - kk * BB, j = rem / B, i = rem - j * B;
    const int k = z0 - 1 + kk;
    T v;
    if (k < 0) v = halo_value<B, T>(g, c, 4, i, j, 0, val, bc);
    else if (k >= B) v = halo_value<B, T>(g, c, 5, i, j, 0, val, bc);
    else v = val(c, (k * B + j) * B + i);
    S[SL::at(i, j, kk)] = v;
  }
  for (int idx = threadIdx.x; idx < 4 * KS * B; idx += NT) {
    const int f = idx / (KS * B), rem = idx - f * (KS * B), kk = rem / B, t = rem - kk * B;
    const int k = z0 + kk;
    const T v = halo_value<B, T>(g, c, f, t, k, 0, val, bc);
    if (f < 2) S[SL::at(f == 0 ? -1 : B, t, kk + 1)] = v;
    else S[SL::at(t, f == 2 ? -1 : B, kk + 1)] = v;
  }
}

// --------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block of NV doubles per thread; result valid in thread 0.
template <int NT, int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) red[q * 32 + warp] = v[q];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double x = lane < NT / 32 ? red[q * 32 + lane] : 0.0;
      v[q] = warp_sum(x);
    }
  }
}

// The same for NV partial sums held in the vector type TV: FP32 partials are summed in
// FP32 within each warp (this part's FP64 rate is a small fraction of its FP32 rate,
// and the warp sums are what every block reaches the grid barrier with) and in FP64
// across the warps; FP64 partials as block_sum.  Result (FP64) valid in thread 0.
template <int NT, int NV, class TV>
__device__ __forceinline__ void block_sum_tv(const TV (&p)[NV], double (&v)[NV], double* red) {
  if constexpr (sizeof(TV) == 8) {
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = double(p[q]);
    block_sum<NT, NV>(v, red);
  } else {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float f[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      f[q] = float(p[q]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) f[q] += __shfl_xor_sync(0xffffffffu, f[q], o);
    }
    __syncthreads();
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < NV; ++q) red[q * 32 + warp] = double(f[q]);
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        double x = lane < NT / 32 ? red[q * 32 + lane] : 0.0;
        v[q] = warp_sum(x);
      }
    }
  }
}

// Last-block election: every block must call this exactly once per launch, after its
// thread 0 has issued the block's accumulator atomics.  The ticket is two-level: a
// block takes a ticket on one of kTickets striped counters (block index mod
// kTickets), the last block of each stripe takes one on the top counter, and the
// last of those is the last block.  One shared counter would serialise every block
// of the launch on a single L2 address.  Counters reset themselves.  Only thread 0
// fences: the last block reads nothing but the accumulators, so the other threads'
// stores need not be visible to it (the next kernel sees them at the launch boundary).
constexpr int kTickets = 32;
constexpr int kTicketWords = 32 * (1 + kTickets);  // one 128-byte line per counter

__device__ __forceinline__ bool last_block(unsigned int* counter) {
  __shared__ int is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int nblk = gridDim.x;
    const unsigned int stripe = blockIdx.x % kTickets;
    const unsigned int in_stripe = (nblk - stripe + kTickets - 1) / kTickets;
    const unsigned int t = atomicAdd(&counter[32 * (1 + stripe)], 1u);
    int last = 0;
    if (t == in_stripe - 1) {
      counter[32 * (1 + stripe)] = 0u;
      __threadfence();
      const unsigned int stripes = nblk < (unsigned)kTickets ? nblk : (unsigned)kTickets;
      const unsigned int u = atomicAdd(&counter[0], 1u);
      if (u == stripes - 1) {
        counter[0] = 0u;
        last = 1;
        __threadfence();
      }
    }
    is_last = last;
  }
  __syncthreads();
  return is_last != 0;
}

__device__ __forceinline__ double ld_acc(const double* p) { return __ldcg(p); }

// Add v to accumulator idx of a sim (this block's stripe).
__device__ __forceinline__ void acc_add(SimState& st, int idx, double v) {
  atomicAdd(&st.acc[blockIdx.x % kStripes][idx], v);
}
// Sum of accumulator idx over the stripes, which are reset to zero (last block only).
__device__ __forceinline__ double acc_take(SimState& st, int idx) {
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kStripes; ++q) {
    s += ld_acc(&st.acc[q][idx]);
    st.acc[q][idx] = 0.0;
  }
  return s;
}

}  // namespace bcm
