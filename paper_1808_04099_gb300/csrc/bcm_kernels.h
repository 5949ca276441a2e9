// bcm_kernels.h -- host-side launch interface of the BCM kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bcm_internal.cuh"

namespace bcm {

// Constants of one cube for the fused PCG, built on the host at grid creation: a
// 432-byte record (a multiple of 16 bytes) that reaches shared memory by one bulk copy
// beside the cube's vectors.
struct alignas(16) FCube {
  int nb[6];          // face neighbours / NB_* codes
  int w3[6];          // Jacobi face weights (thirds) of this cube
  int nbw3[6][6];     // ... of each same-level neighbour (3 elsewhere)
  int nbmask[6];      // bit e: face e of neighbour f has a weight other than 3
  int bc[6];          // the sim's domain-face conditions
  int smask;          // bit f: face f's weight is not the same-level 3
  int has21;          // some face is a 2:1 level interface
  int sim, lvl;
  float wt[6];        // flux weight of face f relative to a same-level face (R7)
  float invtab[kW3];  // 1 / diag(K) by face-weight sum
  float h;            // cell size
};
static_assert(sizeof(FCube) % 16 == 0, "FCube must be a whole number of 16-byte units");

// Device pointers of every field and solver vector (all inside the workspace).
struct Fields {
  void *u, *v, *w, *us, *vs, *ws, *nx, *ny, *nz, *phi, *ub;  // state storage type
  double *p, *b;                                              // FP64 always
  unsigned char *bid, *near;
  void *r, *p0, *p1, *q;  // PCG vectors: FP64 (plain) or FP32 (mixed inner)
  void *w1, *s0, *s1;     // single-pass PCG: second A u buffer and the two A p buffers
  float *e;               // mixed: inner iterate (correction of p)
  float *face;            // fused PCG: [2][n_cubes][6][3][B^2] face planes of r, q, p
  const FCube* fcube;     // fused PCG: per-cube constants [n_cubes]
  unsigned int* guard;    // graph-loop body counter
  unsigned int* bar;      // persistent PCG grid barrier words
  int* err;               // persistent PCG: a barrier wait timed out
};

struct SolveParams {
  double rtol;            // outer (FP64) relative residual target
  double inner_rtol;      // mixed: inner FP32 PCG relative reduction per cycle
  int max_iter;           // FP64 mode: PCG iterations
  int inner_max_iter;     // mixed: inner iterations per cycle
  int max_cycles;         // mixed: defect-correction cycles
  int mixed;
  unsigned long long cond_inner, cond_outer;  // graph conditional handles (0 = none)
  unsigned int* guard;
  int guard_limit;
  int mg;                 // 1: the multigrid preconditioner supplies z (pass A reads it;
                          // the V-cycle's last launch takes the iteration's decisions)
  unsigned long long barrier_timeout_ns;  // persistent PCG: longest wait at a grid barrier
  int recycle;            // mixed + persistent: keep the search direction across cycles
  int pad2;
  // multigrid PCG inside a captured step: body executions of the inner and the outer
  // loop, counted on the device for the launch count ([0], [1]; cumulative)
  unsigned int* body_count;
  // mixed mode, streaming persistent PCG: the FP64 iterate the kernel adds its FP32
  // correction e to at the end of the inner solve (x64 += e, the defect correction's
  // update; the separate k_add_correction launch is then left out), or NULL
  double* x64_add;
};

// Geometric multigrid preconditioner (single-level grids): per-cube levels
// l = 0 .. L (cells per cube edge B >> l) and cube-aggregate levels k = 0 .. M-1
// (aggregate level m = k + 1; k = 0 aggregates cubes).  Per-cube level arrays are in
// the PCG vector type, aggregate arrays in FP64.
constexpr int kMgMaxL = 4;   // log2 of the largest cube edge (16)
constexpr int kMgMaxM = 20;  // aggregate levels
constexpr double kMgOmega = 0.8;  // damped-Jacobi weight of the smoother
constexpr int kMgNuTop = 4;       // Jacobi sweeps on the top aggregate level
constexpr double kMgOver = 1.75;  // scale of the coarse-grid correction
struct MgDev {
  int L, M;
  void* x[kMgMaxL + 1];  // pre-smoothed iterate of level l
  void* y[kMgMaxL + 1];  // corrected iterate of level l (y[0] = z, the PCG's M^-1 r)
  void* r[kMgMaxL + 1];  // residual of level l (r[0] is the PCG residual)
  void* rr;              // level L: residual after pre-smoothing, one value per cube
  int n[kMgMaxM];        // nodes of aggregate level k
  int nnz[kMgMaxM];      // off-diagonal entries of level k
  double *ar[kMgMaxM], *ax[kMgMaxM], *at[kMgMaxM];  // residual, iterate, scratch
  double *diag[kMgMaxM], *val[kMgMaxM];              // K: diagonal, -off-diagonal (CSR)
  int *row[kMgMaxM], *col[kMgMaxM];
  int *cptr[kMgMaxM], *cidx[kMgMaxM];  // children: level k-1 nodes (cubes for k = 0)
  int *parent[kMgMaxM];                // parent at level k of each level k-1 node
};

// Lagrangian particles of the immersed boundary (n = 0: the solid-fraction IB).
// Arrays live in a caller-provided workspace (bcm_set_particles).
struct PartDev {
  int n;
  double* X;        // [3n] positions, xyz interleaved
  double* F;        // [3n] force per particle of the last step (rho = 1)
  const int* sim;   // [n] sim of each particle
  const int* body;  // [n] body (of its sim) that moves it
  const double* dV; // [n] volume weight dc1 dc2 dc3
  int* cube;        // [n] cube containing the particle (-1: outside every cube)
  int* set_start;   // [n_cubes + 1] per-cube sets: particles of cube c are
  int* set_ids;     //   set_ids[set_start[c] .. set_start[c+1])
  int* set_count;   // [n_cubes] scratch: counts, then fill cursors
  const int* lat;   // cube lattice: cube id at (sim, cube coordinates), -1 none
  const int* lat_meta;  // [n_sims][4]: offset into lat, cubes along x, y, z
  int* err;         // set when a particle lies outside every cube
};

struct Ctx {
  DevGrid g;
  Fields f;
  int B;
  int f64;      // state in FP64 (plain mode) or FP32 (mixed mode)
  int solve64;  // pressure solve: FP64 PCG (1) or FP32 inner PCG in FP64 defect correction
  int slabs_a;  // PCG pass A: z-slabs per cube (1, 2 or 4)
  int slabs_b;  // PCG pass B: z-slabs per cube (1, 2 or 4)
  int slabs_p;  // persistent PCG: z-slabs per cube (1, 2 or 4)
  int persistent;  // 1: one cooperative launch per PCG solve; 0: two launches per iteration
  int single_pass; // persistent PCG: one pass and one grid barrier per iteration
  int resident;    // persistent PCG: search direction in shared memory where it fits
  int fused;       // persistent PCG: the single-barrier form with bulk-copy staging
  int slabs_m;     // momentum and right-hand side: z-slabs per 16^3 cube (0: default)
  int lag_bf16;    // mixed mode: N^{n-1} stored as bfloat16
  int use_mg;      // PCG preconditioner: 0 Jacobi, 1 geometric multigrid
  MgDev mg;
  PartDev part;    // Lagrangian particles (part.n > 0: particle IB, no solid fraction)
  int scheme;       // momentum: 0 Adams-Bashforth + central, 1 QUICK + Crank-Nicolson
  double cn_rtol;   // Crank-Nicolson iteration: relative update at which a sim stops
  int cn_max;       //   and its iteration limit per step
  cudaStream_t stream;
};

cudaError_t launch_solid_fraction(const Ctx& x, int sim_filter);
cudaError_t launch_momentum(const Ctx& x);
// QUICK + Crank-Nicolson momentum: explicit half and outflow update, one iteration of
// the implicit half (sims that converged return at once), IB forcing of the result.
cudaError_t launch_cn_explicit(const Ctx& x);
cudaError_t launch_cn_iter(const Ctx& x);
cudaError_t launch_cn_finish(const Ctx& x);
cudaError_t launch_rhs(const Ctx& x);
cudaError_t launch_bmean(const Ctx& x);
cudaError_t launch_solve_begin(const Ctx& x);
cudaError_t launch_residual(const Ctx& x, const SolveParams& prm);
cudaError_t launch_cg_a(const Ctx& x, const SolveParams& prm);
cudaError_t launch_cg_b(const Ctx& x, const SolveParams& prm);
// PCG forms (reported in bcm_stats.pcg_form)
enum { PCG_TWO_LAUNCH = 0, PCG_STREAMING = 1, PCG_SINGLE_PASS = 2, PCG_RESIDENT = 3,
       PCG_MULTIGRID = 4, PCG_FUSED = 5 };
// The persistent PCG in the form the launch shape and the grid select; *form gets it.
cudaError_t launch_pcg(const Ctx& x, const SolveParams& prm, int* form);
cudaError_t launch_pcg1(const Ctx& x, const SolveParams& prm);
cudaError_t launch_pcg_resident(const Ctx& x, const SolveParams& prm, bool* launched);
// The fused single-barrier form (FP32 inner solve, 16^3 cubes); *launched = false when
// the grid does not fit it (the caller falls back to the streaming form).
cudaError_t launch_pcg_fused(const Ctx& x, const SolveParams& prm, bool* launched);
cudaError_t launch_add_correction(const Ctx& x);
cudaError_t launch_correct(const Ctx& x);
cudaError_t launch_step_end(const Ctx& x);
cudaError_t launch_fill_halo(const Ctx& x, const void* f, int f64_field, int kind, double* out);
cudaError_t launch_apply_poisson(const Ctx& x, const double* in, double* out);
// One V-cycle z = M^-1 r on the PCG residual.  mode 0: after the residual kernel
// (<r,z> becomes the PCG's rz); 1: after pass A, doing pass B too (<r,r>), then <r,z>,
// beta and the convergence decision; 2: standalone (every sim, no dot products).
cudaError_t launch_mg_vcycle(const Ctx& x, const SolveParams& prm, int mode);
// Lagrangian particles: per-cube sets from the positions (counting sort); the
// forcing sub-step (interpolation of u~, F, spreading into u*); the position update.
cudaError_t launch_ib_bin(const Ctx& x);
cudaError_t launch_ib_force(const Ctx& x);
cudaError_t launch_ib_move(const Ctx& x);
// wavelet compression of a cell field (bcm_wavelet.cu): codes, Rice parameters and
// record offsets; the encoded stream (zeroed beforehand); decoding into the field
cudaError_t launch_wavelet_analyze(const Ctx& x, const void* field, int f64, double step,
                                   uint32_t* zc, uint32_t* cube_nbits, uint32_t* cube_k,
                                   uint32_t* off, int* err);
cudaError_t launch_wavelet_encode(const Ctx& x, const uint32_t* zc, const uint32_t* cube_nbits,
                                  const uint32_t* cube_k, const uint32_t* off, double step,
                                  uint32_t* out);
// max_payload: the largest payload (words after a record's first) among the records
cudaError_t launch_wavelet_decode(const Ctx& x, void* field, int f64, const uint32_t* in,
                                  size_t words, uint32_t max_payload, double step, uint32_t* off,
                                  int* err);
// test paths on FP64 arrays: out[q] = I[f] at particle q; out += P[F]
cudaError_t launch_ib_interpolate(const Ctx& x, const double* f, double* out);
cudaError_t launch_ib_spread(const Ctx& x, const double* F, double* out);

}  // namespace bcm
