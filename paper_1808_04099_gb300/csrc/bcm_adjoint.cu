// bcm_adjoint.cu -- discrete adjoint of one fractional step (FP64), for gradients of
// the time-averaged drag with respect to the inflow-profile amplitudes and the
// centre of a fixed sphere.
//
// The forward step (section "Numerical algorithm", with the readings of the library):
//   u~  = u + dt (-(c1 N(u) + c0 N_prev) + nu L u)        c1 = 3/2, c0 = -1/2 (first: 1, 0)
//   u*  = u~ + phi (u_s - u~)                              u_s = 0 (fixed body)
//   F_x = sum phi u~_x V / dt                              drag of the step, weight w in J
//   ub' = (1 - kappa) ub + kappa u_0                       kappa = 2 U_c dt / h (outflow)
//   b   = (1/(h dt)) D(u*, ub', a);  K p = -V b;  u' = u* - dt G_c p
// is reversed here with exact transposes of every discrete operator, boundary ghost
// included: a ghost g = alpha u_0 + beta sends its adjoint back to the interior cell
// (alpha), to the outflow face state (beta = 2 ub) or to the inflow amplitudes
// (beta = 2 U (1 + sum a_m s_m)).  K is symmetric, so the adjoint Poisson solve is the
// same Jacobi-PCG.  Single-level grids; bodies: fixed spheres.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "../../include/bcm.h"
#include "bcm_internal.cuh"
#include "bcm_kernels.h"

namespace bcm {
const Ctx* grid_ctx(const bcm_grid* g);
int grid_two_level(const bcm_grid* g);
cudaStream_t grid_stream(const bcm_grid* g);
bcm_status grid_fail(bcm_status st, const char* msg);
}  // namespace bcm

using namespace bcm;

namespace {

constexpr int kNT = 256;

// Adjoint workspace (FP64, n cells each): the 3-vectors carry components x, y, z.
struct AdjFields {
  double *lu[3];      // lambda of u^{n+1} on entry, of u^n on exit
  double *lus[3];     // lambda of u*
  double *lut[3];     // lambda of u~
  double *lN[3];      // lambda of N^n (total)
  double *lNn[3];     // carried 0.5 dt lambda_u~ for the previous step's N
  double *lp, *mu, *bsc;  // lambda of p, adjoint pressure, solve right-hand side
  double *lub, *lub2;     // lambda of the outflow face state (ping-pong)
  double *cg[4];          // FP64 CG vectors of the adjoint Poisson solve
  double *acc;            // [11] FP64 gradient accumulators (caller's dJ): 8 inflow
                          // amplitudes, sphere centre (x, y, z)
};

size_t adj_layout(size_t n, size_t nub, AdjFields* F, unsigned char* base) {
  size_t off = 0;
  auto take = [&](size_t cnt) {
    double* p = base ? (double*)(base + off) : nullptr;
    off += (cnt * sizeof(double) + 255) / 256 * 256;
    return p;
  };
  AdjFields f{};
  for (int c = 0; c < 3; ++c) f.lu[c] = take(n);
  for (int c = 0; c < 3; ++c) f.lus[c] = take(n);
  for (int c = 0; c < 3; ++c) f.lut[c] = take(n);
  for (int c = 0; c < 3; ++c) f.lN[c] = take(n);
  for (int c = 0; c < 3; ++c) f.lNn[c] = take(n);
  f.lp = take(n);
  f.mu = take(n);
  f.bsc = take(n);
  f.lub = take(nub ? nub : 1);
  f.lub2 = take(nub ? nub : 1);
  for (int c = 0; c < 4; ++c) f.cg[c] = take(n);
  if (F) *F = f;
  return off;
}

// ----------------------------------------------------------- cell helpers

template <int B>
struct Cell {
  int c, i, j, k;
  __device__ int q() const { return (k * B + j) * B + i; }
};

// Same-level neighbour across face f, or -1 at a domain face.
template <int B>
__device__ __forceinline__ int nb_index(const DevGrid& g, const Cell<B>& x, int f, int* cell) {
  const int d = f >> 1, side = f & 1;
  int ii[3] = {x.i, x.j, x.k};
  ii[d] += side ? 1 : -1;
  if (ii[d] >= 0 && ii[d] < B) {
    *cell = (ii[2] * B + ii[1]) * B + ii[0];
    return x.c;
  }
  const int n = g.nb[6 * x.c + f];
  if (n < 0) return -1;
  ii[d] = side ? 0 : B - 1;
  *cell = (ii[2] * B + ii[1]) * B + ii[0];
  return n;
}

// tangential coordinates (a, b) of a cell on face f
template <int B>
__device__ __forceinline__ void face_ab(const Cell<B>& x, int f, int* a, int* b) {
  const int d = f >> 1;
  const int ii[3] = {x.i, x.j, x.k};
  *a = ii[tan1(d)];
  *b = ii[tan2(d)];
}

// Velocity ghost rule g = alpha u_0 + beta at a domain face (component e): alpha.
__device__ __forceinline__ double ghost_alpha(int bc, int f, int e) {
  if (bc == BC_SLIP) return (e == (f >> 1)) ? -1.0 : 1.0;
  return -1.0;
}

// d beta / d a_m of an INFLOW face ghost (component e) at tangential (a, b): 2 w_e s_m.
template <int B>
__device__ void inflow_dbeta(const DevGrid& g, int c, int f, int e, int a, int b, double* out8) {
  const int mk[kModes] = {1, 1, 2, 2, 1, 3, 2, 3};
  const int ml[kModes] = {1, 2, 1, 2, 3, 1, 3, 2};
  const SimParams& p = g.sp[g.sim[c]];
  const int d = f >> 1, e1 = tan1(d), e2 = tan2(d);
  const double y = centre<B>(g, c, e1, a) - p.origin[e1];
  const double z = centre<B>(g, c, e2, b) - p.origin[e2];
  for (int m = 0; m < kModes; ++m)
    out8[m] = 2.0 * p.bcvel[f][e] * sin(mk[m] * M_PI * y / p.L[e1]) * sin(ml[m] * M_PI * z / p.L[e2]);
}

// Velocity value of component e at the ghost across domain face f of cell x.
template <int B>
__device__ double ghost_value(const DevGrid& g, const Cell<B>& x, int f, int e, double u0,
                              const double* ub) {
  const SimParams& p = g.sp[g.sim[x.c]];
  const int bc = p.bc[f];
  int a, b;
  face_ab<B>(x, f, &a, &b);
  if (bc == BC_SLIP) return ghost_alpha(bc, f, e) * u0;
  if (bc == BC_OUTFLOW)
    return 2.0 * ub[((size_t)(g.slot[6 * x.c + f] * 3 + e) * B + b) * B + a] - u0;
  return 2.0 * face_velocity<B>(g, x.c, f, e, a, b) - u0;
}

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// add per-thread gradient contributions into the FP64 accumulators (one atomic per warp)
__device__ __forceinline__ void flush_grad(double* acc, const double* v, int n) {
  for (int m = 0; m < n; ++m) {
    const double s = warp_sum_d(v[m]);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(&acc[m], s);
  }
}

// ===========================================================================
// A1: lambda_u* = lambda_u'; lambda_p = -dt G_c^T lambda_u'
// ===========================================================================
template <int B>
__global__ __launch_bounds__(kNT) void k_adj_projection(DevGrid g, AdjFields F) {
  constexpr int B3 = B * B * B;
  const size_t gid = (size_t)blockIdx.x * kNT + threadIdx.x;
  if (gid >= (size_t)g.n_cubes * B3) return;
  Cell<B> x{(int)(gid / B3), (int)(gid % B), (int)((gid / B) % B), (int)((gid / (B * B)) % B)};
  const SimParams& p = g.sp[g.sim[x.c]];
  const double h = p.h0 / double(1 << g.lvl[x.c]);
  double gt = 0.0;  // (G_c^T lambda)(j)
  for (int d = 0; d < 3; ++d) {
    const double lj = F.lu[d][gid];
    F.lus[d][gid] = lj;
    for (int side = 0; side < 2; ++side) {
      const int f = 2 * d + side;
      int cell;
      const int n = nb_index<B>(g, x, f, &cell);
      if (n >= 0) {
        const double ln = F.lu[d][(size_t)n * B3 + cell];
        gt += side ? -ln : ln;  // j is the - neighbour of the cell above, + of the one below
      } else {
        const double ap = p.bc[f] == BC_OUTFLOW ? -1.0 : 1.0;  // pressure ghost alpha
        gt += side ? ap * lj : -ap * lj;
      }
    }
  }
  F.lp[gid] = -p.dt * gt / (2.0 * h);
}

// ===========================================================================
// A3: lambda_b = -V mu;  lambda_u* += D^T lambda_b / (h dt); inflow faces -> dJ/da;
//     outflow faces -> lambda of the new face state
// ===========================================================================
template <int B>
__global__ __launch_bounds__(kNT) void k_adj_rhs(DevGrid g, AdjFields F) {
  constexpr int B3 = B * B * B;
  const size_t gid = (size_t)blockIdx.x * kNT + threadIdx.x;
  double ga[kModes] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (gid < (size_t)g.n_cubes * B3) {
    Cell<B> x{(int)(gid / B3), (int)(gid % B), (int)((gid / B) % B), (int)((gid / (B * B)) % B)};
    const SimParams& p = g.sp[g.sim[x.c]];
    const double h = p.h0 / double(1 << g.lvl[x.c]);
    const double V = h * h * h, s = 1.0 / (h * p.dt);
    const double lbj = -V * F.mu[gid];
    for (int d = 0; d < 3; ++d) {
      double acc = 0.0;
      for (int side = 0; side < 2; ++side) {
        const int f = 2 * d + side;
        int cell;
        const int n = nb_index<B>(g, x, f, &cell);
        if (n >= 0) {
          const double lbn = -V * F.mu[(size_t)n * B3 + cell];
          acc += side ? 0.5 * (lbj - lbn) : 0.5 * (lbn - lbj);
        } else {
          const int bc = p.bc[f];
          int a, b;
          face_ab<B>(x, f, &a, &b);
          const double sgn = side ? s : -s;  // d b / d U_face
          if (bc == BC_OUTFLOW) {
            atomicAdd(&F.lub[((size_t)(g.slot[6 * x.c + f] * 3 + d) * B + b) * B + a],
                      sgn * lbj);
          } else if (bc == BC_INFLOW) {  // the amplitudes matter even where they are 0
            double dbeta[kModes];
            inflow_dbeta<B>(g, x.c, f, d, a, b, dbeta);
            for (int m = 0; m < kModes; ++m) ga[m] += sgn * lbj * 0.5 * dbeta[m];  // U = beta/2
          }
        }
      }
      F.lus[d][gid] += s * acc;
    }
  }
  flush_grad(F.acc, ga, kModes);
}

// Sphere signed distance gradient: d phi / d c for phi = (1 - tanh(d/eps))/2, d = |x-c| - R.
__device__ __forceinline__ void dphi_dc(const double* xc, const bcm_body& bd, double eps,
                                        double* out) {
  double r[3] = {xc[0] - bd.center[0], xc[1] - bd.center[1], xc[2] - bd.center[2]};
  const double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  const double d = rn - bd.axes[0];
  out[0] = out[1] = out[2] = 0.0;
  if (!(d < 20.0 * eps) || rn == 0.0) return;
  const double t = tanh(d / eps);
  const double f = 0.5 * (1.0 - t * t) / eps;  // -d phi / d d
  for (int e = 0; e < 3; ++e) out[e] = f * r[e] / rn;  // d d / d c = -r/|r|
}

// ===========================================================================
// A4a: recompute u~ of the step from (u, N_prev) and reverse IB forcing and drag:
//   lambda_u~ = (1 - phi) lambda_u* + w (V/dt) phi e_x
//   dJ/dc    += sum (d phi/dc) (w (V/dt) u~_x - u~ . lambda_u*)
//   lambda_N  = -c1 dt lambda_u~ + (carried from the next step)
//   carried  <- -c0 dt lambda_u~  (0.5 dt lambda_u~; none for the first step)
// ===========================================================================
template <int B>
__global__ __launch_bounds__(kNT) void k_adj_ib(DevGrid g, AdjFields F, const double* u,
                                                const double* v, const double* w,
                                                const double* nx, const double* ny,
                                                const double* nz, const double* ub,
                                                int first, double drag_weight) {
  constexpr int B3 = B * B * B;
  const size_t gid = (size_t)blockIdx.x * kNT + threadIdx.x;
  double gc[3] = {0.0, 0.0, 0.0};
  if (gid < (size_t)g.n_cubes * B3) {
    Cell<B> x{(int)(gid / B3), (int)(gid % B), (int)((gid / B) % B), (int)((gid / (B * B)) % B)};
    const SimParams& p = g.sp[g.sim[x.c]];
    const double h = p.h0 / double(1 << g.lvl[x.c]);
    const double dt = p.dt, nu = p.nu, V = h * h * h;
    const double* U[3] = {u, v, w};
    const double* Np[3] = {nx, ny, nz};
    // u and its six face neighbours (ghosts at domain faces), per component
    double uc[3], un[3][6];
    for (int e = 0; e < 3; ++e) uc[e] = U[e][gid];
    for (int f = 0; f < 6; ++f) {
      int cell;
      const int n = nb_index<B>(g, x, f, &cell);
      for (int e = 0; e < 3; ++e)
        un[e][f] = n >= 0 ? U[e][(size_t)n * B3 + cell] : ghost_value<B>(g, x, f, e, uc[e], ub);
    }
    double ut[3];
    for (int c = 0; c < 3; ++c) {
      double N = 0.0, L = 0.0;
      for (int d = 0; d < 3; ++d) {
        const double Fp = 0.5 * (uc[d] + un[d][2 * d + 1]) * (0.5 * (uc[c] + un[c][2 * d + 1]));
        const double Fm = 0.5 * (un[d][2 * d] + uc[d]) * (0.5 * (un[c][2 * d] + uc[c]));
        N += Fp - Fm;
        L += un[c][2 * d + 1] - 2.0 * uc[c] + un[c][2 * d];
      }
      N /= h;
      L /= h * h;
      const double Nprev = first ? N : Np[c][gid];
      ut[c] = uc[c] + dt * (-(1.5 * N - 0.5 * Nprev) + nu * L);
    }
    // solid fraction and its centre derivative (fixed spheres; nearest body)
    double phi = 0.0, dphi[3] = {0.0, 0.0, 0.0};
    if (p.n_bodies > 0) {
      const double xc[3] = {centre<B>(g, x.c, 0, x.i), centre<B>(g, x.c, 1, x.j),
                            centre<B>(g, x.c, 2, x.k)};
      double best = INFINITY;
      int bi = 0;
      for (int q = 0; q < p.n_bodies; ++q) {
        const bcm_body& bd = p.bodies[q];
        const double r0 = xc[0] - bd.center[0], r1 = xc[1] - bd.center[1], r2 = xc[2] - bd.center[2];
        const double d = sqrt(r0 * r0 + r1 * r1 + r2 * r2) - bd.axes[0];
        if (d < best) { best = d; bi = q; }
      }
      const double eps = 1.5 * h;
      phi = (best < 20.0 * eps) ? 0.5 * (1.0 - tanh(best / eps)) : 0.0;
      if (bi == 0) dphi_dc(xc, p.bodies[0], eps, dphi);  // gradient w.r.t. body 0's centre
    }
    double lus[3];
    for (int c = 0; c < 3; ++c) lus[c] = F.lus[c][gid];
    const double dragk = drag_weight * V / dt;
    const double c1 = first ? 1.0 : 1.5;
    for (int c = 0; c < 3; ++c) {
      const double lt = (1.0 - phi) * lus[c] + (c == 0 ? dragk * phi : 0.0);
      F.lut[c][gid] = lt;
      F.lN[c][gid] = -c1 * dt * lt + F.lNn[c][gid];
      F.lNn[c][gid] = first ? 0.0 : 0.5 * dt * lt;
    }
    const double s = dragk * ut[0] - (ut[0] * lus[0] + ut[1] * lus[1] + ut[2] * lus[2]);
    for (int e = 0; e < 3; ++e) gc[e] = dphi[e] * s;
  }
  flush_grad(F.acc + kModes, gc, 3);
}

// ===========================================================================
// A4b: lambda_u = lambda_u~ + dt nu L^T lambda_u~ + (dN/du)^T lambda_N
//      + kappa lambda_ub' at outflow cells;  lambda_ub = (1 - kappa) lambda_ub' + ghosts;
//      inflow ghosts -> dJ/da.
// ===========================================================================
template <int B>
__global__ __launch_bounds__(kNT) void k_adj_momentum(DevGrid g, AdjFields F, const double* u,
                                                      const double* v, const double* w,
                                                      const double* ub) {
  constexpr int B3 = B * B * B;
  const size_t gid = (size_t)blockIdx.x * kNT + threadIdx.x;
  double ga[kModes] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (gid < (size_t)g.n_cubes * B3) {
    Cell<B> x{(int)(gid / B3), (int)(gid % B), (int)((gid / B) % B), (int)((gid / (B * B)) % B)};
    const SimParams& p = g.sp[g.sim[x.c]];
    const double h = p.h0 / double(1 << g.lvl[x.c]);
    const double dt = p.dt, nu = p.nu;
    const double* U[3] = {u, v, w};
    double uc[3], lN[3], lt[3];
    for (int e = 0; e < 3; ++e) {
      uc[e] = U[e][gid];
      lN[e] = F.lN[e][gid];
      lt[e] = F.lut[e][gid];
    }
    double out[3] = {lt[0], lt[1], lt[2]};
    const double kdiff = dt * nu / (h * h);
    for (int e = 0; e < 3; ++e) out[e] -= 6.0 * kdiff * lt[e];
    for (int d = 0; d < 3; ++d) {
      for (int side = 0; side < 2; ++side) {
        const int f = 2 * d + side;
        int cell;
        const int n = nb_index<B>(g, x, f, &cell);
        double uo[3], lNo[3] = {0.0, 0.0, 0.0};
        if (n >= 0) {
          const size_t gi = (size_t)n * B3 + cell;
          for (int e = 0; e < 3; ++e) {
            uo[e] = U[e][gi];
            lNo[e] = F.lN[e][gi];
            out[e] += kdiff * F.lut[e][gi];  // L^T: neighbour's lambda_u~
          }
        } else {
          for (int e = 0; e < 3; ++e) uo[e] = ghost_value<B>(g, x, f, e, uc[e], ub);
        }
        // face flux F_dc = (u_d,A + u_d,B)(u_c,A + u_c,B)/4 is + in N(A)/h, - in N(B)/h;
        // this cell is A on its high face (side 1) and B on its low face (side 0)
        double mu[3];
        for (int c = 0; c < 3; ++c)
          mu[c] = side ? (lN[c] - lNo[c]) / h : (lNo[c] - lN[c]) / h;
        const double sd = uc[d] + uo[d];
        double S[3];
        for (int e = 0; e < 3; ++e) {
          double t = 0.25 * mu[e] * sd;
          if (e == d)
            for (int c = 0; c < 3; ++c) t += 0.25 * mu[c] * (uc[c] + uo[c]);
          S[e] = t;
        }
        for (int e = 0; e < 3; ++e) out[e] += S[e];
        if (n < 0) {  // the ghost's adjoint: alpha back to this cell, beta to ub or a
          const int bc = p.bc[f];
          int a, b;
          face_ab<B>(x, f, &a, &b);
          for (int e = 0; e < 3; ++e) {
            const double al = ghost_alpha(bc, f, e);
            const double lbeta = S[e] + kdiff * lt[e];  // convection + diffusion ghost uses
            out[e] += al * lbeta;
            if (bc == BC_OUTFLOW) {
              atomicAdd(&F.lub2[((size_t)(g.slot[6 * x.c + f] * 3 + e) * B + b) * B + a],
                        2.0 * lbeta);
            } else if (bc == BC_INFLOW) {
              double dbeta[kModes];
              inflow_dbeta<B>(g, x.c, f, e, a, b, dbeta);
              for (int m = 0; m < kModes; ++m) ga[m] += lbeta * dbeta[m];
            }
          }
          if (bc == BC_OUTFLOW) {  // ub' = (1-kappa) ub + kappa u_0
            const double kap = p.uconv * dt / (0.5 * h);
            for (int e = 0; e < 3; ++e) {
              const size_t si = ((size_t)(g.slot[6 * x.c + f] * 3 + e) * B + b) * B + a;
              const double lnext = F.lub[si];
              out[e] += kap * lnext;
              atomicAdd(&F.lub2[si], (1.0 - kap) * lnext);
            }
          }
        }
      }
    }
    for (int e = 0; e < 3; ++e) F.lu[e][gid] = out[e];
  }
  flush_grad(F.acc, ga, kModes);
}

// right-hand side of the adjoint Poisson solve: b = -lambda_p / V (so that the solver's
// -V (b - 0) is lambda_p), and a zero start for mu
template <int B>
__global__ __launch_bounds__(kNT) void k_adj_scale(DevGrid g, const double* lp, double* b,
                                                   double* mu, size_t nn) {
  const size_t i = (size_t)blockIdx.x * kNT + threadIdx.x;
  if (i >= nn) return;
  const int c = (int)(i / (B * B * B));
  const double h = g.sp[g.sim[c]].h0 / double(1 << g.lvl[c]);
  b[i] = -lp[i] / (h * h * h);
  mu[i] = 0.0;
}

#define ADJ_TRY(expr)                                                     \
  do {                                                                    \
    cudaError_t e_ = (expr);                                              \
    if (e_ != cudaSuccess) return grid_fail(BCM_E_CUDA, cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

extern "C" size_t bcm_adjoint_bytes(const bcm_grid* grid) {
  if (!grid) return 0;
  const Ctx& x = *grid_ctx(grid);
  const size_t n = (size_t)x.g.n_cubes * x.B * x.B * x.B;
  size_t nub = 0;  // outflow face values: as many as the grid's BCM_UB field
  void* ptr = nullptr;
  size_t cnt = 0;
  int32_t eb = 0;
  if (bcm_field(const_cast<bcm_grid*>(grid), BCM_UB, &ptr, &cnt, &eb) == BCM_OK) nub = cnt;
  return adj_layout(n, nub, nullptr, nullptr);
}

extern "C" bcm_status bcm_adjoint_init(bcm_grid* grid, void* dev_adj, size_t bytes) {
  if (!grid || !dev_adj) return grid_fail(BCM_E_INVALID, "NULL argument");
  const size_t need = bcm_adjoint_bytes(grid);
  if (bytes < need) return grid_fail(BCM_E_INVALID, "adjoint workspace too small");
  ADJ_TRY(cudaMemsetAsync(dev_adj, 0, need, grid_stream(grid)));
  return BCM_OK;
}

extern "C" bcm_status bcm_adjoint_step(bcm_grid* grid, void* dev_adj, size_t bytes,
                                       const void* const* state, int first_step,
                                       double drag_weight, double rtol, int max_iter,
                                       double* dev_dJ) {
  if (!grid || !dev_adj || !state || !dev_dJ) return grid_fail(BCM_E_INVALID, "NULL argument");
  if (grid_two_level(grid)) return grid_fail(BCM_E_INVALID, "the adjoint needs a single-level grid");
  const Ctx& base = *grid_ctx(grid);
  if (!base.f64 || !base.solve64)
    return grid_fail(BCM_E_INVALID, "the adjoint runs on FP64 grids (BCM_PREC_F64)");
  if (base.part.n > 0)
    return grid_fail(BCM_E_INVALID, "the adjoint differentiates the solid-fraction IB, not particles");
  if (base.scheme != 0)
    return grid_fail(BCM_E_INVALID, "the adjoint differentiates the Adams-Bashforth step");
  if (bytes < bcm_adjoint_bytes(grid)) return grid_fail(BCM_E_INVALID, "adjoint workspace too small");
  const size_t n = (size_t)base.g.n_cubes * base.B * base.B * base.B;
  void* ubp = nullptr;
  size_t nub = 0;
  int32_t eb = 0;
  bcm_field(grid, BCM_UB, &ubp, &nub, &eb);
  AdjFields F;
  adj_layout(n, nub, &F, (unsigned char*)dev_adj);
  F.acc = dev_dJ;
  cudaStream_t s = grid_stream(grid);
  const double* u = (const double*)state[0];
  const double* v = (const double*)state[1];
  const double* w = (const double*)state[2];
  const double* nx = (const double*)state[3];
  const double* ny = (const double*)state[4];
  const double* nz = (const double*)state[5];
  const double* ub = (const double*)state[6];
  const unsigned nblk = (unsigned)((n + kNT - 1) / kNT);
  // lambda_ub2 starts at zero; lambda_ub holds the adjoint of the step's new face state
  if (nub) ADJ_TRY(cudaMemsetAsync(F.lub2, 0, nub * sizeof(double), s));
#define ADJ_B(...)                                              \
  switch (base.B) {                                             \
    case 4: { constexpr int B = 4; __VA_ARGS__; break; }        \
    case 8: { constexpr int B = 8; __VA_ARGS__; break; }        \
    case 16: { constexpr int B = 16; __VA_ARGS__; break; }      \
    default: return grid_fail(BCM_E_INVALID, "cells_per_edge"); \
  }
  ADJ_B(k_adj_projection<B><<<nblk, kNT, 0, s>>>(base.g, F));
  ADJ_TRY(cudaGetLastError());
  // adjoint Poisson solve K mu = lambda_p: the solver's rhs is -V (b - mean) with
  // mean = 0 (outflow sims), so b = -lambda_p / V; FP64 CG vectors of the workspace
  {
    Ctx x = base;
    x.persistent = 0;
    x.f.p = F.mu;
    x.f.b = F.bsc;
    x.f.r = F.cg[0];
    x.f.p0 = F.cg[1];
    x.f.p1 = F.cg[2];
    x.f.q = F.cg[3];
    ADJ_B(k_adj_scale<B><<<nblk, kNT, 0, s>>>(base.g, F.lp, F.bsc, F.mu, n));
    ADJ_TRY(cudaGetLastError());
    SolveParams prm{};
    prm.rtol = rtol;
    prm.inner_rtol = 1e-5;
    prm.max_iter = max_iter;
    prm.inner_max_iter = max_iter;
    prm.max_cycles = 1;
    prm.guard = x.f.guard;
    ADJ_TRY(launch_solve_begin(x));
    ADJ_TRY(launch_residual(x, prm));
    int done = 0;
    for (int it = 0; it < max_iter;) {
      ADJ_TRY(cudaMemcpyAsync(&done, x.g.flags, sizeof(int), cudaMemcpyDeviceToHost, s));
      ADJ_TRY(cudaStreamSynchronize(s));
      if (done) break;
      for (int m = 0; m < 8 && it < max_iter; ++m, ++it) {
        ADJ_TRY(launch_cg_a(x, prm));
        ADJ_TRY(launch_cg_b(x, prm));
      }
    }
  }
  ADJ_B(k_adj_rhs<B><<<nblk, kNT, 0, s>>>(base.g, F));
  ADJ_TRY(cudaGetLastError());
  ADJ_B(k_adj_ib<B><<<nblk, kNT, 0, s>>>(base.g, F, u, v, w, nx, ny, nz, ub, first_step,
                                         drag_weight));
  ADJ_TRY(cudaGetLastError());
  ADJ_B(k_adj_momentum<B><<<nblk, kNT, 0, s>>>(base.g, F, u, v, w, ub));
  ADJ_TRY(cudaGetLastError());
  // the step's lambda_ub (of ub^n) becomes the next (earlier) step's lambda_ub'
  if (nub) ADJ_TRY(cudaMemcpyAsync(F.lub, F.lub2, nub * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return BCM_OK;
}
