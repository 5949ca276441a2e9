// bcm_kernels.cu -- sm_103a kernels of the BCM fractional step (arXiv:1808.04099,
// section "Numerical algorithm"): solid fraction, momentum + IB forcing, Poisson
// right-hand side, Jacobi-PCG passes, FP64 residual for defect correction, and the
// projection.  All of them are HBM-bandwidth bound stencils or streams (no dense
// contraction, so no tensor cores): cube-major SoA rows are read coalesced, each
// CTA stages its cube (or a z-slab) plus a one-cell face halo in shared memory, and
// Krylov dot products are reduced with warp shuffles into FP64 per-sim atomics.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bcm_cube.cuh"
#include "bcm_internal.cuh"
#include "bcm_kernels.h"
#include "bcm_stencil.cuh"

namespace bcm {

// ------------------------------------------------------------- body geometry

// Signed distance of point x to a body at time t (body pose precomputed), and the
// rigid-body velocity there.  Sphere: exact; ellipsoid: k0 (k0 - 1) / k1 (R9).
struct Pose {
  double c[3];
  double R[3][3];
  int kind;
  double ax[3], om[3], v[3];
};

__device__ void make_pose(const bcm_body& b, double t, Pose& P) {
  P.kind = b.kind;
  for (int e = 0; e < 3; ++e) {
    P.c[e] = b.center[e] + b.vel[e] * t;
    P.ax[e] = b.axes[e];
    P.om[e] = b.omega[e];
    P.v[e] = b.vel[e];
  }
  const double w = b.quat[0], x = b.quat[1], y = b.quat[2], z = b.quat[3];
  double R0[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                     {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                     {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
  double th[3] = {b.omega[0] * t, b.omega[1] * t, b.omega[2] * t};
  double a = sqrt(th[0] * th[0] + th[1] * th[1] + th[2] * th[2]);
  double Rt[3][3];
  if (a == 0.0) {
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Rt[i][j] = (i == j) ? 1.0 : 0.0;
  } else {
    double k[3] = {th[0] / a, th[1] / a, th[2] / a};
    double cs = cos(a), sn = sin(a);
    double K[3][3] = {{0, -k[2], k[1]}, {k[2], 0, -k[0]}, {-k[1], k[0], 0}};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double kk = 0;
        for (int m = 0; m < 3; ++m) kk += K[i][m] * K[m][j];
        Rt[i][j] = (i == j ? 1.0 : 0.0) + sn * K[i][j] + (1 - cs) * kk;
      }
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int m = 0; m < 3; ++m) acc += Rt[i][m] * R0[m][j];
      P.R[i][j] = acc;
    }
}

__device__ double pose_sd(const Pose& P, const double* x) {
  double r[3] = {x[0] - P.c[0], x[1] - P.c[1], x[2] - P.c[2]};
  if (P.kind == BCM_BODY_SPHERE) return sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]) - P.ax[0];
  double y[3];
  for (int j = 0; j < 3; ++j) y[j] = P.R[0][j] * r[0] + P.R[1][j] * r[1] + P.R[2][j] * r[2];
  double k0 = 0, k1 = 0;
  for (int e = 0; e < 3; ++e) {
    k0 += (y[e] / P.ax[e]) * (y[e] / P.ax[e]);
    k1 += (y[e] / (P.ax[e] * P.ax[e])) * (y[e] / (P.ax[e] * P.ax[e]));
  }
  k0 = sqrt(k0);
  k1 = sqrt(k1);
  if (k1 == 0.0) return -fmin(P.ax[0], fmin(P.ax[1], P.ax[2]));
  return k0 * (k0 - 1.0) / k1;
}

// ===========================================================================
// (a2) solid fraction phi = (1 - tanh(d/eps))/2, eps = 1.5 h, 0 beyond 20 eps (R5)
// ===========================================================================
template <int B, int NT, class T>
__global__ __launch_bounds__(NT) void k_solid_fraction(DevGrid g, T* __restrict__ phi,
                                                       unsigned char* __restrict__ bid,
                                                       unsigned char* __restrict__ near,
                                                       int sim_filter) {
  constexpr int B3 = B * B * B;
  const int c = blockIdx.x;
  const int s = g.sim[c];
  const SimParams& sp = g.sp[s];
  // sim_filter: -1 every sim, -2 sims with moving bodies, >= 0 that sim only
  if (sp.n_bodies == 0 || (sim_filter == -2 && !sp.moving) || (sim_filter >= 0 && s != sim_filter))
    return;
  __shared__ Pose P[kMaxBodies];
  __shared__ int any_near;
  const double t = g.ss[s].step * sp.dt;
  if (threadIdx.x < sp.n_bodies) make_pose(sp.bodies[threadIdx.x], t, P[threadIdx.x]);
  if (threadIdx.x == 0) any_near = 0;
  __syncthreads();
  const double h = cell_h<B>(g, c), eps = 1.5 * h;
  // conservative cube cull: the signed-distance estimate is >= (|y|/amax - 1) amin
  if (threadIdx.x == 0) {
    int nearc = 0;
    for (int bi = 0; bi < sp.n_bodies; ++bi) {
      double d2 = 0.0;
      for (int e = 0; e < 3; ++e) {
        double lo = sp.origin[e] + g.ijk[3 * c + e] * sp.hf + 0.5 * h;
        double hi = lo + (B - 1) * h;
        double q = fmin(fmax(P[bi].c[e], lo), hi) - P[bi].c[e];
        d2 += q * q;
      }
      double amax = fmax(P[bi].ax[0], fmax(P[bi].ax[1], P[bi].ax[2]));
      double amin = fmin(P[bi].ax[0], fmin(P[bi].ax[1], P[bi].ax[2]));
      if (P[bi].kind == BCM_BODY_SPHERE) amax = amin = P[bi].ax[0];
      double dlow = (sqrt(d2) / amax - 1.0) * amin;
      if (dlow < 20.0 * eps * 1.0000001) nearc = 1;
    }
    any_near = nearc;
  }
  __syncthreads();
  if (!any_near) {
    if (near[c]) {
      for (int q = threadIdx.x; q < B3; q += NT) phi[(size_t)c * B3 + q] = T(0);
      __syncthreads();
      if (threadIdx.x == 0) near[c] = 0;
    }
    return;
  }
  for (int q = threadIdx.x; q < B3; q += NT) {
    const int i = q % B, j = (q / B) % B, k = q / (B * B);
    double x[3] = {centre<B>(g, c, 0, i), centre<B>(g, c, 1, j), centre<B>(g, c, 2, k)};
    double best = INFINITY;
    int bb = 0;
    for (int bi = 0; bi < sp.n_bodies; ++bi) {
      double d = pose_sd(P[bi], x);
      if (d < best) {
        best = d;
        bb = bi;
      }
    }
    double f = (best < 20.0 * eps) ? 0.5 * (1.0 - tanh(best / eps)) : 0.0;
    phi[(size_t)c * B3 + q] = T(f);
    bid[(size_t)c * B3 + q] = (unsigned char)bb;
  }
  if (threadIdx.x == 0) near[c] = 1;
}

// ===========================================================================
// QUICK + Crank-Nicolson momentum (Eq. substep1 with the QUICK convection the paper
// names; R20):
//   N_c = (1/h) sum_d [U+ q+ - U- q-], U± the central face velocities, q± the QUICK
//         face values 6/8 C + 3/8 D - 1/8 U (C upwind, D downwind, U upwind of C);
//   u^(k+1) = (E - dt/2 N(u^(k)) + dt nu/2 (sum of the 6 neighbours)/h^2) / (1 + 3 a),
//   E = u^n + dt (-N(u^n) + nu L(u^n))/2, a = dt nu / h^2, from u^(0) = 2 E - u^n,
// until ||u^(k+1) - u^(k)|| <= cn_rtol ||u^(k+1)|| per sim, or the update has reached the
// rounding floor of the arithmetic (<= 64 eps ||u^(k+1)||) and stopped shrinking (its
// square >= 0.99 of the previous one), or cn_max.
// The kernels iterate on the increment d = u - u^n, which is what FP32 can hold to its
// own precision (FP32 iterates of u itself settle ~3 roundings of |u| away from the
// fixed point):
//   d^(k+1) = (E' - dt/2 N(u^n + d^(k)) + a/2 (sum of the 6 neighbours of d^(k))) / (1 + 3a),
//   E' = dt (-N(u^n)/2 + nu L(u^n)),  d^(0) = dt (-N(u^n) + nu L(u^n)),
// the same iteration in exact arithmetic.  Ghosts: u^n + d by the halo rules with the
// outflow values of t^n.  Every halo rule is affine in the field with the same boundary
// value for u^n and u^n + d, so the neighbour sum of d equals that of u^n + d minus that
// of u^n (both with those ghosts): the explicit kernel folds -a/2 (neighbour sum of u^n)
// into E'' = E' - a/2 sum u^n, and an iteration needs the tiles of u^n + d alone,
//   d^(k+1) = (E'' + a/2 (sum of the 6 neighbours of u^n + d^(k)) - dt/2 N(u^n + d^(k))) / (1 + 3a).
// In FP32 the neighbour sum then carries the rounding of u^n + d: at most
// 3a / (1 + 3a) of one rounding of |u| on d, below the rounding of the stored u*.
// QUICK reads two cells upstream, so the slabs carry the paper's two ghost layers.
// Storage: u^n stays in u, E'' in u*, d alternates between two sets of PCG scratch
// vectors (free during the momentum sub-step) by the parity of the sim's iteration
// count; the last launch writes u* = u~ + phi (u_s - u~) and advances the outflow
// values to t^{n+1}.
// ===========================================================================
template <int B, int KS>
struct Slab2 {  // planes z0-2 .. z0+KS+1, each (B+4)^2 with a two-cell x/y ring
  static constexpr int P = B + 4;
  static constexpr int N = (KS + 4) * P * P;
  __device__ __forceinline__ static int at(int i, int j, int kk) {
    return (kk * P + (j + 2)) * P + (i + 2);
  }
};

template <int B, int KS, int NT, class T, class Val, class Bc>
__device__ __forceinline__ void stage_slab2(T* __restrict__ S, const DevGrid& g, int c, int z0,
                                            const Val& val, const Bc& bc) {
  using SL = Slab2<B, KS>;
  constexpr int BB = B * B, Q = BB / 4;
  // the planes, four cells along x per access: own cube, or a same-level z neighbour
  // (its plane B + k below, k - B above); 2:1 and domain faces value by value
  for (int idx = threadIdx.x; idx < (KS + 4) * Q; idx += NT) {
    const int kk = idx / Q, q = idx - kk * Q, j = (4 * q) / B, i0 = 4 * q - j * B;
    const int k = z0 - 2 + kk;
    T v[4];
    int n = c, pl = k;
    if (k < 0 || k >= B) {
      const int f = k < 0 ? 4 : 5;
      n = g.nb[6 * c + f];
      pl = k < 0 ? B + k : k - B;
      if (n < 0) {
#pragma unroll 1
        for (int m = 0; m < 4; ++m)
          v[m] = halo_value<B, T>(g, c, f, i0 + m, j, k < 0 ? -1 - k : k - B, val, bc);
      }
    }
    if (n >= 0) val.get4(n, pl * BB + 4 * q, v);
    const int o = SL::at(i0, j, kk);
    S[o] = v[0];
    S[o + 1] = v[1];
    S[o + 2] = v[2];
    S[o + 3] = v[3];
  }
  for (int idx = threadIdx.x; idx < 8 * KS * B; idx += NT) {
    const int f = idx / (2 * KS * B), rem = idx - f * (2 * KS * B), layer = rem / (KS * B);
    const int rem2 = rem - layer * (KS * B), kk = rem2 / B, t = rem2 - kk * B;
    const T v = halo_value<B, T>(g, c, f, t, z0 + kk, layer, val, bc);
    const int n = (f & 1) ? B + layer : -1 - layer;
    S[f < 2 ? SL::at(n, t, kk + 2) : SL::at(t, n, kk + 2)] = v;
  }
}

// interior values of u^n + d
template <class T>
struct SumVal {
  const T* a;
  const T* d;
  int B3;
  __device__ __forceinline__ T operator()(int c, int cell) const {
    const size_t i = (size_t)c * B3 + cell;
    return a[i] + d[i];
  }
  __device__ __forceinline__ void get4(int c, int cell0, T (&v)[4]) const {
    const size_t i = (size_t)c * B3 + cell0;
    T w[4];
    ld4(a + i, v);
    ld4(d + i, w);
#pragma unroll
    for (int m = 0; m < 4; ++m) v[m] += w[m];
  }
};

template <class T>
__device__ __forceinline__ T quick_face(T pC, T pD, T pU) {
  return T(0.75) * pC + T(0.375) * pD - T(0.125) * pU;
}

// QUICK convection of component comp at tile position o (axis strides off[])
template <class T>
__device__ __forceinline__ T conv_quick(const T* const (&Sf)[3], int comp, int o,
                                        const int (&off)[3], T ih) {
  const T* Sc = Sf[comp];
  T N = T(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const T* Sd = Sf[d];
    const int e = off[d];
    const T Up = T(0.5) * (Sd[o] + Sd[o + e]), Um = T(0.5) * (Sd[o - e] + Sd[o]);
    const T fp = Up >= T(0) ? quick_face(Sc[o], Sc[o + e], Sc[o - e])
                            : quick_face(Sc[o + e], Sc[o], Sc[o + 2 * e]);
    const T fm = Um >= T(0) ? quick_face(Sc[o - e], Sc[o], Sc[o - 2 * e])
                            : quick_face(Sc[o], Sc[o - e], Sc[o + e]);
    N += Up * fp - Um * fm;
  }
  return N * ih;
}

template <int B, int KS, int NT, class T>
__global__ __launch_bounds__(NT) void k_cn_explicit(DevGrid g, const T* __restrict__ u,
                                                    const T* __restrict__ v,
                                                    const T* __restrict__ w, T* __restrict__ e0,
                                                    T* __restrict__ e1, T* __restrict__ e2,
                                                    T* __restrict__ d0, T* __restrict__ d1,
                                                    T* __restrict__ d2, const T* __restrict__ ub) {
  using SL = Slab2<B, KS>;
  constexpr int B3 = B * B * B, NSL = B / KS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S0 = reinterpret_cast<T*>(smem_raw);
  T* S1 = S0 + SL::N;
  T* S2 = S1 + SL::N;
  const int c = blockIdx.x / NSL, z0 = (blockIdx.x % NSL) * KS;
  const int s = g.sim[c];
  const SimParams& sp = g.sp[s];
  if (blockIdx.x == 0) {  // a new momentum solve for every sim
    for (int q = threadIdx.x; q < g.n_sims; q += NT) {
      g.ss[q].cn_iter = 0;
      g.ss[q].cn_done = 0;
      g.ss[q].cn_d2prev = 0.0;
    }
    if (threadIdx.x == 0) g.flags[2] = 0;
  }
  {
    VelocityBC<B, T> b0{&g, &sp, ub, c, 0}, b1{&g, &sp, ub, c, 1}, b2{&g, &sp, ub, c, 2};
    stage_slab2<B, KS, NT>(S0, g, c, z0, FieldVal<T>{u, B3}, b0);
    stage_slab2<B, KS, NT>(S1, g, c, z0, FieldVal<T>{v, B3}, b1);
    stage_slab2<B, KS, NT>(S2, g, c, z0, FieldVal<T>{w, B3}, b2);
  }
  __syncthreads();
  const double hd = cell_h<B>(g, c);
  const T ih = T(1.0 / hd), ih2 = T(1.0 / (hd * hd)), dt = T(sp.dt), nu = T(sp.nu);
  const T half_a = T(0.5 * sp.dt * sp.nu / (hd * hd));
  const T* const Sf[3] = {S0, S1, S2};
  T* Es[3] = {e0, e1, e2};
  T* Ds[3] = {d0, d1, d2};
  const int off[3] = {1, SL::P, SL::P * SL::P};
  for (int q = threadIdx.x; q < KS * B * B; q += NT) {
    const int kk = q / (B * B), rem = q - kk * B * B, j = rem / B, i = rem - j * B;
    const size_t gi = (size_t)c * B3 + ((z0 + kk) * B + j) * B + i;
    const int o = SL::at(i, j, kk + 2);
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      const T* Sc = Sf[comp];
      const T u0 = Sc[o];
      T L = T(0), sn = T(0);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        L += Sc[o + off[d]] - T(2) * u0 + Sc[o - off[d]];
        sn += Sc[o + off[d]] + Sc[o - off[d]];
      }
      const T N = conv_quick<T>(Sf, comp, o, off, ih);
      const T DL = dt * nu * (L * ih2);
      Es[comp][gi] = (T(-0.5) * dt * N + DL) - half_a * sn;  // E'' = E' - a/2 sum u^n
      Ds[comp][gi] = -dt * N + DL;                          // forward-Euler predictor of d
    }
  }
}

// One iteration on the increment; da / db are the two increment sets, read from the
// one the sim's iteration parity selects (k even: da).  The last block takes each
// sim's decision.
template <int B, int KS, int NT, class T>
__global__ __launch_bounds__(NT, sizeof(T) == 4 ? 4 : 3) void k_cn_iter(DevGrid g, const T* __restrict__ u,
                                                const T* __restrict__ v, const T* __restrict__ w,
                                                T* da0, T* da1, T* da2, T* db0, T* db1, T* db2,
                                                const T* __restrict__ e0,
                                                const T* __restrict__ e1,
                                                const T* __restrict__ e2,
                                                const T* __restrict__ ub, double rtol2, int cn_max) {
  using SL = Slab2<B, KS>;
  constexpr int B3 = B * B * B, NSL = B / KS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S0 = reinterpret_cast<T*>(smem_raw);  // u^n + d, three components
  __shared__ double red[2 * 32];
  const int c = blockIdx.x / NSL, z0 = (blockIdx.x % NSL) * KS;
  const int s = g.sim[c];
  const SimParams& sp = g.sp[s];
  SimState& st = g.ss[s];
  const bool active = st.cn_done == 0;
  double vals[2] = {0.0, 0.0};
  if (active) {
    const bool odd = (st.cn_iter & 1) != 0;
    const T* src[3] = {odd ? db0 : da0, odd ? db1 : da1, odd ? db2 : da2};
    T* dst[3] = {odd ? da0 : db0, odd ? da1 : db1, odd ? da2 : db2};
    const T* un[3] = {u, v, w};
    // the iterates are velocities of t^{n+1}: outflow ghosts from u_b^{n+1}
    const T coef = T(sp.uconv * sp.dt / (0.5 * cell_h<B>(g, c)));
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      VelocityBCNext<B, T> vb{&g, &sp, ub, un[comp], c, comp, coef};
      stage_slab2<B, KS, NT>(S0 + comp * SL::N, g, c, z0, SumVal<T>{un[comp], src[comp], B3}, vb);
    }
    __syncthreads();
    const double hd = cell_h<B>(g, c);
    const T ih = T(1.0 / hd), dt = T(sp.dt);
    const T half_a = T(0.5 * sp.dt * sp.nu / (hd * hd));
    const T den = T(1.0 + 3.0 * sp.dt * sp.nu / (hd * hd));
    const T* const Sf[3] = {S0, S0 + SL::N, S0 + 2 * SL::N};
    const T* Es[3] = {e0, e1, e2};
    const int off[3] = {1, SL::P, SL::P * SL::P};
    T dd2 = T(0), uu2 = T(0);
    for (int q = threadIdx.x; q < KS * B * B; q += NT) {
      const int kk = q / (B * B), rem = q - kk * B * B, j = rem / B, i = rem - j * B;
      const size_t gi = (size_t)c * B3 + ((z0 + kk) * B + j) * B + i;
      const int o = SL::at(i, j, kk + 2);
#pragma unroll
      for (int comp = 0; comp < 3; ++comp) {
        const T* Sc = Sf[comp];
        T sn = T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) sn += Sc[o + off[d]] + Sc[o - off[d]];
        const T N = conv_quick<T>(Sf, comp, o, off, ih);
        const T dn = ((Es[comp][gi] + half_a * sn) - T(0.5) * dt * N) / den;
        const T ch = dn - src[comp][gi];
        const T ut = un[comp][gi] + dn;
        dd2 += ch * ch;
        uu2 += ut * ut;
        dst[comp][gi] = dn;
      }
    }
    vals[0] = double(dd2);
    vals[1] = double(uu2);
  }
  block_sum<NT, 2>(vals, red);
  if (threadIdx.x == 0 && active) {
    acc_add(st, ACC_CN_D, vals[0]);
    acc_add(st, ACC_CN_U, vals[1]);
  }
  if (last_block(g.counter)) {
    int alive = 0;
    for (int q = threadIdx.x; q < g.n_sims; q += NT) {
      SimState& t = g.ss[q];
      const double d2 = acc_take(t, ACC_CN_D), u2 = acc_take(t, ACC_CN_U);
      if (t.cn_done) continue;
      // 64 unit roundoffs of the iteration's arithmetic
      const double fl = 64.0 * (sizeof(T) == 8 ? 0x1p-53 : 0x1p-24);
      const bool stalled = t.cn_iter >= 1 && d2 <= fl * fl * u2 && d2 >= 0.99 * t.cn_d2prev;
      t.cn_iter += 1;
      t.cn_d2prev = d2;
      if (d2 <= rtol2 * u2 || stalled || t.cn_iter >= cn_max || !isfinite(d2)) t.cn_done = 1;
      alive |= !t.cn_done;
    }
    alive = __syncthreads_or(alive);
    if (threadIdx.x == 0) g.flags[2] = !alive;
  }
}

// u* = u~ + phi (u_s - u~) with u~ = u^n + d (the sim's last increment), the drag (R5),
// and the convective outflow values advanced to t^{n+1} from u^n (R8).
template <int B, int NT, class T>
__global__ __launch_bounds__(NT) void k_cn_finish(DevGrid g, const T* __restrict__ u,
                                                  const T* __restrict__ v,
                                                  const T* __restrict__ w, const T* da0,
                                                  const T* da1, const T* da2, const T* db0,
                                                  const T* db1, const T* db2, T* us, T* vs,
                                                  T* ws, const T* __restrict__ phi,
                                                  const unsigned char* __restrict__ bid,
                                                  T* __restrict__ ub) {
  constexpr int B3 = B * B * B;
  __shared__ double red[3 * 32];
  const int c = blockIdx.x;
  const int s = g.sim[c];
  const SimParams& sp = g.sp[s];
  // iteration k writes the second set (db) when k is even: the last one is cn_iter - 1
  const bool last_even = ((g.ss[s].cn_iter - 1) & 1) == 0;
  const T* dl[3] = {last_even ? db0 : da0, last_even ? db1 : da1, last_even ? db2 : da2};
  const T* un[3] = {u, v, w};
  T* outs[3] = {us, vs, ws};
  const bool has_phi = g.near[c] != 0;
  const double t = g.ss[s].step * sp.dt;
  T fsum[3] = {T(0), T(0), T(0)};
  for (int q = threadIdx.x; q < B3; q += NT) {
    const int k = q / (B * B), j = (q / B) % B, i = q % B;
    const size_t gi = (size_t)c * B3 + q;
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
      const T ut = un[comp][gi] + dl[comp][gi];
      const T du = ph * (usb[comp] - ut);
      outs[comp][gi] = ut + du;
      fsum[comp] += du;
    }
  }
  // convective outflow: u_b^{n+1} = u_b - U_c dt (u_b - u_0) / (h/2), u_0 from u^n
  const double hd = cell_h<B>(g, c);
  for (int f = 0; f < 6; ++f) {
    const int sl = g.slot[6 * c + f];
    if (sl < 0) continue;
    const int d = f >> 1, side = f & 1;
    const T coef = T(sp.uconv * sp.dt / (0.5 * hd));
    for (int q = threadIdx.x; q < 3 * B * B; q += NT) {
      const int comp = q / (B * B), rem = q - comp * B * B, bb = rem / B, a = rem - bb * B;
      const T u0 = un[comp][(size_t)c * B3 + cell_of<B>(d, side ? B - 1 : 0, a, bb)];
      T* pb = &ub[((size_t)(sl * 3 + comp) * B + bb) * B + a];
      *pb = *pb - coef * (*pb - u0);
    }
  }
  if (has_phi) {
    double vals[3] = {double(fsum[0]), double(fsum[1]), double(fsum[2])};
    block_sum<NT, 3>(vals, red);
    if (threadIdx.x == 0) {
      const double scale = -hd * hd * hd / sp.dt;
      for (int e = 0; e < 3; ++e) atomicAdd(&g.ss[s].drag_acc[e], vals[e] * scale);
    }
  }
}

// Step bookkeeping: drag, divergence ratio, time step counter.
__global__ void k_step_end(DevGrid g) {
  for (int s = threadIdx.x; s < g.n_sims; s += blockDim.x) {
    SimState& t = g.ss[s];
    for (int e = 0; e < 3; ++e) {
      t.drag[e] = t.drag_acc[e];
      t.drag_sum[e] += t.drag_acc[e];
      t.drag_acc[e] = 0.0;
    }
    t.drag_n += 1;
    const double dn = acc_take(t, ACC_DIVN), dd = acc_take(t, ACC_DIVD);
    t.div_num = dn;
    t.div_den = dd;
    t.step += 1;
    t.ab2_restart = 0;
  }
}

// Volume mean of b per all-Neumann sim (standalone pressure solves).
template <int B, int NT>
__global__ __launch_bounds__(NT) void k_bmean(DevGrid g, const double* __restrict__ b) {
  constexpr int B3 = B * B * B;
  __shared__ double red[32];
  const int c = blockIdx.x;
  const int s = g.sim[c];
  double acc = 0.0;
  for (int q = threadIdx.x; q < B3; q += NT) acc += b[(size_t)c * B3 + q];
  double vals[1] = {acc};
  block_sum<NT, 1>(vals, red);
  if (threadIdx.x == 0 && g.sp[s].all_neumann) acc_add(g.ss[s], ACC_BSUM, vals[0]);
  if (last_block(g.counter)) {
    for (int q = threadIdx.x; q < g.n_sims; q += NT) {
      SimState& st = g.ss[q];
      const double bs = acc_take(st, ACC_BSUM);
      st.bmean = g.sp[q].all_neumann ? bs / g.sp[q].n_cells : 0.0;
    }
  }
}

// Reset per-solve state before a pressure solve; zero the graph-loop guard.
__global__ void k_solve_begin(DevGrid g, unsigned int* guard) {
  for (int s = threadIdx.x; s < g.n_sims; s += blockDim.x) {
    SimState& t = g.ss[s];
    t.iter = 0;
    t.done = 0;
    t.outer_done = 0;
    t.cycles = 0;
    t.total_iters = 0;
    t.converged = 0;
    t.nonfinite = 0;
    t.zero_rhs = 0;
    t.umax_bits = 0ull;
    t.fz_valid = 0;
  }
  if (threadIdx.x == 0) guard[0] = 0u;
}

// ===========================================================================
// Test-path kernels: the paper's two-layer halo fill and y = K x.
// ===========================================================================
template <int B, int NT, class T>
__global__ __launch_bounds__(NT) void k_fill_halo(DevGrid g, const T* __restrict__ f, int kind,
                                                  const T* __restrict__ ub,
                                                  double* __restrict__ out) {
  constexpr int B3 = B * B * B, G = B + 4;
  const int c = blockIdx.x;
  const SimParams& sp = g.sp[g.sim[c]];
  double* o = out + (size_t)c * G * G * G;
  struct DV {
    const T* f;
    __device__ __forceinline__ double operator()(int cc, int cell) const {
      return double(f[(size_t)cc * B3 + cell]);
    }
  } val{f};
  for (int q = threadIdx.x; q < G * G * G; q += NT) {
    const int i = q % G - 2, j = (q / G) % G - 2, k = q / (G * G) - 2;
    const int out_i = (i < 0 || i >= B), out_j = (j < 0 || j >= B), out_k = (k < 0 || k >= B);
    double vv = 0.0;
    if (!out_i && !out_j && !out_k) {
      vv = val(c, (k * B + j) * B + i);
    } else if (out_i + out_j + out_k == 1) {
      int f2, a, bb, layer;
      if (out_i) { f2 = i < 0 ? 0 : 1; layer = i < 0 ? -1 - i : i - B; a = j; bb = k; }
      else if (out_j) { f2 = j < 0 ? 2 : 3; layer = j < 0 ? -1 - j : j - B; a = i; bb = k; }
      else { f2 = k < 0 ? 4 : 5; layer = k < 0 ? -1 - k : k - B; a = i; bb = j; }
      if (kind == 3) {
        vv = halo_value<B, double>(g, c, f2, a, bb, layer, val, PressureBC{&sp});
      } else {
        struct VB {
          const DevGrid* g;
          const SimParams* sp;
          const T* ub;
          int c, comp;
          __device__ double operator()(int fc, int a2, int b2, double u0) const {
            const int bc = sp->bc[fc];
            if (bc == BC_SLIP) return (comp == (fc >> 1)) ? -u0 : u0;
            if (bc == BC_OUTFLOW)
              return 2.0 * double(ub[((size_t)(g->slot[6 * c + fc] * 3 + comp) * B + b2) * B + a2]) - u0;
            return 2.0 * face_velocity<B>(*g, c, fc, comp, a2, b2) - u0;
          }
        } vb{&g, &sp, ub, c, kind};
        vv = halo_value<B, double>(g, c, f2, a, bb, layer, val, vb);
      }
    }
    o[q] = vv;
  }
}

// ===========================================================================
// Launchers
// ===========================================================================

template <class T>
static cudaError_t solid_fraction_t(const Ctx& x, int sim_filter) {
  BCM_DISPATCH_B(x.B, {
    constexpr int NT = threads_for<B>();
    k_solid_fraction<B, NT, T><<<x.g.n_cubes, NT, 0, x.stream>>>(
        x.g, (T*)x.f.phi, x.f.bid, x.f.near, sim_filter);
  });
  return cudaGetLastError();
}
cudaError_t launch_solid_fraction(const Ctx& x, int sim_filter) {
  if (x.part.n > 0) return cudaSuccess;  // Lagrangian particles: no solid fraction
  return x.f64 ? solid_fraction_t<double>(x, sim_filter) : solid_fraction_t<float>(x, sim_filter);
}

// QUICK + Crank-Nicolson: z-slabs of 16^3 cubes, 4 planes in FP32 (three (B+4)^2 x 8
// tiles, 38 KB) and 2 in FP64 (three x 6 tiles, 58 KB)
template <int B, class T>
constexpr int cn_slab() { return B == 16 ? (sizeof(T) == 4 ? 4 : 2) : B; }

template <class T>
static cudaError_t cn_explicit_t(const Ctx& x) {
  BCM_DISPATCH_B(x.B, {
    constexpr int NT = threads_for<B>(), KS = cn_slab<B, T>();
    const size_t sm = 3 * sizeof(T) * Slab2<B, KS>::N;
    auto kern = k_cn_explicit<B, KS, NT, T>;
    cudaError_t e = allow_smem(kern, sm);
    if (e != cudaSuccess) return e;
    kern<<<x.g.n_cubes * (B / KS), NT, sm, x.stream>>>(
        x.g, (const T*)x.f.u, (const T*)x.f.v, (const T*)x.f.w, (T*)x.f.us, (T*)x.f.vs,
        (T*)x.f.ws, (T*)x.f.w1, (T*)x.f.s0, (T*)x.f.s1, (const T*)x.f.ub);
  });
  return cudaGetLastError();
}
cudaError_t launch_cn_explicit(const Ctx& x) {
  return x.f64 ? cn_explicit_t<double>(x) : cn_explicit_t<float>(x);
}

template <class T>
static cudaError_t cn_iter_t(const Ctx& x) {
  BCM_DISPATCH_B(x.B, {
    constexpr int NT = threads_for<B>(), KS = cn_slab<B, T>();
    const size_t sm = 3 * sizeof(T) * Slab2<B, KS>::N;
    auto kern = k_cn_iter<B, KS, NT, T>;
    cudaError_t e = allow_smem(kern, sm);
    if (e != cudaSuccess) return e;
    kern<<<x.g.n_cubes * (B / KS), NT, sm, x.stream>>>(
        x.g, (const T*)x.f.u, (const T*)x.f.v, (const T*)x.f.w, (T*)x.f.w1, (T*)x.f.s0,
        (T*)x.f.s1, (T*)x.f.r, (T*)x.f.p0, (T*)x.f.p1, (const T*)x.f.us, (const T*)x.f.vs,
        (const T*)x.f.ws, (const T*)x.f.ub, x.cn_rtol * x.cn_rtol, x.cn_max);
  });
  return cudaGetLastError();
}
cudaError_t launch_cn_iter(const Ctx& x) {
  return x.f64 ? cn_iter_t<double>(x) : cn_iter_t<float>(x);
}

template <class T>
static cudaError_t cn_finish_t(const Ctx& x) {
  BCM_DISPATCH_B(x.B, {
    constexpr int NT = threads_for<B>();
    k_cn_finish<B, NT, T><<<x.g.n_cubes, NT, 0, x.stream>>>(
        x.g, (const T*)x.f.u, (const T*)x.f.v, (const T*)x.f.w, (const T*)x.f.w1,
        (const T*)x.f.s0, (const T*)x.f.s1, (const T*)x.f.r, (const T*)x.f.p0,
        (const T*)x.f.p1, (T*)x.f.us, (T*)x.f.vs, (T*)x.f.ws, (const T*)x.f.phi, x.f.bid,
        (T*)x.f.ub);
  });
  return cudaGetLastError();
}
cudaError_t launch_cn_finish(const Ctx& x) {
  return x.f64 ? cn_finish_t<double>(x) : cn_finish_t<float>(x);
}

cudaError_t launch_bmean(const Ctx& x) {
  BCM_DISPATCH_B(x.B, {
    constexpr int NT = threads_for<B>();
    k_bmean<B, NT><<<x.g.n_cubes, NT, 0, x.stream>>>(x.g, x.f.b);
  });
  return cudaGetLastError();
}

cudaError_t launch_solve_begin(const Ctx& x) {
  k_solve_begin<<<1, 128, 0, x.stream>>>(x.g, x.f.guard);
  return cudaGetLastError();
}

cudaError_t launch_step_end(const Ctx& x) {
  k_step_end<<<1, 128, 0, x.stream>>>(x.g);
  return cudaGetLastError();
}

template <class T>
static cudaError_t fill_halo_t(const Ctx& x, const void* f, int kind, double* out) {
  BCM_DISPATCH_B(x.B, {
    constexpr int NT = threads_for<B>();
    k_fill_halo<B, NT, T><<<x.g.n_cubes, NT, 0, x.stream>>>(x.g, (const T*)f, kind,
                                                            (const T*)x.f.ub, out);
  });
  return cudaGetLastError();
}
cudaError_t launch_fill_halo(const Ctx& x, const void* f, int f64_field, int kind, double* out) {
  return f64_field ? fill_halo_t<double>(x, f, kind, out) : fill_halo_t<float>(x, f, kind, out);
}

}  // namespace bcm
