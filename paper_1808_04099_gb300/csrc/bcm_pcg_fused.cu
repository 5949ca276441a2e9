// bcm_pcg_fused.cu -- persistent Jacobi-PCG with one grid barrier per iteration, for the
// FP32 inner solve on 16^3 cubes (Eq. poisson; Saad, Alg. 9.1).
//
// The textbook iteration needs two global reductions: <p, K p> for alpha, then <r, z>
// for beta.  Here both come out of one pass.  Pass m takes alpha_{m-1} and beta_m and
// computes, cell by cell,
//     q_{m-1} = K p_{m-1},   x_m = x_{m-1} + alpha_{m-1} p_{m-1},
//     r_m = r_{m-1} - alpha_{m-1} q_{m-1},   z_m = D^-1 r_m,
//     p_m = z_m + beta_m p_{m-1},   q_m = K p_m,
// with the sums <p_m, q_m>, <q_m, z_m>, <q_m, D^-1 q_m>, <r_m, r_m> and <r_m, z_m>.
// After the barrier alpha_m = <r_m, z_m> / <p_m, q_m>, and since r_{m+1} = r_m -
// alpha_m q_m, <r_{m+1}, z_{m+1}> = <r_m, z_m> - 2 alpha_m <q_m, z_m> + alpha_m^2 <q_m,
// D^-1 q_m> follows from the same sums, which gives beta_{m+1} (the exact <r, z> of
// every pass still sets alpha).  The iterates are those of the textbook PCG in exact
// arithmetic; the convergence test reads <r_{m-1}, r_{m-1}> one pass later, and x_{m-1}
// is already stored then.  q is never stored: the pass applies K to p_{m-1} again
// (from the same staged tile), which costs shared-memory arithmetic instead of two
// vector streams.
//
// Work: one block of 256 threads per SM, each thread one x-row (16 cells) of the cube in
// hand, so both x faces end every thread's row and its x neighbours are its own values;
// block p owns a contiguous run of cubes by the paper's linear distribution
// (Eq. loaddist).  r, p and x are updated in place (only their owner touches a cube's
// cells); neighbours read a cube's boundary planes of r, q, p from a face array
// [parity][cube][face][r,q,p][16x16] that every pass writes in the other parity.  A
// cube's r, p, x (3 x 16 KB), its six neighbours' face blocks (3 KB each) and its
// constant record reach shared memory by bulk asynchronous copies (cp.async.bulk,
// completion on an mbarrier), two cubes ahead of the arithmetic in three rotating
// slots; the first two cubes of a pass have their own data copied before the grid
// barrier that ends the previous pass.  Values across the faces are read (or formed)
// from the staged face planes where they are needed, domain ghosts in place; only cubes
// with 2:1 faces stage ghosts first.  The first pass of a solve takes the residual
// kernel's r (and, resuming a defect-correction cycle, the previous direction) by
// plain loads for the halo.
//
// Every wait is bounded: mbarrier waits and the grid barrier give up after the solver's
// barrier timeout, set the error flag, wait (at most one second) for the block's copies
// in flight and return; the host reports BCM_E_TIMEOUT.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bcm_bulk.cuh"
#include "bcm_cube.cuh"
#include "bcm_internal.cuh"
#include "bcm_kernels.h"
#include "bcm_persist.cuh"

namespace bcm {

namespace {

constexpr int FB = 16, FBB = FB * FB, FB3 = FB * FB * FB;
constexpr int kFaceVals = 3 * FBB;        // r, q, p of one face plane
constexpr int kCubeFace = 6 * kFaceVals;  // face-array floats per cube and parity
constexpr int kMaxBlockCubes = 256;       // cubes one block may own
constexpr int kMaxFusedSims = 160;        // per-sim scalars fit beside the three stages

constexpr int kSlots = 3;                 // stage slots: two cubes ahead of the one in hand

struct alignas(128) FStage {
  float R[FB3], P[FB3];   // r_{m-1}, p_{m-1} (R then holds p_m)
  float F[6][kFaceVals];  // neighbour face planes: r, q, p each
  FCube cs;               // the cube's constants
};

struct FShared {
  FStage st[kSlots];
  float G1[6][FBB];       // 2:1 ghosts of p_{m-1}
  float G2[2][6][FBB];    // p_m across every face that is not a domain face, by cube parity
  unsigned long long mbar[kSlots];
  double red[ACC_FZ_N * 32];
  int bnb[kMaxBlockCubes][6];  // face neighbours of the block's cubes
  int bsim[kMaxBlockCubes];    // and their sims
  int cube[kMaxBlockCubes];    // this pass's cubes (local index; sims still running)
  int warp_n[32];
  int n_list;
  int pre[2];   // cubes (local index) whose own data was prefetched into slots 0 and 1
  int any_alive, any_finished;  // decisions of the pass: a sim runs / a sim just finished
};

// per-sim scalars after FShared in dynamic shared memory
struct FSim {
  double rzp;      // <r, z> the current direction is formed with
  float alpha, beta, gamma;
  int rpar;        // face-array parity this pass reads
  int done, cont;  // finished; first pass resumes the previous direction
};
// the three stages, the ghosts and the tables, the per-sim scalars of kMaxFusedSims sims
// and the kernels' static shared memory fit one block per SM (227 KB)
static_assert((sizeof(FShared) + 15) / 16 * 16 + sizeof(FSim) * kMaxFusedSims + 256 <= 232448,
              "fused PCG shared memory exceeds the per-block limit");

__device__ __forceinline__ float4 ld4s(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4s(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

// (i, j, k) of the cell at tangential (a, b) on face f of a cube, in the plane of that face
__device__ __forceinline__ void face_cell(int f, int a, int b, int& i, int& j, int& k) {
  const int d = f >> 1, n = (f & 1) ? FB - 1 : 0;
  int q[3];
  q[d] = n;
  q[tan1(d)] = a;
  q[tan2(d)] = b;
  i = q[0];
  j = q[1];
  k = q[2];
}

// Sum over the block of NV FP32 partials, in FP64 from the warp level up (FP32 warp
// shuffles: the part's FP64 rate is a small fraction of its FP32 rate); result in
// thread 0.
template <int NT, int NV>
__device__ __forceinline__ void block_sum_f(float (&v)[NV], double (&out)[NV], double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) red[q * 32 + warp] = double(v[q]);
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double x = lane < NT / 32 ? red[q * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      out[q] = x;
    }
  }
}

struct FusedArgs {
  const float* rp;  // residual kernel's r (first pass of a solve)
  float *r, *p, *x;
  float* face;
  const FCube* fc;  // per-cube constants
};

__device__ __forceinline__ size_t face_off(int par, int n_cubes, int c, int f) {
  return ((size_t)par * n_cubes + c) * kCubeFace + (size_t)f * kFaceVals;
}

// What the 2:1 ghosts need (kept out of the hot path's registers: the function is not
// inlined).  mode: kOldP p_{m-1} of the face planes, kNewP p_m from their r, q, p,
// kFirst the first pass of a solve (the residual kernel's r, and the resumed direction).
enum { kOldP = 0, kNewP = 1, kFirst = 2 };
struct GhostCtx {
  const int *aux, *ijk, *lvl, *w3, *sim;
  const SimParams* sp;
  const float *face, *rp;
  int max_level, nc, rpar, mode, cont;
  float alpha, beta, gamma;
};

// p at cell (a, b) of face fn of cube nn (from its face planes of the last pass, or,
// in the first pass, the residual kernel's r and the resumed direction).
// Face planes are written by other SMs during the launch: read them at L2 (__ldcg), past
// this SM's L1, which is not kept coherent with other SMs' stores.
__device__ float p_face(const GhostCtx& x, int nn, int fn, int a, int b) {
  const float* F = x.face + face_off(x.rpar, x.nc, nn, fn);
  const int o = b * FB + a;
  if (x.mode == kOldP) return __ldcg(F + 2 * FBB + o);
  int ii, jj, kk;
  face_cell(fn, a, b, ii, jj, kk);
  const SimParams& sp = x.sp[x.sim[nn]];
  const float iv = float(sp.invdiag[x.lvl[nn]][s3_of<FB>(x.w3 + 6 * nn, ii, jj, kk)]);
  if (x.mode == kNewP) {
    const float r = fmaf(-x.alpha, __ldcg(F + FBB + o), __ldcg(F + o));
    return fmaf(x.beta, __ldcg(F + 2 * FBB + o), r * iv);
  }
  const float r = x.rp[(size_t)nn * FB3 + (kk * FB + jj) * FB + ii];
  float pn = r * iv;
  if (x.cont) pn = fmaf(x.gamma, __ldcg(F + 2 * FBB + o) - __ldcg(F + o) * iv, pn);
  return pn;
}

// Poisson ghost across the 2:1 face f of cube c at (a, b) (R7): the coarse cell across
// the face (this cube fine), or the mean of the four fine cells touching this coarse
// face cell.
__device__ __noinline__ float ghost_21(const GhostCtx& x, int c, int f, int a, int b, int code) {
  const int d = f >> 1;
  if (code == NB_COARSE) {
    const int C = x.aux[(6 * c + f) * 4];
    const int sf = 1 << (x.max_level - x.lvl[c]), sc = 2 * sf;
    const int Ac = (x.ijk[3 * c + tan1(d)] + a * sf - x.ijk[3 * C + tan1(d)]) / sc;
    const int Bc = (x.ijk[3 * c + tan2(d)] + b * sf - x.ijk[3 * C + tan2(d)]) / sc;
    return p_face(x, C, f ^ 1, Ac, Bc);
  }
  const int qa = (2 * a) / FB, qb = (2 * b) / FB;
  const int Fc = x.aux[(6 * c + f) * 4 + qb * 2 + qa];
  const int fa = 2 * a - qa * FB, fb = 2 * b - qb * FB;
  return 0.25f * (p_face(x, Fc, f ^ 1, fa, fb) + p_face(x, Fc, f ^ 1, fa + 1, fb) +
                  p_face(x, Fc, f ^ 1, fa, fb + 1) + p_face(x, Fc, f ^ 1, fa + 1, fb + 1));
}

__device__ __forceinline__ void ld4v(const float* p, float (&v)[4]) {
  const float4 a = ld4s(p);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}

// 1 / diag(K) of the same-level neighbour's cell across face f at tangential (a, b)
__device__ __forceinline__ float nb_inv(const FCube& cs, int f, int a, int b) {
  if (cs.nbmask[f] == 0) return cs.invtab[18];
  int i, j, k;
  face_cell(f ^ 1, a, b, i, j, k);
  return cs.invtab[s3_of<FB>(cs.nbw3[f], i, j, k)];
}

// The mirror factor of a domain face (the ghost is the mirror cell's value, Neumann,
// negated at the outflow's Dirichlet 0), 0 for a face that is not a domain face.
__device__ __forceinline__ float dom_sign(const FCube& cs, int f) {
  return cs.nb[f] == NB_BOUNDARY ? (cs.bc[f] == BC_OUTFLOW ? -1.f : 1.f) : 0.f;
}

// q = K p on quad u from the tile T (the cube's p, x fastest) and what lies across the
// cube's faces: for a face that is not a domain face the value comes from the plane at
// across + f * stride (16 x 16, tangential (a, b) at b * 16 + a), for a domain face it is
// the mirror cell's value times dom_sign.  h times the sum over the six faces of
// (p_c - p_nb), 2:1 faces weighted (R7).  No branch on the lane: a face cell reads its
// plane where an interior cell reads the tile.  The x neighbours inside the cube come from
// the adjacent quads of the warp (lanes hold consecutive quads); every lane of the warp
// must call it.
__device__ __forceinline__ void stencil_quad(const FCube& cs, const float* T, const float* across,
                                             int stride, const float (&pv)[4], int u,
                                             float (&qv)[4]) {
  const int i0 = (u & 3) * 4, j = (u >> 2) & 15, kz = u >> 6;
  const float left = __shfl_up_sync(0xffffffffu, pv[3], 1);
  const float right = __shfl_down_sync(0xffffffffu, pv[0], 1);
  float sum[4];
  {
    const bool f0 = i0 == 0, f1 = i0 == FB - 4;
    const float g0 = across[kz * FB + j], g1 = across[stride + kz * FB + j];
    const float s0 = dom_sign(cs, 0), s1 = dom_sign(cs, 1);
    const float xl = f0 ? (s0 != 0.f ? s0 * pv[0] : g0) : left;
    const float xr = f1 ? (s1 != 0.f ? s1 * pv[3] : g1) : right;
    const float wl = f0 ? cs.wt[0] : 1.f, wr = f1 ? cs.wt[1] : 1.f;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float xm = e == 0 ? xl : pv[e - 1], xp = e == 3 ? xr : pv[e + 1];
      sum[e] = (e == 0 ? wl : 1.f) * (pv[e] - xm) + (e == 3 ? wr : 1.f) * (pv[e] - xp);
    }
  }
  auto side = [&](int f, bool inside, int off, int o) {
    const float* src = inside ? T + 4 * u + off : across + f * stride + o;
    const float4 a = ld4s(src);
    float nv[4] = {a.x, a.y, a.z, a.w};
    const float w = inside ? 1.f : cs.wt[f];
    const float sg = inside ? 0.f : dom_sign(cs, f);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (sg != 0.f) nv[e] = sg * pv[e];
      sum[e] = fmaf(w, pv[e] - nv[e], sum[e]);
    }
  };
  side(2, j > 0, -FB, kz * FB + i0);
  side(3, j < FB - 1, FB, kz * FB + i0);
  side(4, kz > 0, -FBB, j * FB + i0);
  side(5, kz < FB - 1, FBB, j * FB + i0);
#pragma unroll
  for (int e = 0; e < 4; ++e) qv[e] = cs.h * sum[e];
}

// 1 / diag(K) of the four cells of quad (i0, j, kz): the face-weight sum differs from
// the interior one only on the cube's faces (R7), and along x only at the quad's ends.
__device__ __forceinline__ void quad_inv(const FCube& cs, int i0, int j, int kz, float (&iv)[4]) {
  if (cs.smask == 0) {
    iv[0] = iv[1] = iv[2] = iv[3] = cs.invtab[18];
    return;
  }
  const int s = 18 + (j == 0 ? cs.w3[2] - 3 : 0) + (j == FB - 1 ? cs.w3[3] - 3 : 0) +
                (kz == 0 ? cs.w3[4] - 3 : 0) + (kz == FB - 1 ? cs.w3[5] - 3 : 0);
  iv[0] = cs.invtab[s + (i0 == 0 ? cs.w3[0] - 3 : 0)];
  iv[1] = iv[2] = cs.invtab[s];
  iv[3] = cs.invtab[s + (i0 == FB - 4 ? cs.w3[1] - 3 : 0)];
}

// Quad u of vector v on the face planes it lies on (written parity).
__device__ __forceinline__ void face_store(float* fw, int v, const float (&x)[4], int u) {
  const int i0 = (u & 3) * 4, j = (u >> 2) & 15, kz = u >> 6;
  float* b = fw + v * FBB;
  if (i0 == 0) b[0 * kFaceVals + kz * FB + j] = x[0];
  if (i0 == FB - 4) b[1 * kFaceVals + kz * FB + j] = x[3];
  if (j == 0) st4s(b + 2 * kFaceVals + kz * FB + i0, x[0], x[1], x[2], x[3]);
  if (j == FB - 1) st4s(b + 3 * kFaceVals + kz * FB + i0, x[0], x[1], x[2], x[3]);
  if (kz == 0) st4s(b + 4 * kFaceVals + j * FB + i0, x[0], x[1], x[2], x[3]);
  if (kz == FB - 1) st4s(b + 5 * kFaceVals + j * FB + i0, x[0], x[1], x[2], x[3]);
}

}  // namespace

constexpr int FNT = 1024;  // threads per block: one x-quad of the cube in hand each

__global__ __launch_bounds__(FNT, 1) void k_pcg_fused(DevGrid g, FusedArgs A, SolveParams prm,
                                                      unsigned int* bar, int* err) {
  constexpr int NT = FNT, NW = NT / 32;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  FShared& S = *reinterpret_cast<FShared*>(smem_raw);
  FSim* sim = reinterpret_cast<FSim*>(smem_raw + (sizeof(FShared) + 15) / 16 * 16);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int nsim = g.n_sims, nc = g.n_cubes;
  const bool inner = prm.mixed != 0;
  const int kmax = inner ? prm.inner_max_iter : prm.max_iter;
  const unsigned long long limit = prm.barrier_timeout_ns;
  // my cubes by the linear load-balanced distribution
  const int P = gridDim.x, pb = blockIdx.x;
  const int Lq = nc / P, Rq = nc % P;
  const int c0 = pb * Lq + min(pb, Rq), ncub = (nc + P - pb - 1) / P;
  // this thread's quad (cells i0 .. i0+3 of row (j, kz)) and, for lanes 0 .. 11 of every
  // warp, one of the 384 face quads whose values across the face it forms
  const int i0 = (t & 3) * 4, j = (t >> 2) & 15, kz = t >> 6;
  const int gq = lane < 12 ? 12 * warp + lane : -1;

  for (int s = t; s < nsim; s += NT) {
    sim[s].done = g.ss[s].done ? 1 : 0;
    sim[s].rpar = g.ss[s].fz_par & 1;
  }
  for (int i = t; i < 7 * ncub; i += NT) {  // the block's neighbour table and sims
    const int q = i / 7, e = i - 7 * q;
    if (e < 6) S.bnb[q][e] = g.nb[6 * (c0 + q) + e];
    else S.bsim[q] = g.sim[c0 + q];
  }
  if (t == 0) {
    // two arrivals per phase: the cube's own data, then its neighbours' face planes
    for (int k = 0; k < kSlots; ++k) mbar_init(&S.mbar[k], 2);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    S.pre[0] = S.pre[1] = -1;
    S.any_alive = S.any_finished = 0;
  }
  __syncthreads();
  unsigned phase[kSlots] = {0u, 0u, 0u};
  int pend[kSlots] = {0, 0, 0};  // copies issued into a slot and not yet waited for
  GridBarrier gb;
  gb.init(bar, err, limit);
  bool failed = false;
  constexpr int IW = NW - 1;  // the warp that issues copies

  // own data of cube ql into slot sl (issuing warp): r and p (the residual kernel's r
  // and the previous direction in the first pass) and the constants
  auto issue_own = [&](int ql, int sl, bool first) {
    const int c = c0 + ql;
    const FSim& fs = sim[S.bsim[ql]];
    FStage& stg = S.st[sl];
    const size_t base = (size_t)c * FB3;
    const float* src = nullptr;
    float* dst = nullptr;
    if (lane == 0) {
      src = (first ? A.rp : A.r) + base;
      dst = stg.R;
    } else if (lane == 1 && (!first || fs.cont)) {
      src = A.p + base;
      dst = stg.P;
    }
    const bool ocopy = src != nullptr, rcopy = lane == 3;
    unsigned bytes = (ocopy ? 4u * FB3 : 0u) + (rcopy ? (unsigned)sizeof(FCube) : 0u);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
    if (lane == 0) mbar_expect_tx(&S.mbar[sl], bytes);
    __syncwarp();
    if (ocopy) bulk_g2s(dst, src, 4u * FB3, &S.mbar[sl]);
    if (rcopy) bulk_g2s(&stg.cs, A.fc + c, (unsigned)sizeof(FCube), &S.mbar[sl]);
  };
  // the neighbours' face planes of cube ql into slot sl (issuing warp)
  auto issue_faces = [&](int ql, int sl, bool first, bool none) {
    // the planes were written by other blocks before the grid barrier this thread has
    // passed (acquire by thread 0, block barrier): order that before the bulk reads
    fence_async_global();
    const FSim& fs = sim[S.bsim[ql]];
    int n = -1;
    if (lane < 6) n = S.bnb[ql][lane];
    const bool fcopy = !none && lane < 6 && n >= 0 && (!first || fs.cont);
    unsigned bytes = fcopy ? 4u * kFaceVals : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
    if (lane == 0) mbar_expect_tx(&S.mbar[sl], bytes);
    __syncwarp();
    if (fcopy)
      bulk_g2s(S.st[sl].F[lane], A.face + face_off(fs.rpar, nc, n, lane ^ 1), 4u * kFaceVals,
               &S.mbar[sl]);
  };

  for (int m = 0;; ++m) {
    const bool first = (m == 0);
    // ---- decisions for pass m (the same in every block): warp w takes sims w, w + NW ..;
    // its lanes read the 5 x kStripes sums of the last pass together
    int alive = 0, finished = 0;
    for (int s = warp; s < nsim; s += NW) {
      FSim& fs = sim[s];
      if (fs.done) continue;
      SimState& st = g.ss[s];
      double v[ACC_FZ_N] = {0.0, 0.0, 0.0, 0.0, 0.0};
      if (m == 0) {
        v[3] = st.rr;
        v[4] = st.rz;
      } else {
        const int b0 = ACC_SLOT_FZ + ACC_FZ_N * ((m - 1) % 3);
        // lane = q * 8 + stripe for the first four sums, lanes 0..7 again for the fifth
        double a = ld_acc(&st.acc[lane & 7][b0 + (lane >> 3)]);
        double b5 = lane < kStripes ? ld_acc(&st.acc[lane][b0 + 4]) : 0.0;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b5 += __shfl_xor_sync(0xffffffffu, b5, o);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = __shfl_sync(0xffffffffu, a, 8 * q);
        v[4] = __shfl_sync(0xffffffffu, b5, 0);
      }
      if (lane != 0) continue;
      const double pq = v[0], qz = v[1], qdq = v[2], rr = v[3], rz = v[4];
      const int iters = m > 0 ? m - 1 : 0;  // x updates done so far
      const double tol2 = inner ? st.inner_tol2 : st.tol2;
      const bool bad = !isfinite(rr) || !isfinite(rz) || !isfinite(pq) || !isfinite(qz) ||
                       !isfinite(qdq);
      if (bad || rr <= tol2 || iters >= kmax) {
        fs.done = 1;
        finished = 1;
        if (blockIdx.x == 0) {  // single writer of the solve's results
          st.iter = iters;
          st.total_iters += iters;
          st.rr = rr;
          st.done = 1;
          if (m > 0) {  // r, p and the faces of pass m-1 are the state to resume from
            st.fz_par = fs.rpar ^ 1;
            st.fz_valid = 1;
            st.fz_rzpred = fs.rzp;
          }
          if (bad) st.nonfinite = 1;
          if (!inner) {
            st.rr64 = rr;
            st.converged = !bad && rr <= tol2;
          }
        }
        continue;
      }
      if (m == 0) {
        const bool cont = st.cont != 0 && st.fz_valid != 0;
        fs.cont = cont ? 1 : 0;
        fs.alpha = 0.f;
        fs.beta = 0.f;
        fs.gamma = (cont && st.fz_rzpred > 0.0) ? float(rz / st.fz_rzpred) : 0.f;
        fs.rzp = rz;
        fs.rpar = st.fz_par & 1;
      } else {
        const double al = (pq != 0.0) ? rz / pq : 0.0;
        const double rzp = rz - 2.0 * al * qz + al * al * qdq;
        fs.alpha = float(al);
        fs.beta = (rzp > 0.0 && rz > 0.0) ? float(rzp / rz) : 0.f;
        fs.rzp = rzp;
        fs.rpar ^= 1;  // read what pass m-1 wrote
        fs.cont = 0;
      }
      alive = 1;
    }
    // one barrier publishes the decisions and whether the cube list changed
    if (alive) S.any_alive = 1;
    if (finished) S.any_finished = 1;
    __syncthreads();
    alive = S.any_alive;
    finished = S.any_finished;
    if (!alive) break;
    if (blockIdx.x == 0)  // clear the slot pass m+1 fills (held pass m-2's sums)
      for (int i = t; i < nsim * kStripes; i += NT) {
        SimState& st = g.ss[i / kStripes];
        const int b0 = ACC_SLOT_FZ + ACC_FZ_N * ((m + 1) % 3);
#pragma unroll
        for (int q = 0; q < ACC_FZ_N; ++q) st.acc[i % kStripes][b0 + q] = 0.0;
      }
    // ---- this pass's cubes: those of running sims, in order (a warp-ballot compaction),
    // rebuilt when a sim has finished
    if (first || finished) {
      const bool mine = t < ncub && !sim[S.bsim[t]].done;
      const unsigned bal = __ballot_sync(0xffffffffu, mine);
      if (lane == 0) S.warp_n[warp] = __popc(bal);
      __syncthreads();
      int off = 0;
      for (int w = 0; w < warp; ++w) off += S.warp_n[w];
      if (mine) S.cube[off + __popc(bal & ((1u << lane) - 1u))] = t;
      if (t == NT - 1) S.n_list = off + __popc(bal);
      __syncthreads();
    }
    const int nl = S.n_list;

    // the first two cubes: their own data may already be on its way (prefetched before
    // the barrier); the face planes follow now.  Every thread decides alike from the
    // same shared tables whether a prefetch went unused (then the issuing warp completes
    // its phase and lets it land first).
    for (int q = 0; q < 2; ++q) {
      const int pq = S.pre[q];
      const bool unused = pq >= 0 && (q >= nl || S.cube[q] != pq);
      if (unused) {
        if (warp == IW) {
          issue_faces(pq, q, false, true);
          mbar_wait(&S.mbar[q], phase[q], 1000000000ull);
        }
        phase[q] ^= 1u;
        pend[q] = 0;
      }
      if (q < nl) {
        if (warp == IW) {
          if (unused || pq != S.cube[q]) issue_own(S.cube[q], q, first);
          issue_faces(S.cube[q], q, first, false);
        }
        pend[q] = 1;
      }
    }

    // dot-product partials of the block's current sim
    float acc[ACC_FZ_N] = {0.f, 0.f, 0.f, 0.f, 0.f};  // pq, qz, qdq, rr, rz
    int psim = -1;
    auto flush = [&]() {
      double out[ACC_FZ_N];
      block_sum_f<NT, ACC_FZ_N>(acc, out, S.red);
      if (t == 0) {
        SimState& st = g.ss[psim];
        const int b0 = ACC_SLOT_FZ + ACC_FZ_N * (m % 3);
#pragma unroll
        for (int q = 0; q < ACC_FZ_N; ++q) acc_add(st, b0 + q, out[q]);
      }
#pragma unroll
      for (int q = 0; q < ACC_FZ_N; ++q) acc[q] = 0.f;
    };

    // x of the first cube (plain loads, one cube ahead from then on)
    float xn[4] = {0.f, 0.f, 0.f, 0.f};
    if (!first && nl > 0) ld4v(A.x + (size_t)(c0 + S.cube[0]) * FB3 + 4 * t, xn);
    for (int q = 0; q < nl; ++q) {
      const int sl = q % kSlots, ql = S.cube[q], c = c0 + ql, s = S.bsim[ql];
      if (psim >= 0 && psim != s) flush();
      psim = s;
      float xc[4] = {xn[0], xn[1], xn[2], xn[3]};
      if (!first && q + 1 < nl) ld4v(A.x + (size_t)(c0 + S.cube[q + 1]) * FB3 + 4 * t, xn);
      // a timed-out wait leaves the stage unread by the warp: every barrier below is a
      // vote on it, so all threads leave the loop together
      const bool okw = __all_sync(0xffffffffu, mbar_wait(&S.mbar[sl], phase[sl], limit));
      const FSim& fs = sim[s];
      const FCube& cs = S.st[sl].cs;
      FStage& stg = S.st[sl];
      const bool cont = fs.cont != 0;
      const float alpha = fs.alpha, beta = fs.beta, gamma = fs.gamma;
      float* fw = A.face + face_off(fs.rpar ^ 1, nc, c, 0);  // this cube's faces, written
      const size_t base = (size_t)c * FB3;
      float (*G2)[FBB] = S.G2[q & 1];
      if (okw && cs.has21 && !first) {
        // 2:1 faces: the flux-form ghosts (R7) of p_{m-1}, between two barriers (the
        // previous cube may still read G1)
        if (__syncthreads_or(!okw)) {
          failed = true;
          break;
        }
        if (gq >= 0) {  // every face plane of p_{m-1} into G1 (the stencil reads one array)
          const int f = gq >> 6, qf = gq & 63, a0 = 4 * (qf & 3), b = qf >> 2;
          const int n = cs.nb[f], o = b * FB + a0;
          if (n >= 0) {
            float pq4[4];
            ld4v(stg.F[f] + 2 * FBB + o, pq4);
            st4s(&S.G1[f][o], pq4[0], pq4[1], pq4[2], pq4[3]);
          } else if (n < NB_BOUNDARY) {
            const GhostCtx gc{g.aux, g.ijk, g.lvl, g.w3, g.sim, g.sp, A.face, A.rp,
                              g.max_level, nc, fs.rpar, kOldP, 0, alpha, beta, gamma};
            for (int e = 0; e < 4; ++e) S.G1[f][o + e] = ghost_21(gc, c, f, a0 + e, b, n);
          }
        }
        __syncthreads();
      }
      float zv[4], pv[4], iv[4];
      if (okw) {
        // ---- p_m across the faces (lanes 0..11 of every warp, one face quad each)
        if (gq >= 0) {
          const int f = gq >> 6, qf = gq & 63, a0 = 4 * (qf & 3), b = qf >> 2;
          const int n = cs.nb[f], o = b * FB + a0;
          if (n >= 0) {  // same level: formed from the neighbour's planes of r, q, p
            float gv[4];
            if (first && !cont) {
#pragma unroll
              for (int e = 0; e < 4; ++e) gv[e] = 0.f;
            }
            const float* F = stg.F[f];
            float fr[4] = {0.f, 0.f, 0.f, 0.f}, fq[4] = {0.f, 0.f, 0.f, 0.f},
                  fp[4] = {0.f, 0.f, 0.f, 0.f};
            if (!first || cont) {
              ld4v(F + o, fr);
              ld4v(F + FBB + o, fq);
              ld4v(F + 2 * FBB + o, fp);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float ivn = nb_inv(cs, f, a0 + e, b);
              if (!first) {
                gv[e] = fmaf(beta, fp[e], fmaf(-alpha, fq[e], fr[e]) * ivn);
              } else {
                int ii, jj, kk;
                face_cell(f ^ 1, a0 + e, b, ii, jj, kk);
                gv[e] = A.rp[(size_t)n * FB3 + (kk * FB + jj) * FB + ii] * ivn;
                if (cont) gv[e] = fmaf(gamma, fp[e] - fr[e] * ivn, gv[e]);
              }
            }
            st4s(&G2[f][o], gv[0], gv[1], gv[2], gv[3]);
          } else if (n < NB_BOUNDARY) {  // 2:1 face: flux-form ghost (R7)
            const GhostCtx gc{g.aux, g.ijk, g.lvl, g.w3, g.sim, g.sp, A.face, A.rp,
                              g.max_level, nc, fs.rpar, first ? kFirst : kNewP, cont ? 1 : 0,
                              alpha, beta, gamma};
            for (int e = 0; e < 4; ++e) G2[f][o + e] = ghost_21(gc, c, f, a0 + e, b, n);
          }
        }
        // ---- q_{m-1} = K p_{m-1}, then r_m, x_m, p_m of my quad
        quad_inv(cs, i0, j, kz, iv);
        float rv[4], po[4] = {0.f, 0.f, 0.f, 0.f};
        ld4v(stg.R + 4 * t, rv);
        if (!first || cont) ld4v(stg.P + 4 * t, po);
        if (!first) {
          // p_{m-1} across the faces: the staged planes, or G1 on a cube with 2:1 faces
          const float* acr = cs.has21 ? &S.G1[0][0] : stg.F[0] + 2 * FBB;
          const int stride = cs.has21 ? FBB : kFaceVals;
          float qo[4];
          stencil_quad(cs, stg.P, acr, stride, po, t, qo);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            xc[e] = fmaf(alpha, po[e], xc[e]);
            rv[e] = fmaf(-alpha, qo[e], rv[e]);
          }
          st4s(A.x + base + 4 * t, xc[0], xc[1], xc[2], xc[3]);
        }
        float ro[4] = {0.f, 0.f, 0.f, 0.f};
        if (first && cont) ld4v(A.r + base + 4 * t, ro);  // the previous recurrence residual
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          zv[e] = rv[e] * iv[e];
          if (!first) pv[e] = fmaf(beta, po[e], zv[e]);
          else if (cont) pv[e] = fmaf(gamma, po[e] - ro[e] * iv[e], zv[e]);  // z + g (p - D^-1 r)
          else pv[e] = zv[e];
          acc[3] = fmaf(rv[e], rv[e], acc[3]);
          acc[4] = fmaf(rv[e], zv[e], acc[4]);
        }
        // p_m replaces r in the stage (only this thread reads its quad of R)
        st4s(stg.R + 4 * t, pv[0], pv[1], pv[2], pv[3]);
        st4s(A.r + base + 4 * t, rv[0], rv[1], rv[2], rv[3]);
        st4s(A.p + base + 4 * t, pv[0], pv[1], pv[2], pv[3]);
        face_store(fw, 0, rv, t);
        face_store(fw, 2, pv, t);
      }
      // one barrier: the copies had landed for every thread, the tile and G2 hold p_m
      if (__syncthreads_or(!okw)) {  // the slot's copies stay pending
        failed = true;
        break;
      }
      phase[sl] ^= 1u;
      pend[sl] = 0;
      // the slot of cube q-1 is free (every thread fenced its accesses before the
      // barrier above): refill it with cube q+2
      if (q + 2 < nl) {
        const int s2 = (q + 2) % kSlots;
        if (warp == IW) {
          issue_own(S.cube[q + 2], s2, first);
          issue_faces(S.cube[q + 2], s2, first, false);
        }
        pend[s2] = 1;
      }
      // ---- B: q_m = K p_m on my quad
      {
        float qv[4];
        stencil_quad(cs, stg.R, &G2[0][0], FBB, pv, t, qv);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          acc[0] = fmaf(pv[e], qv[e], acc[0]);
          acc[1] = fmaf(qv[e], zv[e], acc[1]);
          acc[2] = fmaf(qv[e] * iv[e], qv[e], acc[2]);
        }
        face_store(fw, 1, qv, t);
      }
      // this thread is done with the slot: order its accesses before the slot's next
      // bulk copy (issued after a later barrier)
      fence_async_shared();
    }
    if (failed) break;
    // this pass's global writes, before the barrier, for the next pass's bulk copies
    // (the flush's barriers order every thread's fence before the prefetch below)
    fence_async_global();
    if (psim >= 0) flush();
    else __syncthreads();
    // prefetch the own data of this pass's first two cubes for the next pass (this
    // block wrote it; their face planes wait for the barrier)
    if (warp == IW)
      for (int q = 0; q < 2 && q < nl; ++q) issue_own(S.cube[q], q, false);
    if (t == 0) {
      for (int q = 0; q < 2; ++q) S.pre[q] = q < nl ? S.cube[q] : -1;
      S.any_alive = S.any_finished = 0;  // every thread read them at the pass's start
    }
    for (int q = 0; q < 2 && q < nl; ++q) pend[q] = 1;
    if (!gb.sync()) {
      failed = true;
      break;
    }
  }
  if (failed) {
    if (t == 0) atomicExch(err, 1);
  }
  // a prefetch that no pass used: complete its phase (no face planes) and let it land;
  // on failure let every copy in flight land (a copy of at most 68 KB takes
  // microseconds; the drain is bounded by one second, not by the solver's timeout, which
  // a test may set to nanoseconds)
  __syncthreads();
  if (warp == IW)
    for (int q = 0; q < 2; ++q)
      if (S.pre[q] >= 0 && pend[q]) issue_faces(S.pre[q], q, false, true);
  for (int sl = 0; sl < kSlots; ++sl)
    if (pend[sl]) mbar_wait(&S.mbar[sl], phase[sl], 1000000000ull);
  if (failed) return;
  if (blockIdx.x == 0 && t == 0) g.flags[0] = 1;
}

// ---------------------------------------------------------------- launcher

cudaError_t launch_pcg_fused(const Ctx& x, const SolveParams& prm, bool* launched) {
  *launched = false;
  if (x.solve64 || x.B != FB || !x.f.face || !x.f.fcube || x.g.n_sims > kMaxFusedSims)
    return cudaSuccess;
  const size_t sm = (sizeof(FShared) + 15) / 16 * 16 + sizeof(FSim) * (size_t)x.g.n_sims;
  auto kern = k_pcg_fused;
  {
    const cudaError_t e = allow_dynamic_smem(kern, sm);
    if (e != cudaSuccess) return e;
  }
  int maxg = 0;
  const int rc = max_coresident(kern, FNT, sm, &maxg);
  if (rc) return (cudaError_t)rc;
  if (maxg < 1) return cudaSuccess;
  const int grid = x.g.n_cubes < maxg ? x.g.n_cubes : maxg;
  if ((x.g.n_cubes + grid - 1) / grid > kMaxBlockCubes) return cudaSuccess;
  DevGrid gg = x.g;
  FusedArgs a;
  a.rp = (const float*)x.f.r;
  a.r = (float*)x.f.w1;
  a.p = (float*)x.f.p0;
  a.x = x.f.e;
  a.face = x.f.face;
  a.fc = x.f.fcube;
  SolveParams pp = prm;
  unsigned int* bar = x.f.bar;
  int* err = x.f.err;
  void* args[] = {&gg, &a, &pp, &bar, &err};
  *launched = true;
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(FNT), args, sm, x.stream);
}

}  // namespace bcm
