// bcm_cube.cuh -- block-level helpers of the whole-cube stencil kernels:
// per-cube constants in shared memory, 4-wide vector access along x, and staging
// of a pressure-like field (Neumann / outflow-Dirichlet ghosts) with its face halo.
#pragma once

#include "bcm_internal.cuh"

namespace bcm {

// ---- four consecutive values along x: one float4, or two double2 (16-byte accesses)
__device__ __forceinline__ void ld4(const float* __restrict__ p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* __restrict__ p, double (&v)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* __restrict__ p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* __restrict__ p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// ---- per-cube constants shared by a block
template <class TV>
struct CubeSh {
  int nb[6];        // face neighbours / NB_* codes
  int w3[6];        // Jacobi face weights (thirds) of this cube
  int nbw3[6][6];   // ... of each same-level neighbour
  int bc[6];        // the sim's domain-face conditions
  int has21;        // some face of this cube is a 2:1 level interface
  int smask;        // bit f set: face f's Jacobi weight is not the same-level 3 (thirds)
  int nbmask[6];    // ... of each same-level neighbour
  TV wt[6];         // flux weight of a face relative to a same-level face: 1, 2/3, 4/3
  TV invtab[kW3];   // 1 / diag(K) by face-weight sum
};

// Needs blockDim.x >= 37 (neighbour masks need 70; smaller blocks compute them in a
// loop below); the caller synchronises afterwards.
template <class TV>
__device__ __forceinline__ void load_cube(CubeSh<TV>& cs, const DevGrid& g, int c) {
  const int t = threadIdx.x;
  if (!bcm_expect(g, c >= 0 && c < g.n_cubes, CHK_CUBE)) c = 0;
  int s = g.sim[c], lv = g.lvl[c];
  if (!bcm_expect(g, s >= 0 && s < g.n_sims && lv >= 0 && lv <= g.max_level, CHK_SIM)) {
    s = 0;  // read valid tables; the host reports the failure
    lv = 0;
  }
  const SimParams& sp = g.sp[s];
  if (t < 6) {
    const int n = checked_nb(g, g.nb[6 * c + t]);
    cs.nb[t] = n;
    cs.w3[t] = g.w3[6 * c + t];
    cs.bc[t] = sp.bc[t];
    // R7: a fine face towards a coarse cube carries A/d = h_f / 1.5, a coarse face
    // towards four fine cubes 4 (h_f^2 / 0.75 h_c) = (4/3) h_c
    cs.wt[t] = n == NB_COARSE ? TV(2.0 / 3.0) : (n == NB_FINE ? TV(4.0 / 3.0) : TV(1));
  }
  if (t == 0) {
    int any = 0, m = 0;
    for (int f = 0; f < 6; ++f) {
      any |= checked_nb(g, g.nb[6 * c + f]) < NB_BOUNDARY;
      m |= (g.w3[6 * c + f] != 3) << f;
    }
    cs.has21 = any;
    cs.smask = m;
  }
  if (blockDim.x >= 70 ? (t >= 64 && t < 70) : (t == 1)) {
    const int f0 = blockDim.x >= 70 ? t - 64 : 0, f1 = blockDim.x >= 70 ? f0 + 1 : 6;
    for (int f = f0; f < f1; ++f) {
      int m = 0;
      for (int e = 0; e < 6; ++e) m |= (g.nbw3[36 * c + 6 * f + e] != 3) << e;
      cs.nbmask[f] = m;
    }
  }
  if (t < 36) cs.nbw3[t / 6][t - 6 * (t / 6)] = g.nbw3[36 * c + t];
  if (t < kW3) cs.invtab[t] = TV(sp.invdiag[lv][t]);
}

// Face-weight sum (thirds) of cell (i, j, k) of a cube with face weights w3.
template <int B>
__device__ __forceinline__ int s3_of(const int* w3, int i, int j, int k) {
  return 18 + (i == 0 ? w3[0] - 3 : 0) + (i == B - 1 ? w3[1] - 3 : 0) +
         (j == 0 ? w3[2] - 3 : 0) + (j == B - 1 ? w3[3] - 3 : 0) +
         (k == 0 ? w3[4] - 3 : 0) + (k == B - 1 ? w3[5] - 3 : 0);
}

// 1 / diag(K) of a cell of any cube, from the global tables (2:1 neighbours).
template <int B, class TV>
__device__ __forceinline__ TV inv_diag_any(const DevGrid& g, int cube, int cell) {
  const int i = cell % B, j = (cell / B) % B, k = cell / (B * B);
  return TV(g.sp[g.sim[cube]].invdiag[g.lvl[cube]][s3_of<B>(g.w3 + 6 * cube, i, j, k)]);
}

// Poisson ghost across a 2:1 face f of cube c at tangential (a, b) (R7): the coarse
// cell across the face (fine side), or the mean of the four fine cells that touch
// the coarse face cell (coarse side).  valg(cube, cell) is the field value.  On the
// multigrid's per-cube level lsh the cells span 2^lsh level-0 cells (B per edge).
template <int B, class TV, class ValG>
__device__ __forceinline__ TV poisson_ghost_21(const DevGrid& g, int c, int f, int a, int b,
                                               int code, const ValG& valg, int lsh = 0) {
  const int d = f >> 1, side = f & 1;
  if (code == NB_COARSE) {
    const int C = g.aux[(6 * c + f) * 4];
    if (!bcm_expect(g, C >= 0 && C < g.n_cubes, CHK_AUX)) return TV(0);
    const int sf = (1 << (g.max_level - g.lvl[c])) << lsh, sc = 2 * sf;
    const int A = (g.ijk[3 * c + tan1(d)] + a * sf - g.ijk[3 * C + tan1(d)]) / sc;
    const int Bb = (g.ijk[3 * c + tan2(d)] + b * sf - g.ijk[3 * C + tan2(d)]) / sc;
    if (!bcm_expect(g, A >= 0 && A < B && Bb >= 0 && Bb < B, CHK_CELL)) return TV(0);
    return valg(C, cell_of<B>(d, side ? 0 : B - 1, A, Bb));
  }
  const int qa = (2 * a) / B, qb = (2 * b) / B;
  const int F = g.aux[(6 * c + f) * 4 + qb * 2 + qa];
  if (!bcm_expect(g, F >= 0 && F < g.n_cubes, CHK_AUX)) return TV(0);
  const int fa = 2 * a - qa * B, fb = 2 * b - qb * B;
  TV sum = TV(0);
  for (int bb = 0; bb < 2; ++bb)
    for (int aa = 0; aa < 2; ++aa) sum += valg(F, cell_of<B>(d, side ? 0 : B - 1, fa + aa, fb + bb));
  return TV(0.25) * sum;
}

// Tile positions of face f's ghost cell and of its mirror interior cell at (a, b).
template <int B>
__device__ __forceinline__ int ghost_pos(int f, int a, int b) {
  using SL = Slab<B, B>;
  switch (f) {
    case 0: return SL::at(-1, a, b + 1);
    case 1: return SL::at(B, a, b + 1);
    case 2: return SL::at(a, -1, b + 1);
    case 3: return SL::at(a, B, b + 1);
    case 4: return SL::at(a, b, 0);
    default: return SL::at(a, b, B + 1);
  }
}
template <int B>
__device__ __forceinline__ int mirror_pos(int f, int a, int b) {
  using SL = Slab<B, B>;
  switch (f) {
    case 0: return SL::at(0, a, b + 1);
    case 1: return SL::at(B - 1, a, b + 1);
    case 2: return SL::at(a, 0, b + 1);
    case 3: return SL::at(a, B - 1, b + 1);
    case 4: return SL::at(a, b, 1);
    default: return SL::at(a, b, B);
  }
}

// Stage a pressure-like field of a whole cube into the (B+2)^3 tile S:
//   own4(q4, i0, j, k, v[4]) -> the 4 cells starting at cell 4*q4 of this cube;
//   nbv(f, n, cell)          -> a cell of same-level neighbour n across face f;
// domain faces get the pressure ghost (mirror, or minus the mirror at outflow).
// Ends with the tile complete and the block synchronised.
template <int B, int NT, class TV, class Own, class Nbv, class ValG>
__device__ __forceinline__ void stage_pressure_cube(TV* __restrict__ S, const CubeSh<TV>& cs,
                                                    const DevGrid& g, int c, const Own& own4,
                                                    const Nbv& nbv, const ValG& valg) {
  using SL = Slab<B, B>;
  constexpr int B3 = B * B * B, BB = B * B;
  poison_tile(S, SL::N);
  for (int q4 = threadIdx.x; q4 < B3 / 4; q4 += NT) {
    const int cell = 4 * q4, i0 = cell % B, j = (cell / B) % B, k = cell / BB;
    TV v[4];
    own4(q4, i0, j, k, v);
    const int o = SL::at(i0, j, k + 1);
    S[o] = v[0];
    S[o + 1] = v[1];
    S[o + 2] = v[2];
    S[o + 3] = v[3];
  }
  for (int idx = threadIdx.x; idx < 6 * BB; idx += NT) {
    const int f = idx / BB, t = idx - f * BB, b = t / B, a = t - b * B;
    const int n = cs.nb[f];
    if (n >= 0) S[ghost_pos<B>(f, a, b)] = nbv(f, n, cell_of<B>(f >> 1, (f & 1) ? 0 : B - 1, a, b));
    else if (n < NB_BOUNDARY) S[ghost_pos<B>(f, a, b)] = poisson_ghost_21<B, TV>(g, c, f, a, b, n, valg);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 6 * BB; idx += NT) {
    const int f = idx / BB, t = idx - f * BB, b = t / B, a = t - b * B;
    if (cs.nb[f] == NB_BOUNDARY) {
      const TV m = S[mirror_pos<B>(f, a, b)];
      S[ghost_pos<B>(f, a, b)] = cs.bc[f] == BC_OUTFLOW ? -m : m;
    }
  }
  __syncthreads();
}

// Stage planes z0-1 .. z0+KS of a pressure-like field into the (KS+2)(B+2)^2 tile S,
// with the x/y face ring on the KS own planes:
//   val4(cube, cell0, face, v[4]) -> cells cell0..cell0+3 of `cube` (face = -1 for this
//                                    cube, else the face across which it lies);
//   val1(face, n, cell)          -> one cell of same-level neighbour n across face;
// domain faces get the pressure ghost (mirror, or minus the mirror at outflow).
// Ends with the tile complete and the block synchronised.
template <int B, int KS, int NT, class TV, class Val4, class Val1, class ValG>
__device__ __forceinline__ void stage_pressure_slab(TV* __restrict__ S, const CubeSh<TV>& cs,
                                                    const DevGrid& g, int c, int z0,
                                                    const Val4& val4, const Val1& val1,
                                                    const ValG& valg, int lsh = 0) {
  using SL = Slab<B, KS>;
  constexpr int BB = B * B, Q = BB / 4;
  poison_tile(S, SL::N);
  for (int idx = threadIdx.x; idx < (KS + 2) * Q; idx += NT) {
    const int kk = idx / Q, q = idx - kk * Q;
    const int j = (4 * q) / B, i0 = 4 * q - j * B;
    const int k = z0 - 1 + kk;
    TV v[4];
    bool have = true;
    if (k >= 0 && k < B) {
      val4(c, k * BB + 4 * q, -1, v);
    } else {
      const int f = k < 0 ? 4 : 5, n = cs.nb[f];
      if (n >= 0) {
        val4(n, (k < 0 ? B - 1 : 0) * BB + 4 * q, f, v);
      } else if (n < NB_BOUNDARY) {
#pragma unroll
        for (int m = 0; m < 4; ++m)
          v[m] = poisson_ghost_21<B, TV>(g, c, f, i0 + m, j, n, valg, lsh);
      } else {
        have = false;
      }
    }
    if (have) {
      const int o = SL::at(i0, j, kk);
      S[o] = v[0];
      S[o + 1] = v[1];
      S[o + 2] = v[2];
      S[o + 3] = v[3];
    }
  }
#pragma unroll 4
  for (int idx = threadIdx.x; idx < 4 * KS * B; idx += NT) {
    const int f = idx / (KS * B), rem = idx - f * (KS * B), kk = rem / B, t = rem - kk * B;
    const int n = cs.nb[f];
    if (n >= 0) {
      const TV v = val1(f, n, cell_of<B>(f >> 1, (f & 1) ? 0 : B - 1, t, z0 + kk));
      S[f < 2 ? SL::at(f == 0 ? -1 : B, t, kk + 1) : SL::at(t, f == 2 ? -1 : B, kk + 1)] = v;
    } else if (n < NB_BOUNDARY) {
      const TV v = poisson_ghost_21<B, TV>(g, c, f, t, z0 + kk, n, valg, lsh);
      S[f < 2 ? SL::at(f == 0 ? -1 : B, t, kk + 1) : SL::at(t, f == 2 ? -1 : B, kk + 1)] = v;
    }
  }
  __syncthreads();
  // domain faces: the ghost mirrors an own cell staged above (x/y ring and z planes
  // touch disjoint ghosts); a cube without domain faces needs no second pass
  const bool lo = (z0 == 0 && cs.nb[4] == NB_BOUNDARY);
  const bool hi = (z0 + KS == B && cs.nb[5] == NB_BOUNDARY);
  const bool ring = cs.nb[0] == NB_BOUNDARY || cs.nb[1] == NB_BOUNDARY ||
                    cs.nb[2] == NB_BOUNDARY || cs.nb[3] == NB_BOUNDARY;
  if (ring || lo || hi) {
    if (ring)
      for (int idx = threadIdx.x; idx < 4 * KS * B; idx += NT) {
        const int f = idx / (KS * B), rem = idx - f * (KS * B), kk = rem / B, t = rem - kk * B;
        if (cs.nb[f] == NB_BOUNDARY) {
          const int gpos = f < 2 ? SL::at(f == 0 ? -1 : B, t, kk + 1) : SL::at(t, f == 2 ? -1 : B, kk + 1);
          const int mpos = f < 2 ? SL::at(f == 0 ? 0 : B - 1, t, kk + 1)
                                 : SL::at(t, f == 2 ? 0 : B - 1, kk + 1);
          const TV m = S[mpos];
          S[gpos] = cs.bc[f] == BC_OUTFLOW ? -m : m;
        }
      }
    if (lo || hi)
      for (int idx = threadIdx.x; idx < 2 * BB; idx += NT) {
        const int top = idx / BB, t = idx - top * BB, j = t / B, i = t - j * B;
        if (top ? hi : lo) {
          const TV m = S[SL::at(i, j, top ? KS : 1)];
          S[SL::at(i, j, top ? KS + 1 : 0)] = cs.bc[top ? 5 : 4] == BC_OUTFLOW ? -m : m;
        }
      }
    __syncthreads();
  }
}

// Row j of the column that thread slot t (0 .. B*B-1, i = t % B) works on in the column
// marches.  With B = 16 a warp covers two rows; rows w and w + 8 lie 8 (B+2) = 144
// words apart in the tile (16 mod 32 banks), so the two half-warps never share a
// bank, where rows w and w + 1 (18 words apart) would conflict on two banks.
template <int B>
__device__ __forceinline__ int column_row(int t) {
  const int jj = t / B;
  return B == 16 ? (jj >> 1) | ((jj & 1) << 3) : jj;
}

// sum over the six faces of (p_c - p_nb) at tile position o (the 7-point K stencil / h)
template <int B, class TV, int KS = B>
__device__ __forceinline__ TV stencil_sum(const TV* __restrict__ S, int o) {
  using SL = Slab<B, KS>;
  const TV pc = S[o];
  return (pc - S[o - 1]) + (pc - S[o + 1]) + (pc - S[o - SL::P]) + (pc - S[o + SL::P]) +
         (pc - S[o - SL::P * SL::P]) + (pc - S[o + SL::P * SL::P]);
}

// The K stencil sum with 2:1 faces weighted (R7): cell (i, j, k) of the cube (k is the
// cube's plane index), tile position o.
template <int B, class TV, int KS = B>
__device__ __forceinline__ TV stencil_sum_w(const TV* __restrict__ S, int o, const CubeSh<TV>& cs,
                                            int i, int j, int k) {
  using SL = Slab<B, KS>;
  TV acc = stencil_sum<B, TV, KS>(S, o);
  if (cs.has21) {
    const TV pc = S[o];
    if (i == 0) acc += (cs.wt[0] - TV(1)) * (pc - S[o - 1]);
    if (i == B - 1) acc += (cs.wt[1] - TV(1)) * (pc - S[o + 1]);
    if (j == 0) acc += (cs.wt[2] - TV(1)) * (pc - S[o - SL::P]);
    if (j == B - 1) acc += (cs.wt[3] - TV(1)) * (pc - S[o + SL::P]);
    if (k == 0) acc += (cs.wt[4] - TV(1)) * (pc - S[o - SL::P * SL::P]);
    if (k == B - 1) acc += (cs.wt[5] - TV(1)) * (pc - S[o + SL::P * SL::P]);
  }
  return acc;
}

}  // namespace bcm
