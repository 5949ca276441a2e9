// bcm_api.cu -- host runtime and C ABI of the BCM library (see include/bcm.h).
//
// Grid build ("Building Cube Method": cubes kept in linear arrays with corner,
// size and adjacency), workspace layout, and the drivers of the fractional step
// ("Numerical algorithm"): FracTimeStep -> PoissonSolve -> velocity correction.
// The host never touches field data; every arithmetic step runs in the kernels of
// bcm_kernels.cu on the grid's stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdarg.h>
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <string>
#include <array>
#include <map>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/bcm.h"
#include "bcm_internal.cuh"
#include "bcm_kernels.h"

using namespace bcm;

// NVTX range around a phase of the step (no-op unless a profiler is attached): the
// ranges name the paper's sub-steps in a timeline and let a profiler select the
// kernels of one phase.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

static thread_local std::string g_last_error;

static bcm_status fail(bcm_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(BCM_E_CUDA, "%s failed: %s (%d)", #expr, cudaGetErrorString(e_), (int)e_); \
  } while (0)

// --------------------------------------------------------------- workspace

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t u, v, w, us, vs, ws, nx, ny, nz, phi, ub, p, b, bid, near_, r, p0, p1, q, e, w1, s0, s1;
  size_t face, fcube;  // fused PCG face planes and per-cube records (mixed, 16^3 cubes)
  size_t nb, aux, sim, lvl, ijk, w3, nbw3, slot, sp, ss, counter, flags, guard, bar, err;
  size_t total;
  size_t n_slots;
};

struct HostTables {
  std::vector<int> nb, aux, sim, lvl, ijk, w3, nbw3, slot;
  std::vector<SimParams> sp;
  int n_slots = 0;
  int two_level = 0;
};

int face_axis(int f) { return f >> 1; }

// Multigrid hierarchy of a grid of one or two levels (see bcm_mg.cu): per-cube level
// sizes and the cube-aggregate levels as CSR tables (Galerkin sums of the cube graph).
struct MgAgg {
  int n = 0;                          // nodes
  std::vector<int> row, col, cptr, cidx, parent;
  std::vector<double> val, diag;
};
struct MgHost {
  bool ok = false;
  int L = 0;
  std::vector<size_t> n;  // per-cube level cells, l = 0 .. L
  std::vector<MgAgg> agg;
};
struct MgLayout {
  size_t x[kMgMaxL + 1], y[kMgMaxL + 1], r[kMgMaxL + 1], rr;
  size_t ar[kMgMaxM], ax[kMgMaxM], at[kMgMaxM], diag[kMgMaxM], val[kMgMaxM];
  size_t row[kMgMaxM], col[kMgMaxM], cptr[kMgMaxM], cidx[kMgMaxM], parent[kMgMaxM];
};

bcm_status validate(const bcm_grid_desc* d) {
  if (!d) return fail(BCM_E_INVALID, "desc is NULL");
  if (d->n_sims < 1 || d->n_cubes < 1) return fail(BCM_E_INVALID, "empty grid");
  if (d->cells_per_edge != 4 && d->cells_per_edge != 8 && d->cells_per_edge != 16)
    return fail(BCM_E_INVALID, "cells_per_edge must be 4, 8 or 16");
  if (d->max_level < 0 || d->max_level > 1) return fail(BCM_E_INVALID, "max_level must be 0 or 1");
  if (d->precision != BCM_PREC_F64 && d->precision != BCM_PREC_F32_REFINE &&
      d->precision != BCM_PREC_F64_REFINE)
    return fail(BCM_E_INVALID, "unknown precision %d", d->precision);
  if (d->lagged_bf16 != 0 && (d->lagged_bf16 != 1 || d->precision != BCM_PREC_F32_REFINE))
    return fail(BCM_E_INVALID, "lagged_bf16 must be 0, or 1 with BCM_PREC_F32_REFINE");
  if (!d->sim_cube_offset || !d->cube_ijk || !d->cube_level || !d->sim_extent ||
      !d->sim_origin || !d->sim_h0 || !d->sim_bc || !d->sim_bc_vel || !d->sim_nu ||
      !d->sim_dt || !d->sim_uconv)
    return fail(BCM_E_INVALID, "a descriptor array is NULL");
  if (d->sim_cube_offset[0] != 0 || d->sim_cube_offset[d->n_sims] != d->n_cubes)
    return fail(BCM_E_INVALID, "sim_cube_offset must run from 0 to n_cubes");
  for (int s = 0; s < d->n_sims; ++s) {
    if (d->sim_cube_offset[s + 1] <= d->sim_cube_offset[s])
      return fail(BCM_E_INVALID, "sim %d has no cubes", s);
    if (!(d->sim_h0[s] > 0) || !(d->sim_dt[s] > 0) || !(d->sim_nu[s] >= 0))
      return fail(BCM_E_INVALID, "sim %d: h0, dt must be > 0 and nu >= 0", s);
    for (int f = 0; f < 6; ++f) {
      int bc = d->sim_bc[6 * s + f];
      if (bc < BC_WALL || bc > BC_PERIODIC) return fail(BCM_E_INVALID, "sim %d: bad bc", s);
      int opp = d->sim_bc[6 * s + (f ^ 1)];
      if ((bc == BC_PERIODIC) != (opp == BC_PERIODIC))
        return fail(BCM_E_INVALID, "sim %d: periodic faces must come in pairs", s);
    }
  }
  for (int c = 0; c < d->n_cubes; ++c)
    if (d->cube_level[c] < 0 || d->cube_level[c] > d->max_level)
      return fail(BCM_E_INVALID, "cube %d: level out of range", c);
  return BCM_OK;
}

struct Key {
  int s, l, x, y, z;
  bool operator==(const Key& o) const {
    return s == o.s && l == o.l && x == o.x && y == o.y && z == o.z;
  }
};
struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int v : {k.s, k.l, k.x, k.y, k.z}) h = (h ^ (uint32_t)v) * 1099511628211ull;
    return (size_t)h;
  }
};

int wrapi(int x, int n) { return ((x % n) + n) % n; }

// Face adjacency, Jacobi face weights and outflow slots for every cube.
bcm_status build_tables(const bcm_grid_desc* d, HostTables& T) {
  const int n = d->n_cubes, B = d->cells_per_edge, ML = d->max_level;
  std::unordered_map<Key, int, KeyHash> index;
  index.reserve((size_t)n * 2);
  T.sim.resize(n);
  T.lvl.resize(n);
  T.ijk.assign(d->cube_ijk, d->cube_ijk + 3 * (size_t)n);
  for (int s = 0; s < d->n_sims; ++s)
    for (int c = d->sim_cube_offset[s]; c < d->sim_cube_offset[s + 1]; ++c) {
      T.sim[c] = s;
      T.lvl[c] = d->cube_level[c];
      Key k{s, T.lvl[c], T.ijk[3 * c], T.ijk[3 * c + 1], T.ijk[3 * c + 2]};
      if (!index.emplace(k, c).second) return fail(BCM_E_INVALID, "duplicate cube %d", c);
      const int sp = B << (ML - T.lvl[c]);
      for (int e = 0; e < 3; ++e) {
        int x = T.ijk[3 * c + e];
        if (x < 0 || x + sp > d->sim_extent[3 * s + e] || x % sp != 0)
          return fail(BCM_E_INVALID, "cube %d lies outside its domain or off its lattice", c);
      }
    }
  auto find = [&](int s, int l, int x, int y, int z) {
    auto it = index.find(Key{s, l, x, y, z});
    return it == index.end() ? -1 : it->second;
  };
  T.nb.assign(6 * (size_t)n, NB_BOUNDARY);
  T.aux.assign(24 * (size_t)n, -1);
  T.w3.assign(6 * (size_t)n, 3);
  T.slot.assign(6 * (size_t)n, -1);
  int slots = 0;
  for (int c = 0; c < n; ++c) {
    const int s = T.sim[c], l = T.lvl[c];
    const int sp = B << (ML - l);
    const int* ext = d->sim_extent + 3 * s;
    for (int f = 0; f < 6; ++f) {
      const int dd = face_axis(f), side = f & 1, bc = d->sim_bc[6 * s + f];
      int X[3] = {T.ijk[3 * c], T.ijk[3 * c + 1], T.ijk[3 * c + 2]};
      const bool edge = side ? (X[dd] + sp == ext[dd]) : (X[dd] == 0);
      if (edge && bc != BC_PERIODIC) {
        T.nb[6 * c + f] = NB_BOUNDARY;
        T.w3[6 * c + f] = (bc == BC_OUTFLOW) ? 6 : 0;
        if (bc == BC_OUTFLOW) T.slot[6 * c + f] = slots++;
        continue;
      }
      int Y[3] = {X[0], X[1], X[2]};
      Y[dd] = wrapi(X[dd] + (side ? sp : -sp), ext[dd]);
      int m = find(s, l, Y[0], Y[1], Y[2]);
      if (m >= 0) {
        T.nb[6 * c + f] = m;
        continue;
      }
      if (l > 0) {  // coarser neighbour
        int P[3] = {X[0], X[1], X[2]}, Q[3];
        P[dd] = wrapi(X[dd] + (side ? sp : -1), ext[dd]);
        for (int e = 0; e < 3; ++e) Q[e] = P[e] / (2 * sp) * (2 * sp);
        m = find(s, l - 1, Q[0], Q[1], Q[2]);
        if (m >= 0) {
          T.nb[6 * c + f] = NB_COARSE;
          T.aux[(6 * c + f) * 4] = m;
          T.w3[6 * c + f] = 2;
          T.two_level = 1;
          continue;
        }
      }
      if (l < ML) {  // four finer neighbours
        const int fsp = sp / 2;
        bool ok = true;
        for (int qb = 0; qb < 2; ++qb)
          for (int qa = 0; qa < 2; ++qa) {
            int Z[3] = {X[0], X[1], X[2]};
            Z[dd] = wrapi(X[dd] + (side ? sp : -fsp), ext[dd]);
            Z[tan1(dd)] += qa * fsp;
            Z[tan2(dd)] += qb * fsp;
            int mm = find(s, l + 1, Z[0], Z[1], Z[2]);
            T.aux[(6 * c + f) * 4 + qb * 2 + qa] = mm;
            if (mm < 0) ok = false;
          }
        if (ok) {
          T.nb[6 * c + f] = NB_FINE;
          T.w3[6 * c + f] = 4;
          T.two_level = 1;
          continue;
        }
      }
      return fail(BCM_E_INVALID, "cube %d face %d has no neighbour (hole or level jump > 1)", c, f);
    }
  }
  T.n_slots = slots;
  T.nbw3.assign(36 * (size_t)n, 3);
  for (int c = 0; c < n; ++c)
    for (int f = 0; f < 6; ++f) {
      const int m = T.nb[6 * c + f];
      if (m >= 0)
        for (int e = 0; e < 6; ++e) T.nbw3[36 * c + 6 * f + e] = T.w3[6 * m + e];
    }
  // per-sim constants
  T.sp.assign(d->n_sims, SimParams{});
  for (int s = 0; s < d->n_sims; ++s) {
    SimParams& p = T.sp[s];
    memset(&p, 0, sizeof p);
    p.h0 = d->sim_h0[s];
    p.hf = d->sim_h0[s] / double(1 << ML);
    p.nu = d->sim_nu[s];
    p.dt = d->sim_dt[s];
    p.uconv = d->sim_uconv[s];
    p.all_neumann = 1;
    for (int e = 0; e < 3; ++e) {
      p.origin[e] = d->sim_origin[3 * s + e];
      p.extent[e] = d->sim_extent[3 * s + e];
      p.L[e] = p.extent[e] * p.hf;
    }
    for (int f = 0; f < 6; ++f) {
      p.bc[f] = d->sim_bc[6 * s + f];
      if (p.bc[f] == BC_OUTFLOW) p.all_neumann = 0;
      for (int e = 0; e < 3; ++e) p.bcvel[f][e] = d->sim_bc_vel[18 * s + 3 * f + e];
    }
    p.cube_begin = d->sim_cube_offset[s];
    p.cube_end = d->sim_cube_offset[s + 1];
    p.n_cells = (p.cube_end - p.cube_begin) * B * B * B;
    for (int l = 0; l < 2; ++l) {
      const double h = p.h0 / double(1 << l);
      for (int w = 0; w < kW3; ++w) p.invdiag[l][w] = w > 0 ? 3.0 / (h * w) : 0.0;
    }
    for (int l = 0; l < 2; ++l)
      for (int w = 0; w < kW3; ++w) p.invdiag32[l][w] = (float)p.invdiag[l][w];
    p.h032 = (float)p.h0;
  }
  return BCM_OK;
}

// Aggregate levels: cubes of one sim whose cube coordinates shifted right by m agree
// form one node of level m = k + 1; edge weights are the Galerkin sums of the cube
// graph, whose faces carry B^2 h (4^L fine faces of coefficient h) and whose outflow
// faces add 2 B^2 h to the diagonal.
MgHost mg_build(const bcm_grid_desc* d, const HostTables& T) {
  MgHost m;
  const int B = d->cells_per_edge, nc = d->n_cubes, ML = d->max_level;
  while ((1 << m.L) < B) ++m.L;
  for (int l = 0; l <= m.L; ++l) m.n.push_back((size_t)nc * (B >> l) * (B >> l) * (B >> l));
  // a cube's coordinates in cubes of its own level (corner units: finest cells)
  auto cube_coord = [&](int c, int e) {
    return d->cube_ijk[3 * c + e] / (B << (ML - d->cube_level[c]));
  };
  int ext = 1;
  for (int s = 0; s < d->n_sims; ++s) {
    int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-1, -1, -1};
    for (int c = d->sim_cube_offset[s]; c < d->sim_cube_offset[s + 1]; ++c)
      for (int e = 0; e < 3; ++e) {
        const int x = cube_coord(c, e) >> d->cube_level[c];  // level-0 cube units
        lo[e] = lo[e] < x ? lo[e] : x;
        hi[e] = hi[e] > x ? hi[e] : x;
      }
    for (int e = 0; e < 3; ++e) ext = ext > hi[e] - lo[e] + 1 ? ext : hi[e] - lo[e] + 1;
  }
  int M = 1;
  while ((1 << M) < ext) ++M;
  M += ML;  // first the refined cubes join their level-0 parents, one level per step
  if (M > kMgMaxM) return m;
  // level "k = -1": the cube graph.  Key: sim, level, cube coordinates at that level.
  // A face of a cube of level l carries B^2 faces of coefficient h_l; a 2:1 face links
  // a fine cube and its coarse neighbour with B^2 fine faces of coefficient h_f / 1.5
  // (R7), entered once from each side.
  std::vector<std::array<int, 5>> key(nc);
  std::vector<std::map<int, double>> edges(nc);
  std::vector<double> bnd(nc, 0.0);
  for (int c = 0; c < nc; ++c) {
    const int s = T.sim[c], lv = d->cube_level[c];
    const double h = d->sim_h0[s] / double(1 << lv);
    const double a = double(B) * B * h;
    key[c] = {s, lv, cube_coord(c, 0), cube_coord(c, 1), cube_coord(c, 2)};
    for (int f = 0; f < 6; ++f) {
      const int nb = T.nb[6 * c + f];
      if (nb >= 0) {
        if (nb != c) edges[c][nb] += a;
      } else if (nb == NB_BOUNDARY) {
        if (d->sim_bc[6 * s + f] == BC_OUTFLOW) bnd[c] += 2.0 * a;
      } else if (nb == NB_COARSE) {  // this cube is the fine side
        edges[c][T.aux[(6 * c + f) * 4]] += a / 1.5;
      } else {  // NB_FINE: four fine cubes of half the cell size
        for (int q = 0; q < 4; ++q) edges[c][T.aux[(6 * c + f) * 4 + q]] += 0.5 * a / 1.5;
      }
    }
  }
  for (int k = 0; k < M; ++k) {
    MgAgg g;
    std::map<std::array<int, 5>, int> ids;
    const int np = (int)key.size();
    g.parent.resize(np);
    std::vector<std::array<int, 5>> nkey;
    int top_level = 0;
    for (int u = 0; u < np; ++u) top_level = top_level > key[u][1] ? top_level : key[u][1];
    for (int u = 0; u < np; ++u) {
      // refined cubes of the finest level remaining join their parents; once every node
      // is of level 0, nodes join 2x2x2
      std::array<int, 5> kk = key[u];
      if (top_level == 0 || kk[1] == top_level) {
        kk[1] = kk[1] > 0 ? kk[1] - 1 : 0;
        kk[2] >>= 1;
        kk[3] >>= 1;
        kk[4] >>= 1;
      }
      auto it = ids.find(kk);
      int id;
      if (it == ids.end()) {
        id = (int)nkey.size();
        ids.emplace(kk, id);
        nkey.push_back(kk);
      } else {
        id = it->second;
      }
      g.parent[u] = id;
    }
    g.n = (int)nkey.size();
    std::vector<std::map<int, double>> ne(g.n);
    std::vector<double> nbnd(g.n, 0.0);
    std::vector<std::vector<int>> kids(g.n);
    for (int u = 0; u < np; ++u) {
      const int U = g.parent[u];
      kids[U].push_back(u);
      nbnd[U] += bnd[u];
      for (const auto& e : edges[u]) {
        const int V = g.parent[e.first];
        if (V != U) ne[U][V] += e.second;
      }
    }
    g.row.push_back(0);
    g.cptr.push_back(0);
    for (int U = 0; U < g.n; ++U) {
      double dsum = nbnd[U];
      for (const auto& e : ne[U]) {
        g.col.push_back(e.first);
        g.val.push_back(e.second);
        dsum += e.second;
      }
      g.diag.push_back(dsum);
      g.row.push_back((int)g.col.size());
      for (int u : kids[U]) g.cidx.push_back(u);
      g.cptr.push_back((int)g.cidx.size());
    }
    m.agg.push_back(std::move(g));
    key = std::move(nkey);
    edges = std::move(ne);
    bnd = std::move(nbnd);
  }
  m.ok = true;
  return m;
}

// Per-cube constant records of the fused PCG (the same values the other PCG forms
// derive in shared memory from the tables at every launch).
void fused_records(const HostTables& T, int n, FCube* out) {
  for (int c = 0; c < n; ++c) {
    FCube& r = out[c];
    memset(&r, 0, sizeof r);
    const int s = T.sim[c], l = T.lvl[c];
    const SimParams& sp = T.sp[s];
    r.sim = s;
    r.lvl = l;
    r.smask = 0;
    r.has21 = 0;
    for (int f = 0; f < 6; ++f) {
      const int nb = T.nb[6 * c + f];
      r.nb[f] = nb;
      r.w3[f] = T.w3[6 * c + f];
      r.bc[f] = sp.bc[f];
      r.smask |= (r.w3[f] != 3) << f;
      r.has21 |= nb < NB_BOUNDARY;
      r.wt[f] = nb == NB_COARSE ? 2.0f / 3.0f : (nb == NB_FINE ? 4.0f / 3.0f : 1.0f);
      int m = 0;
      for (int e = 0; e < 6; ++e) {
        r.nbw3[f][e] = T.nbw3[36 * c + 6 * f + e];
        m |= (r.nbw3[f][e] != 3) << e;
      }
      r.nbmask[f] = m;
    }
    for (int w = 0; w < kW3; ++w) r.invtab[w] = (float)sp.invdiag[l][w];
    r.h = (float)(sp.h0 / double(1 << l));
  }
}

Layout plan(const bcm_grid_desc* d, int n_slots, const MgHost& mg, MgLayout* ml) {
  Layout L{};
  const size_t n = (size_t)d->n_cubes * d->cells_per_edge * d->cells_per_edge * d->cells_per_edge;
  const size_t S = d->precision == BCM_PREC_F32_REFINE ? 4 : 8;  // state storage
  const size_t V = d->precision == BCM_PREC_F64 ? 8 : 4;         // PCG vector storage
  const size_t nub = (size_t)n_slots * 3 * d->cells_per_edge * d->cells_per_edge;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + (bytes ? bytes : 1));
    return o;
  };
  L.u = take(n * S); L.v = take(n * S); L.w = take(n * S);
  L.us = take(n * S); L.vs = take(n * S); L.ws = take(n * S);
  L.nx = take(n * S); L.ny = take(n * S); L.nz = take(n * S);
  L.phi = take(n * S); L.ub = take(nub * S);
  L.p = take(n * 8); L.b = take(n * 8);
  L.bid = take(n); L.near_ = take(d->n_cubes);
  L.r = take(n * V); L.p0 = take(n * V); L.p1 = take(n * V); L.q = take(n * V);
  L.e = take(d->precision == BCM_PREC_F64 ? 0 : n * 4);  // FP32 inner iterate
  L.w1 = take(n * V); L.s0 = take(n * V); L.s1 = take(n * V);
  // fused PCG: r, q, p on the six face planes of every cube, two parities
  const bool fused_ok = d->precision != BCM_PREC_F64 && d->cells_per_edge == 16;
  L.face = fused_ok ? take((size_t)2 * d->n_cubes * 6 * 3 * 16 * 16 * sizeof(float)) : 0;
  L.fcube = fused_ok ? take(sizeof(FCube) * d->n_cubes) : 0;
  L.nb = take(6 * sizeof(int) * d->n_cubes);
  L.aux = take(24 * sizeof(int) * d->n_cubes);
  L.sim = take(sizeof(int) * d->n_cubes);
  L.lvl = take(sizeof(int) * d->n_cubes);
  L.ijk = take(3 * sizeof(int) * d->n_cubes);
  L.w3 = take(6 * sizeof(int) * d->n_cubes);
  L.nbw3 = take(36 * sizeof(int) * d->n_cubes);
  L.slot = take(6 * sizeof(int) * d->n_cubes);
  L.sp = take(sizeof(SimParams) * d->n_sims);
  L.ss = take(sizeof(SimState) * d->n_sims);
  L.counter = take(sizeof(unsigned int) * kTicketWords);
  L.flags = take(64);
  L.guard = take(64);
  L.bar = take(sizeof(unsigned int) * (kTicketWords + 32));
  L.err = take(64);
  if (mg.ok && ml) {  // multigrid preconditioner
    for (int l = 0; l <= mg.L; ++l) {
      ml->x[l] = take(mg.n[l] * V);
      ml->y[l] = take(mg.n[l] * V);
      ml->r[l] = l ? take(mg.n[l] * V) : 0;
    }
    ml->rr = take((size_t)d->n_cubes * V);
    size_t prev = (size_t)d->n_cubes;
    for (size_t k = 0; k < mg.agg.size(); ++k) {
      const MgAgg& a = mg.agg[k];
      ml->ar[k] = take(a.n * 8);
      ml->ax[k] = take(a.n * 8);
      ml->at[k] = take(a.n * 8);
      ml->diag[k] = take(a.n * 8);
      ml->val[k] = take(a.val.size() * 8);
      ml->row[k] = take((a.n + 1) * sizeof(int));
      ml->col[k] = take(a.col.size() * sizeof(int));
      ml->cptr[k] = take((a.n + 1) * sizeof(int));
      ml->cidx[k] = take(prev * sizeof(int));
      ml->parent[k] = take(prev * sizeof(int));
      prev = (size_t)a.n;
    }
  }
  L.total = off;
  L.n_slots = n_slots;
  return L;
}

}  // namespace

struct KernelTimer {
  bool on = false;
  std::vector<cudaEvent_t> pool;   // pairs (start, end)
  std::vector<int> cls;            // class of each recorded pair
  size_t used = 0;
  double total_ms[BCM_NKERNELS] = {};
  long long launches[BCM_NKERNELS] = {};
};

struct StepGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t capture_stream = nullptr;
  cudaStream_t body_stream[2] = {nullptr, nullptr};  // capture of conditional bodies
  int mg = 0;                  // multigrid PCG: conditional loops in the step
  size_t body_kernels[2] = {0, 0};  // kernel nodes of the inner and the outer loop body
  unsigned int counted[2] = {0, 0};  // body executions already in the launch count
  double rtol = 0.0;
  int max_iter = 0, cycles = 0;
  int slabs_p = 0, single_pass = 0, resident = 0, fused = 0;  // the PCG launch shape captured
  int slabs_m = -1;  // the momentum / right-hand-side slabs captured
  double inner_rtol = 0.0;
  int persistent_slabs = 0;
  int recycle = -1;
  int gen = -1;        // the grid's launch generation the graph was captured at
  size_t kernels = 0;  // kernel nodes in the captured step
};

// The multigrid PCG's iteration (pass A, pass B, V-cycle) as one CUDA graph, captured
// once per set of solver parameters and launch shape and replayed between flag reads.
struct MgIterGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t capture_stream = nullptr;
  SolveParams key{};
  int slabs_a = 0, slabs_b = 0, valid = 0;
  long long kernels = 0;  // kernel nodes per replay
};

struct bcm_grid {
  bcm_grid_desc desc;
  StepGraph sg;
  MgIterGraph mgg;
  int graph_cycles = 0;      // graph steps: defect-correction cycles per solve (0: from rtol)
  double inner_rtol = -1.0;  // mixed: inner FP32 PCG reduction per cycle (< 0: automatic)
  int max_cycles = 30;       // mixed: FP64 residual evaluations per solve
  int check_every = 8;       // host-driven loops: iterations between flag reads
  double barrier_timeout_s = 2.0;  // persistent PCG: longest grid-barrier wait
  int recycle = 1;           // mixed + persistent: reliable updates instead of restarts
  int pcg_form = 0;          // PCG form of the last solve (PCG_*)
  int mg_ok = 0;             // the grid has a multigrid hierarchy
  int gen = 0;               // bumped when the kernels of a step change (geometry,
                             // particles, momentum scheme): captured steps are redone
  KernelTimer timer;
  long long launch_count = 0;
  HostTables T;
  Layout L;
  unsigned char* ws = nullptr;
  cudaStream_t stream = nullptr;
  Ctx ctx;
  int B = 0, f64 = 1, solve64 = 1;  // state FP64; pressure solve FP64 (else FP32 inner)
  size_t n_cells = 0;
  int device = 0;
};

namespace {

// Issue one kernel launch of class k; with timing on, bracket it by two events.
template <class F>
bcm_status run(bcm_grid* g, int k, F&& launch) {
  KernelTimer& t = g->timer;
  if (t.on) {
    if (t.used + 2 > t.pool.size()) {
      for (int q = 0; q < 256; ++q) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreate(&e));
        t.pool.push_back(e);
      }
    }
    CUDA_TRY(cudaEventRecord(t.pool[t.used], g->stream));
  }
  CUDA_TRY(launch());
  g->launch_count += 1;
  if (t.on) {
    CUDA_TRY(cudaEventRecord(t.pool[t.used + 1], g->stream));
    t.cls.push_back(k);
    t.used += 2;
  }
  return BCM_OK;
}

#define RUN(k, expr)                                             \
  do {                                                           \
    bcm_status s_ = run(g, (k), [&]() { return (expr); });       \
    if (s_ != BCM_OK) return s_;                                 \
  } while (0)

// Fold recorded event pairs into per-class totals (synchronises the stream).
bcm_status drain_timer(bcm_grid* g) {
  KernelTimer& t = g->timer;
  if (t.used == 0) return BCM_OK;
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  for (size_t q = 0; q < t.cls.size(); ++q) {
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, t.pool[2 * q], t.pool[2 * q + 1]));
    t.total_ms[t.cls[q]] += ms;
    t.launches[t.cls[q]] += 1;
  }
  t.cls.clear();
  t.used = 0;
  return BCM_OK;
}

}  // namespace

// Read-only views of a grid for other translation units of the library.
namespace bcm {
const Ctx* grid_ctx(const bcm_grid* g) { return &g->ctx; }
int grid_two_level(const bcm_grid* g) { return g->T.two_level; }
int grid_device(const bcm_grid* g) { return g->device; }
cudaStream_t grid_stream(const bcm_grid* g) { return g->stream; }
bcm_status grid_fail(bcm_status st, const char* msg) { return fail(st, "%s", msg); }
}  // namespace bcm

// ------------------------------------------------------------------ ABI

extern "C" const char* bcm_last_error(void) { return g_last_error.c_str(); }

extern "C" size_t bcm_workspace_bytes(const bcm_grid_desc* desc) {
  if (validate(desc) != BCM_OK) return 0;
  HostTables T;
  if (build_tables(desc, T) != BCM_OK) return 0;
  MgLayout ml;
  return plan(desc, T.n_slots, mg_build(desc, T), &ml).total;
}

extern "C" bcm_status bcm_create_grid(const bcm_grid_desc* desc, void* dev_workspace, size_t bytes,
                                      void* cuda_stream, bcm_grid** out) {
  if (!out) return fail(BCM_E_INVALID, "out is NULL");
  *out = nullptr;
  bcm_status st = validate(desc);
  if (st != BCM_OK) return st;
  bcm_grid* g = new bcm_grid();
  g->desc = *desc;
  st = build_tables(desc, g->T);
  if (st != BCM_OK) {
    delete g;
    return st;
  }
  const MgHost mgh = mg_build(desc, g->T);
  MgLayout ml{};
  g->L = plan(desc, g->T.n_slots, mgh, &ml);
  g->mg_ok = mgh.ok ? 1 : 0;
  if (!dev_workspace || bytes < g->L.total) {
    size_t need = g->L.total;
    delete g;
    return fail(BCM_E_INVALID, "workspace too small: need %zu bytes", need);
  }
  if (((uintptr_t)dev_workspace) % kAlign) {
    delete g;
    return fail(BCM_E_INVALID, "workspace must be %zu-byte aligned", kAlign);
  }
  cudaGetDevice(&g->device);
  g->ws = (unsigned char*)dev_workspace;
  g->stream = (cudaStream_t)cuda_stream;
  g->B = desc->cells_per_edge;
  g->f64 = desc->precision != BCM_PREC_F32_REFINE;
  g->solve64 = desc->precision == BCM_PREC_F64;
  g->n_cells = (size_t)desc->n_cubes * g->B * g->B * g->B;
  const Layout& L = g->L;
  unsigned char* W = g->ws;
  cudaStream_t s = g->stream;
  const int n = desc->n_cubes;
  auto fail_free = [&](bcm_status code) {
    delete g;
    return code;
  };
#define UP(off, vec, bytes)                                                              \
  do {                                                                                   \
    cudaError_t e_ = cudaMemcpyAsync(W + (off), (vec), (bytes), cudaMemcpyHostToDevice, s); \
    if (e_ != cudaSuccess)                                                               \
      return fail_free(fail(BCM_E_CUDA, "table upload: %s", cudaGetErrorString(e_)));     \
  } while (0)
  {
    cudaError_t e = cudaMemsetAsync(W, 0, L.total, s);
    if (e != cudaSuccess) return fail_free(fail(BCM_E_CUDA, "memset: %s", cudaGetErrorString(e)));
  }
  UP(L.nb, g->T.nb.data(), sizeof(int) * 6 * n);
  UP(L.aux, g->T.aux.data(), sizeof(int) * 24 * n);
  UP(L.sim, g->T.sim.data(), sizeof(int) * n);
  UP(L.lvl, g->T.lvl.data(), sizeof(int) * n);
  UP(L.ijk, g->T.ijk.data(), sizeof(int) * 3 * n);
  UP(L.w3, g->T.w3.data(), sizeof(int) * 6 * n);
  UP(L.nbw3, g->T.nbw3.data(), sizeof(int) * 36 * n);
  UP(L.slot, g->T.slot.data(), sizeof(int) * 6 * n);
  UP(L.sp, g->T.sp.data(), sizeof(SimParams) * desc->n_sims);
  std::vector<FCube> fcubes;
  if (L.fcube) {
    fcubes.resize(n);
    fused_records(g->T, n, fcubes.data());
    UP(L.fcube, fcubes.data(), sizeof(FCube) * n);
  }
  for (size_t k = 0; mgh.ok && k < mgh.agg.size(); ++k) {
    const MgAgg& a = mgh.agg[k];
    UP(ml.diag[k], a.diag.data(), a.diag.size() * sizeof(double));
    if (!a.val.empty()) UP(ml.val[k], a.val.data(), a.val.size() * sizeof(double));
    UP(ml.row[k], a.row.data(), a.row.size() * sizeof(int));
    if (!a.col.empty()) UP(ml.col[k], a.col.data(), a.col.size() * sizeof(int));
    UP(ml.cptr[k], a.cptr.data(), a.cptr.size() * sizeof(int));
    UP(ml.cidx[k], a.cidx.data(), a.cidx.size() * sizeof(int));
    UP(ml.parent[k], a.parent.data(), a.parent.size() * sizeof(int));
  }
#undef UP
  {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_free(fail(BCM_E_CUDA, "create sync: %s", cudaGetErrorString(e)));
  }
  Ctx& x = g->ctx;
  x.B = g->B;
  x.f64 = g->f64;
  x.solve64 = g->solve64;
  x.slabs_a = 1;
  x.slabs_b = 1;
  x.slabs_p = (g->B == 16 && g->solve64) ? 2 : 1;
  // measured on GB300 at 4.2M cells: the persistent solver is on par in FP32 and
  // slower in FP64 (ALU-bound passes), so FP64 defaults to two launches per iteration
  x.persistent = (!g->solve64 && desc->n_sims <= 256) ? 1 : 0;
  x.single_pass = 0;
  x.resident = 0;
  x.fused = 0;  // the fused single-barrier form: selected by bcm_set_launch(5, ...)
  x.slabs_m = 0;  // the momentum / right-hand-side slab depth: bcm_set_stencil_slabs
  x.lag_bf16 = desc->lagged_bf16;
  x.stream = s;
  DevGrid& G = x.g;
  G.n_cubes = n;
  G.n_sims = desc->n_sims;
  G.max_level = desc->max_level;
  G.two_level = g->T.two_level;
  G.nb = (const int*)(W + L.nb);
  G.aux = (const int*)(W + L.aux);
  G.sim = (const int*)(W + L.sim);
  G.lvl = (const int*)(W + L.lvl);
  G.ijk = (const int*)(W + L.ijk);
  G.w3 = (const int*)(W + L.w3);
  G.nbw3 = (const int*)(W + L.nbw3);
  G.slot = (const int*)(W + L.slot);
  G.near = (const unsigned char*)(W + L.near_);
  G.sp = (const SimParams*)(W + L.sp);
  G.ss = (SimState*)(W + L.ss);
  G.counter = (unsigned int*)(W + L.counter);
  G.flags = (int*)(W + L.flags);
  G.check = (int*)(W + L.err) + 8;  // a word of its own in the error block
  Fields& F = x.f;
  F.u = W + L.u; F.v = W + L.v; F.w = W + L.w;
  F.us = W + L.us; F.vs = W + L.vs; F.ws = W + L.ws;
  F.nx = W + L.nx; F.ny = W + L.ny; F.nz = W + L.nz;
  F.phi = W + L.phi; F.ub = W + L.ub;
  F.p = (double*)(W + L.p); F.b = (double*)(W + L.b);
  F.bid = W + L.bid; F.near = W + L.near_;
  F.r = W + L.r; F.p0 = W + L.p0; F.p1 = W + L.p1; F.q = W + L.q;
  F.e = g->solve64 ? nullptr : (float*)(W + L.e);
  F.w1 = W + L.w1; F.s0 = W + L.s0; F.s1 = W + L.s1;
  F.face = L.face ? (float*)(W + L.face) : nullptr;
  F.fcube = L.fcube ? (const FCube*)(W + L.fcube) : nullptr;
  F.guard = (unsigned int*)(W + L.guard);
  F.bar = (unsigned int*)(W + L.bar);
  F.err = (int*)(W + L.err);
  x.use_mg = 0;
  x.mg = MgDev{};
  x.part = PartDev{};
  x.scheme = 0;
  x.cn_rtol = g->f64 ? 1e-10 : 2e-8;
  x.cn_max = 50;
  if (mgh.ok) {
    MgDev& D = x.mg;
    D.L = mgh.L;
    D.M = (int)mgh.agg.size();
    for (int l = 0; l <= mgh.L; ++l) {
      D.x[l] = W + ml.x[l];
      D.y[l] = W + ml.y[l];
      D.r[l] = l ? (void*)(W + ml.r[l]) : F.r;
    }
    D.rr = W + ml.rr;
    for (int k = 0; k < D.M; ++k) {
      D.n[k] = mgh.agg[k].n;
      D.nnz[k] = (int)mgh.agg[k].col.size();
      D.ar[k] = (double*)(W + ml.ar[k]);
      D.ax[k] = (double*)(W + ml.ax[k]);
      D.at[k] = (double*)(W + ml.at[k]);
      D.diag[k] = (double*)(W + ml.diag[k]);
      D.val[k] = (double*)(W + ml.val[k]);
      D.row[k] = (int*)(W + ml.row[k]);
      D.col[k] = (int*)(W + ml.col[k]);
      D.cptr[k] = (int*)(W + ml.cptr[k]);
      D.cidx[k] = (int*)(W + ml.cidx[k]);
      D.parent[k] = (int*)(W + ml.parent[k]);
    }
  }
  *out = g;
  return BCM_OK;
}

extern "C" bcm_status bcm_destroy_grid(bcm_grid* g) {
  if (g) {
    for (cudaEvent_t e : g->timer.pool) cudaEventDestroy(e);
    if (g->sg.exec) cudaGraphExecDestroy(g->sg.exec);
    if (g->sg.graph) cudaGraphDestroy(g->sg.graph);
    if (g->sg.capture_stream) cudaStreamDestroy(g->sg.capture_stream);
    for (cudaStream_t bs : g->sg.body_stream)
      if (bs) cudaStreamDestroy(bs);
    if (g->mgg.exec) cudaGraphExecDestroy(g->mgg.exec);
    if (g->mgg.graph) cudaGraphDestroy(g->mgg.graph);
    if (g->mgg.capture_stream) cudaStreamDestroy(g->mgg.capture_stream);
  }
  delete g;
  return BCM_OK;
}

extern "C" bcm_status bcm_field(bcm_grid* g, int field, void** dev_ptr, size_t* count,
                                int32_t* elem_bytes) {
  if (!g || !dev_ptr) return fail(BCM_E_INVALID, "NULL argument");
  const Layout& L = g->L;
  const int S = g->f64 ? 8 : 4;
  size_t off = 0, cnt = g->n_cells;
  int eb = S;
  switch (field) {
    case BCM_U: off = L.u; break;
    case BCM_V: off = L.v; break;
    case BCM_W: off = L.w; break;
    case BCM_P: off = L.p; eb = 8; break;
    case BCM_PHI: off = L.phi; break;
    case BCM_NX: off = L.nx; eb = g->ctx.lag_bf16 ? 2 : S; break;
    case BCM_NY: off = L.ny; eb = g->ctx.lag_bf16 ? 2 : S; break;
    case BCM_NZ: off = L.nz; eb = g->ctx.lag_bf16 ? 2 : S; break;
    case BCM_USTAR: off = L.us; break;
    case BCM_VSTAR: off = L.vs; break;
    case BCM_WSTAR: off = L.ws; break;
    case BCM_RHS: off = L.b; eb = 8; break;
    case BCM_UB: off = L.ub; cnt = (size_t)L.n_slots * 3 * g->B * g->B; break;
    default: return fail(BCM_E_INVALID, "unknown field %d", field);
  }
  *dev_ptr = g->ws + off;
  if (count) *count = cnt;
  if (elem_bytes) *elem_bytes = eb;
  return BCM_OK;
}

extern "C" bcm_status bcm_set_geometry(bcm_grid* g, int sim, const bcm_body* bodies, int n_bodies,
                                       const double* inflow_modes) {
  if (!g || sim < 0 || sim >= g->desc.n_sims) return fail(BCM_E_INVALID, "bad grid or sim");
  g->gen += 1;
  if (n_bodies < 0 || n_bodies > kMaxBodies)
    return fail(BCM_E_BOUNDS, "n_bodies must be in [0, %d]", kMaxBodies);
  if (n_bodies > 0 && !bodies) return fail(BCM_E_INVALID, "bodies is NULL");
  SimParams& p = g->T.sp[sim];
  p.n_bodies = n_bodies;
  p.moving = 0;
  for (int b = 0; b < kMaxBodies; ++b) memset(&p.bodies[b], 0, sizeof(bcm_body));
  for (int b = 0; b < n_bodies; ++b) {
    const bcm_body& bd = bodies[b];
    if (bd.kind != BCM_BODY_SPHERE && bd.kind != BCM_BODY_ELLIPSOID)
      return fail(BCM_E_INVALID, "body %d: unknown kind", b);
    for (int e = 0; e < 3; ++e)
      if (!(bd.axes[e] > 0) && !(bd.kind == BCM_BODY_SPHERE && e > 0))
        return fail(BCM_E_INVALID, "body %d: axes must be > 0", b);
    p.bodies[b] = bd;
    for (int e = 0; e < 3; ++e)
      if (bd.vel[e] != 0.0 || bd.omega[e] != 0.0) p.moving = 1;
  }
  p.has_modes = 0;
  for (int m = 0; m < kModes; ++m) {
    p.modes[m] = inflow_modes ? inflow_modes[m] : 0.0;
    if (p.modes[m] != 0.0) p.has_modes = 1;
  }
  CUDA_TRY(cudaMemcpyAsync(g->ws + g->L.sp + sizeof(SimParams) * sim, &p, sizeof(SimParams),
                           cudaMemcpyHostToDevice, g->stream));
  // the host copy must stay valid until the copy has run
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  RUN(BCM_K_SOLID_FRACTION, launch_solid_fraction(g->ctx, sim));
  return BCM_OK;
}

extern "C" bcm_status bcm_set_step(bcm_grid* g, int step) {
  if (!g || step < 0) return fail(BCM_E_INVALID, "bad grid or step");
  for (int s = 0; s < g->desc.n_sims; ++s)
    CUDA_TRY(cudaMemcpyAsync(g->ws + g->L.ss + sizeof(SimState) * s + offsetof(SimState, step),
                             &step, sizeof(int), cudaMemcpyHostToDevice, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return BCM_OK;
}

extern "C" bcm_status bcm_reset_time(bcm_grid* g) {
  if (!g) return fail(BCM_E_INVALID, "grid is NULL");
  std::vector<SimState> zero(g->desc.n_sims);
  memset(zero.data(), 0, sizeof(SimState) * zero.size());
  CUDA_TRY(cudaMemcpyAsync(g->ws + g->L.ss, zero.data(), sizeof(SimState) * zero.size(),
                           cudaMemcpyHostToDevice, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return BCM_OK;
}

extern "C" bcm_status bcm_drag_mean(bcm_grid* g, int reset, double* out) {
  if (!g || !out) return fail(BCM_E_INVALID, "NULL argument");
  const int ns = g->desc.n_sims;
  std::vector<SimState> st(ns);
  CUDA_TRY(cudaMemcpyAsync(st.data(), g->ws + g->L.ss, sizeof(SimState) * ns,
                           cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  for (int q = 0; q < ns; ++q)
    for (int e = 0; e < 3; ++e)
      out[3 * q + e] = st[q].drag_n ? st[q].drag_sum[e] / st[q].drag_n : 0.0;
  if (reset) {
    const size_t a = offsetof(SimState, drag_sum), b = offsetof(SimState, drag_n) + sizeof(int);
    for (int q = 0; q < ns; ++q)
      CUDA_TRY(cudaMemsetAsync(g->ws + g->L.ss + sizeof(SimState) * q + a, 0, b - a, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
  }
  return BCM_OK;
}

// ----------------------------------------------------------- solve drivers

namespace {


bcm_status read_flags(bcm_grid* g, int flags[2]) {
  CUDA_TRY(cudaMemcpyAsync(flags, g->ws + g->L.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                           g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return BCM_OK;
}

// Jacobi-PCG on K p = -V (b - mean), warm start p (Saad Alg. 9.1); FP64 vectors, or
// FP32 inner PCG inside FP64 defect correction (mixed).  Persistent mode runs each
// PCG solve as one cooperative launch; the two-launch mode reads the device
// convergence flags every check_every iterations.  Finished sims skip their cubes.
bcm_status read_err(bcm_grid* g) {
  int words[9] = {0};  // [0] barrier timeout, [8] failed index check (checked build)
  CUDA_TRY(cudaMemcpyAsync(words, g->ws + g->L.err, sizeof words, cudaMemcpyDeviceToHost,
                           g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  const int err = words[0];
  if (words[8]) {
    CUDA_TRY(cudaMemsetAsync(g->ws + g->L.err + 8 * sizeof(int), 0, sizeof(int), g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    return fail(BCM_E_BOUNDS, "index check %d failed in a kernel (checked build)", words[8]);
  }
  if (err) {
    // a timed-out solve leaves barrier and ticket counters mid-count: start them afresh
    CUDA_TRY(cudaMemsetAsync(g->ws + g->L.err, 0, sizeof(int), g->stream));
    CUDA_TRY(cudaMemsetAsync(g->ws + g->L.bar, 0, sizeof(unsigned int) * (kTicketWords + 32),
                             g->stream));
    CUDA_TRY(cudaMemsetAsync(g->ws + g->L.counter, 0, sizeof(unsigned int) * kTicketWords,
                             g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    return fail(BCM_E_TIMEOUT, "a grid barrier of the persistent PCG timed out");
  }
  return BCM_OK;
}

// Inner FP32 reduction per defect-correction cycle.  Measured on the 4.2M-cell sphere
// flow: restarting the inner CG every cycle works best at 1e-5 (3 cycles, ~1500
// iterations per step); keeping its search direction (reliable updates) needs the FP64
// residual to replace the FP32 one often, every 0.1 reduction (~10 cycles, ~1200
// iterations, 13 % less time per step); at 1e-5 the kept direction loses conjugacy.
double effective_inner_rtol(const bcm_grid* g, bool recycle) {
  if (g->inner_rtol > 0) return g->inner_rtol;
  // measured on the 4.2M-cell sphere flow with the multigrid PCG: 1e-4 per cycle takes
  // 85 inner iterations per step in 3 cycles (1e-5: 88, 1e-3: 108, 1e-6: 97)
  if (g->ctx.use_mg) return 1e-4;
  return recycle ? 0.1 : 1e-5;
}

bcm_status mg_iteration_graph(bcm_grid* g, const SolveParams& prm, cudaGraphExec_t* out) {
  MgIterGraph& m = g->mgg;
  if (m.valid && memcmp(&m.key, &prm, sizeof prm) == 0 && m.slabs_a == g->ctx.slabs_a &&
      m.slabs_b == g->ctx.slabs_b) {
    *out = m.exec;
    return BCM_OK;
  }
  if (m.exec) CUDA_TRY(cudaGraphExecDestroy(m.exec));
  if (m.graph) CUDA_TRY(cudaGraphDestroy(m.graph));
  m.exec = nullptr;
  m.graph = nullptr;
  m.valid = 0;
  if (!m.capture_stream) CUDA_TRY(cudaStreamCreateWithFlags(&m.capture_stream, cudaStreamNonBlocking));
  Ctx x = g->ctx;
  x.stream = m.capture_stream;
  CUDA_TRY(cudaStreamBeginCapture(m.capture_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = launch_cg_a(x, prm);
  if (e == cudaSuccess) e = launch_mg_vcycle(x, prm, 1);  // pass B inside
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(m.capture_stream, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(BCM_E_CUDA, "multigrid iteration capture: %s",
                cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  m.graph = graph;
  size_t nn = 0;
  CUDA_TRY(cudaGraphGetNodes(graph, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) CUDA_TRY(cudaGraphGetNodes(graph, nodes.data(), &nn));
  m.kernels = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType ty;
    CUDA_TRY(cudaGraphNodeGetType(nd, &ty));
    m.kernels += ty == cudaGraphNodeTypeKernel;
  }
  CUDA_TRY(cudaGraphInstantiate(&m.exec, graph, 0));
  m.key = prm;
  m.slabs_a = g->ctx.slabs_a;
  m.slabs_b = g->ctx.slabs_b;
  m.valid = 1;
  *out = m.exec;
  return BCM_OK;
}

bcm_status solve(bcm_grid* g, double rtol, int max_iter) {
  Ctx& x = g->ctx;
  const bool mg = x.use_mg != 0;  // multigrid-preconditioned CG: two launches + V-cycle
  SolveParams prm{};
  prm.rtol = rtol;
  prm.mg = mg ? 1 : 0;
  prm.recycle = (g->recycle && x.persistent && !mg) ? 1 : 0;
  prm.inner_rtol = effective_inner_rtol(g, prm.recycle != 0);
  prm.max_iter = max_iter;
  prm.inner_max_iter = max_iter;
  prm.max_cycles = g->max_cycles;
  prm.mixed = g->solve64 ? 0 : 1;
  prm.guard = x.f.guard;
  prm.guard_limit = 0;
  prm.barrier_timeout_ns = (unsigned long long)(g->barrier_timeout_s * 1e9);
  RUN(BCM_K_MISC, launch_solve_begin(x));
  RUN(BCM_K_RESIDUAL, launch_residual(x, prm));
  if (mg) RUN(BCM_K_MG, launch_mg_vcycle(x, prm, 0));
  g->pcg_form = mg ? PCG_MULTIGRID : PCG_TWO_LAUNCH;  // persistent launches set theirs
  int flags[2] = {0, 0};
  bcm_status st;
  // the multigrid iteration converges in a few iterations: read the flags more often
  const int every = mg ? (g->check_every < 2 ? g->check_every : 2) : g->check_every;
  // with kernel timing off the multigrid iteration replays one captured graph
  const bool mg_graph = mg && !g->timer.on;
  cudaGraphExec_t mg_exec = nullptr;
  if (mg_graph && (st = mg_iteration_graph(g, prm, &mg_exec)) != BCM_OK) return st;
  if (x.persistent && !mg) {
    if (g->solve64) {
      RUN(BCM_K_PCG, launch_pcg(x, prm, &g->pcg_form));
      return read_err(g);
    }
    // defect correction: cycles are issued in batches; a finished sim makes every
    // kernel of a later cycle return at once, so the host reads the flags rarely.  The
    // streaming form adds its correction to the FP64 iterate itself.
    SolveParams pin = prm;
    pin.x64_add = x.f.p;
    int cycles = 0, batch = 2;
    while (cycles < g->max_cycles) {
      for (int b = 0; b < batch && cycles < g->max_cycles; ++b, ++cycles) {
        RUN(BCM_K_PCG, launch_pcg(x, pin, &g->pcg_form));
        if (g->pcg_form != PCG_STREAMING) RUN(BCM_K_ADD_CORRECTION, launch_add_correction(x));
        RUN(BCM_K_RESIDUAL, launch_residual(x, prm));
      }
      if ((st = read_flags(g, flags)) != BCM_OK) return st;
      if ((st = read_err(g)) != BCM_OK) return st;
      if (flags[1]) break;
      batch = 1;
    }
    return BCM_OK;
  }
  if ((st = read_flags(g, flags)) != BCM_OK) return st;
  if (g->solve64) {
    int it = 0;
    while (!flags[0] && it < max_iter) {
      for (int m = 0; m < every && it < max_iter; ++m, ++it)
      {
        if (mg_graph) {  // pass A and the V-cycle (with pass B) as one graph
          CUDA_TRY(cudaGraphLaunch(mg_exec, g->stream));
          g->launch_count += g->mgg.kernels;
          continue;
        }
        RUN(BCM_K_CG_A, launch_cg_a(x, prm));
        if (mg)
          RUN(BCM_K_MG, launch_mg_vcycle(x, prm, 1));  // pass B inside
        else
          RUN(BCM_K_CG_B, launch_cg_b(x, prm));
      }
      if ((st = read_flags(g, flags)) != BCM_OK) return st;
    }
    return BCM_OK;
  }
  int cycles = 0;
  while (!flags[1] && cycles <= g->max_cycles) {
    int it = 0;
    while (!flags[0] && it < max_iter) {
      for (int m = 0; m < every && it < max_iter; ++m, ++it)
      {
        if (mg_graph) {  // pass A and the V-cycle (with pass B) as one graph
          CUDA_TRY(cudaGraphLaunch(mg_exec, g->stream));
          g->launch_count += g->mgg.kernels;
          continue;
        }
        RUN(BCM_K_CG_A, launch_cg_a(x, prm));
        if (mg)
          RUN(BCM_K_MG, launch_mg_vcycle(x, prm, 1));  // pass B inside
        else
          RUN(BCM_K_CG_B, launch_cg_b(x, prm));
      }
      if ((st = read_flags(g, flags)) != BCM_OK) return st;
    }
    RUN(BCM_K_ADD_CORRECTION, launch_add_correction(x));
    RUN(BCM_K_RESIDUAL, launch_residual(x, prm));
    if (mg) RUN(BCM_K_MG, launch_mg_vcycle(x, prm, 0));
    if ((st = read_flags(g, flags)) != BCM_OK) return st;
    ++cycles;
  }
  return BCM_OK;
}

// Launches inside the conditional loops of captured multigrid steps: the kernel nodes
// of each loop body times the body executions the device counted since the last call.
bcm_status graph_body_launches(bcm_grid* g) {
  StepGraph& sg = g->sg;
  if (!sg.body_kernels[0] && !sg.body_kernels[1]) return BCM_OK;
  unsigned int n[2] = {0u, 0u};
  CUDA_TRY(cudaMemcpyAsync(n, g->ctx.f.guard + 4, sizeof n, cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  for (int q = 0; q < 2; ++q) {
    g->launch_count += (long long)sg.body_kernels[q] * (long long)(n[q] - sg.counted[q]);
    sg.counted[q] = n[q];
  }
  return BCM_OK;
}

bcm_status collect(bcm_grid* g, bcm_stats* out) {
  bcm_status est = read_err(g);
  if (est != BCM_OK) return est;
  if ((est = graph_body_launches(g)) != BCM_OK) return est;
  if (g->ctx.part.n > 0) {
    int perr = 0;
    CUDA_TRY(cudaMemcpyAsync(&perr, g->ctx.part.err, sizeof(int), cudaMemcpyDeviceToHost,
                             g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (perr) return fail(BCM_E_BOUNDS, "a Lagrangian particle lies outside every cube");
  }
  std::vector<SimState> ss(g->desc.n_sims);
  CUDA_TRY(cudaMemcpyAsync(ss.data(), g->ws + g->L.ss, sizeof(SimState) * ss.size(),
                           cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  bcm_status st = BCM_OK;
  for (size_t s = 0; s < ss.size(); ++s) {
    const SimState& t = ss[s];
    bcm_stats& o = out[s];
    o.cg_iters = t.total_iters;
    o.refine_cycles = g->solve64 ? 0 : t.cycles;
    o.steps = t.step;
    o.converged = t.converged;
    o.rel_resid = t.bb > 0 ? sqrt(t.rr64 / t.bb) : 0.0;
    o.div_rel = t.div_den > 0 ? sqrt(t.div_num / t.div_den) : 0.0;
    for (int e = 0; e < 3; ++e) o.drag[e] = t.drag[e];
    double um;
    memcpy(&um, &t.umax_bits, sizeof um);
    o.umax = um;
    o.pcg_form = g->pcg_form;
    o.cn_iters = g->ctx.scheme ? t.cn_iter : 0;
    if (t.nonfinite) st = BCM_E_NONFINITE;
    else if (!t.converged && st == BCM_OK) st = BCM_E_NOT_CONVERGED;
  }
  if (st == BCM_E_NONFINITE) return fail(st, "non-finite residual");
  if (st == BCM_E_NOT_CONVERGED) return fail(st, "pressure solve did not reach rtol");
  return st;
}

}  // namespace

namespace {
// The momentum sub-step: Adams-Bashforth + central in one launch, or QUICK +
// Crank-Nicolson: explicit half, iterations read back every four launches, forcing.
bcm_status momentum_substep(bcm_grid* g) {
  Ctx& x = g->ctx;
  if (x.scheme == 0) {
    RUN(BCM_K_MOMENTUM, launch_momentum(x));
    return BCM_OK;
  }
  RUN(BCM_K_MOMENTUM, launch_cn_explicit(x));
  int it = 0;
  while (it < x.cn_max) {
    for (int m = 0; m < 4 && it < x.cn_max; ++m, ++it) RUN(BCM_K_MOMENTUM, launch_cn_iter(x));
    int done = 0;
    CUDA_TRY(cudaMemcpyAsync(&done, g->ws + g->L.flags + 2 * sizeof(int), sizeof(int),
                             cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (done) break;
  }
  RUN(BCM_K_MOMENTUM, launch_cn_finish(x));
  return BCM_OK;
}
}  // namespace

extern "C" bcm_status bcm_step(bcm_grid* g, int n_steps, double rtol, int max_iter,
                               bcm_stats* stats) {
  if (!g) return fail(BCM_E_INVALID, "grid is NULL");
  if (n_steps < 0 || !(rtol > 0) || max_iter < 1)
    return fail(BCM_E_INVALID, "need n_steps >= 0, rtol > 0, max_iter >= 1");
  Ctx& x = g->ctx;
  bool moving = false;
  for (const auto& p : g->T.sp) moving |= (p.n_bodies > 0 && p.moving);
  bcm_status last = BCM_OK;
  const bool particles = x.part.n > 0;
  for (int n = 0; n < n_steps; ++n) {
    NvtxRange step_range("bcm_step");
    if (moving && !particles) RUN(BCM_K_SOLID_FRACTION, launch_solid_fraction(x, -2));
    {
      NvtxRange r("momentum_ib");
      bcm_status sm = momentum_substep(g);
      if (sm != BCM_OK) return sm;
      if (particles) {  // forcing by the Lagrangian particles: force, then spreading
        RUN(BCM_K_IB, launch_ib_force(x));
        g->launch_count += 1;
      }
    }
    {
      NvtxRange r("pressure_poisson");
      RUN(BCM_K_RHS, launch_rhs(x));
      bcm_status st = solve(g, rtol, max_iter);
      if (st != BCM_OK) return st;
    }
    {
      NvtxRange r("projection");
      RUN(BCM_K_CORRECT, launch_correct(x));
      RUN(BCM_K_MISC, launch_step_end(x));
    }
    if (particles && moving) {  // move, then rebuild the per-cube sets
      RUN(BCM_K_IB, launch_ib_move(x));
      g->launch_count += 3;
    }
  }
  if (stats) last = collect(g, stats);
  return last;
}

// Kernel nodes of a graph (its own nodes; a conditional node's body is not counted).
cudaError_t count_kernels(cudaGraph_t graph, size_t* out) {
  size_t nn = 0;
  cudaError_t e = cudaGraphGetNodes(graph, nullptr, &nn);
  if (e != cudaSuccess) return e;
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn && (e = cudaGraphGetNodes(graph, nodes.data(), &nn)) != cudaSuccess) return e;
  *out = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    if ((e = cudaGraphNodeGetType(nd, &t)) != cudaSuccess) return e;
    if (t == cudaGraphNodeTypeKernel) ++*out;
  }
  return cudaSuccess;
}

// A condition handle on the graph stream s is capturing into (value 1 at every launch
// of the graph).
cudaError_t capture_handle(cudaStream_t s, cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus st;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &graph, nullptr, nullptr, nullptr);
  if (e != cudaSuccess) return e;
  if (st != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  return cudaGraphConditionalHandleCreate(h, graph, 1u, cudaGraphCondAssignDefault);
}

// Appends a while node of handle h after the work captured on s so far and begins the
// capture of its body on stream bs (ended by the caller).
cudaError_t capture_while(cudaStream_t s, cudaGraphConditionalHandle h, cudaStream_t bs) {
  cudaStreamCaptureStatus st;
  cudaGraph_t graph = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &graph, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, graph, deps, nullptr, nd, &p)) != cudaSuccess) return e;
  if ((e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                               cudaStreamSetCaptureDependencies)) != cudaSuccess)
    return e;
  return cudaStreamBeginCaptureToGraph(bs, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal);
}

// The multigrid PCG of a captured step, with the loops the eager solve runs on the host
// as conditional while nodes.  Inner loop (one PCG iteration: pass A, then the V-cycle
// with pass B inside), run while the V-cycle's decisions leave a sim running or until
// the guard of max_iter x (max_cycles + 1) body executions; mixed mode wraps it in the
// defect-correction loop (V-cycle z = M^-1 r of the new residual, the inner loop, x +=
// e, the FP64 residual), run while the residual leaves a sim correcting.
bcm_status capture_mg_solve(bcm_grid* g, const Ctx& x0, SolveParams prm) {
  StepGraph& sg = g->sg;
  for (cudaStream_t& bs : sg.body_stream)
    if (!bs) CUDA_TRY(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
  prm.mg = 1;
  prm.recycle = 0;
  prm.max_cycles = g->max_cycles;  // the loop ends when the residual says so
  prm.body_count = x0.f.guard + 4;
  prm.guard_limit = prm.max_iter * (prm.max_cycles + 1) + 1;
  CUDA_TRY(cudaMemsetAsync(x0.f.guard, 0, sizeof(unsigned int), x0.stream));  // per step
  Ctx xi = x0;
  auto inner_body = [&](cudaStream_t outer, const SolveParams& pin) -> bcm_status {
    cudaGraphConditionalHandle hin = (cudaGraphConditionalHandle)pin.cond_inner;
    xi.stream = sg.body_stream[1];
    CUDA_TRY(capture_while(outer, hin, xi.stream));
    cudaError_t e = launch_cg_a(xi, pin);
    if (e == cudaSuccess) e = launch_mg_vcycle(xi, pin, 1);  // pass B inside
    cudaGraph_t body = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(xi.stream, &body);
    CUDA_TRY(e);
    CUDA_TRY(e2);
    CUDA_TRY(count_kernels(body, &sg.body_kernels[0]));
    return BCM_OK;
  };
  SolveParams pres = prm;  // the residual kernel sets no loop condition of the inner loop
  pres.cond_inner = 0;
  if (g->solve64) {
    cudaGraphConditionalHandle hin;
    CUDA_TRY(capture_handle(x0.stream, &hin));
    SolveParams pin = prm;
    pin.cond_inner = (unsigned long long)hin;
    CUDA_TRY(launch_residual(x0, pres));
    CUDA_TRY(launch_mg_vcycle(x0, pin, 0));
    sg.body_kernels[1] = 0;
    return inner_body(x0.stream, pin);
  }
  cudaGraphConditionalHandle hout;
  CUDA_TRY(capture_handle(x0.stream, &hout));
  pres.cond_outer = (unsigned long long)hout;
  CUDA_TRY(launch_residual(x0, pres));
  Ctx xo = x0;
  xo.stream = sg.body_stream[0];
  CUDA_TRY(capture_while(x0.stream, hout, xo.stream));
  bcm_status st = BCM_OK;
  cudaGraphConditionalHandle hin;
  cudaError_t e = capture_handle(xo.stream, &hin);
  SolveParams pin = prm;
  pin.cond_inner = (unsigned long long)hin;
  pin.cond_outer = 0;
  if (e == cudaSuccess) e = launch_mg_vcycle(xo, pin, 0);
  if (e == cudaSuccess) st = inner_body(xo.stream, pin);
  if (e == cudaSuccess && st == BCM_OK) e = launch_add_correction(xo);
  if (e == cudaSuccess && st == BCM_OK) e = launch_residual(xo, pres);
  cudaGraph_t body = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(xo.stream, &body);
  if (st != BCM_OK) return st;
  CUDA_TRY(e);
  CUDA_TRY(e2);
  CUDA_TRY(count_kernels(body, &sg.body_kernels[1]));
  return BCM_OK;
}

// One step as a CUDA graph: no host synchronisation inside.  The PCG is the
// persistent kernel (one launch per solve); mixed mode issues a fixed budget of
// defect-correction cycles whose kernels return at once for sims already converged.
namespace {
bcm_status issue_graph_step(bcm_grid* g, cudaStream_t s, double rtol, int max_iter, int cycles) {
  Ctx x = g->ctx;
  x.stream = s;
  bool moving = false;
  for (const auto& p : g->T.sp) moving |= (p.n_bodies > 0 && p.moving);
  SolveParams prm{};
  prm.rtol = rtol;
  prm.recycle = g->recycle;
  prm.inner_rtol = effective_inner_rtol(g, prm.recycle != 0);
  prm.max_iter = max_iter;
  prm.inner_max_iter = max_iter;
  prm.max_cycles = cycles;
  prm.mixed = g->solve64 ? 0 : 1;
  prm.guard = x.f.guard;
  prm.barrier_timeout_ns = (unsigned long long)(g->barrier_timeout_s * 1e9);
  const bool particles = x.part.n > 0;
  if (moving && !particles) CUDA_TRY(launch_solid_fraction(x, -2));
  if (x.scheme == 0) {
    CUDA_TRY(launch_momentum(x));
  } else {  // QUICK + Crank-Nicolson: the full iteration budget (converged sims return)
    CUDA_TRY(launch_cn_explicit(x));
    for (int it = 0; it < x.cn_max; ++it) CUDA_TRY(launch_cn_iter(x));
    CUDA_TRY(launch_cn_finish(x));
  }
  if (particles) CUDA_TRY(launch_ib_force(x));
  CUDA_TRY(launch_rhs(x));
  CUDA_TRY(launch_solve_begin(x));
  if (x.use_mg) {
    const bcm_status st = capture_mg_solve(g, x, prm);
    if (st != BCM_OK) return st;
    g->pcg_form = PCG_MULTIGRID;
  } else if (g->solve64) {
    CUDA_TRY(launch_residual(x, prm));
    CUDA_TRY(launch_pcg(x, prm, &g->pcg_form));
  } else {
    CUDA_TRY(launch_residual(x, prm));
    SolveParams pin = prm;  // the streaming form adds its correction itself
    pin.x64_add = x.f.p;
    for (int c = 0; c < cycles; ++c) {
      CUDA_TRY(launch_pcg(x, pin, &g->pcg_form));
      if (g->pcg_form != PCG_STREAMING) CUDA_TRY(launch_add_correction(x));
      CUDA_TRY(launch_residual(x, prm));
    }
  }
  CUDA_TRY(launch_correct(x));
  CUDA_TRY(launch_step_end(x));
  if (particles && moving) CUDA_TRY(launch_ib_move(x));
  return BCM_OK;
}
}  // namespace

extern "C" bcm_status bcm_step_graph(bcm_grid* g, int n_steps, double rtol, int max_iter,
                                     bcm_stats* stats) {
  if (!g) return fail(BCM_E_INVALID, "grid is NULL");
  if (n_steps < 0 || !(rtol > 0) || max_iter < 1)
    return fail(BCM_E_INVALID, "need n_steps >= 0, rtol > 0, max_iter >= 1");
  if (g->desc.n_sims > 256)
    return fail(BCM_E_BOUNDS, "graph steps use the persistent PCG: at most 256 sims per grid");
  StepGraph& sg = g->sg;
  int cycles = 0;
  if (!g->solve64) {  // enough cycles for rtol at the inner reduction per cycle, plus margin
    const double eta = effective_inner_rtol(g, g->recycle != 0);
    cycles = g->graph_cycles > 0 ? g->graph_cycles
                                 : (int)ceil(log(rtol) / log(eta)) + 4;
    if (cycles > g->max_cycles) cycles = g->max_cycles;
    if (cycles < 2) cycles = 2;
  }
  if (!sg.exec || sg.rtol != rtol || sg.max_iter != max_iter || sg.cycles != cycles ||
      sg.inner_rtol != g->inner_rtol || sg.recycle != g->recycle ||
      sg.slabs_p != g->ctx.slabs_p || sg.single_pass != g->ctx.single_pass ||
      sg.resident != g->ctx.resident || sg.fused != g->ctx.fused || sg.gen != g->gen ||
      sg.mg != g->ctx.use_mg || (sg.mg && sg.cycles != g->max_cycles) ||
      sg.slabs_m != g->ctx.slabs_m) {
    bcm_status bst = graph_body_launches(g);  // the old loops' launches so far
    if (bst != BCM_OK) return bst;
    sg.body_kernels[0] = sg.body_kernels[1] = 0;
    if (sg.exec) CUDA_TRY(cudaGraphExecDestroy(sg.exec));
    if (sg.graph) CUDA_TRY(cudaGraphDestroy(sg.graph));
    sg.exec = nullptr;
    sg.graph = nullptr;
    if (!sg.capture_stream)
      CUDA_TRY(cudaStreamCreateWithFlags(&sg.capture_stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamBeginCapture(sg.capture_stream, cudaStreamCaptureModeThreadLocal));
    bcm_status st = issue_graph_step(g, sg.capture_stream, rtol, max_iter, cycles);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(sg.capture_stream, &graph);
    if (st != BCM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return fail(BCM_E_CUDA, "step capture: %s", cudaGetErrorString(e));
    sg.graph = graph;
    size_t nn = 0;
    CUDA_TRY(cudaGraphGetNodes(sg.graph, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) CUDA_TRY(cudaGraphGetNodes(sg.graph, nodes.data(), &nn));
    sg.kernels = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      CUDA_TRY(cudaGraphNodeGetType(nd, &t));
      if (t == cudaGraphNodeTypeKernel) ++sg.kernels;
    }
    CUDA_TRY(cudaGraphInstantiate(&sg.exec, sg.graph, 0));
    sg.rtol = rtol;
    sg.max_iter = max_iter;
    sg.cycles = cycles;
    sg.inner_rtol = g->inner_rtol;
    sg.recycle = g->recycle;
    sg.slabs_p = g->ctx.slabs_p;
    sg.single_pass = g->ctx.single_pass;
    sg.resident = g->ctx.resident;
    sg.fused = g->ctx.fused;
    sg.gen = g->gen;
    sg.mg = g->ctx.use_mg;
    if (sg.mg) sg.cycles = g->max_cycles;
    sg.slabs_m = g->ctx.slabs_m;
  }
  NvtxRange r("bcm_step_graph");
  for (int n = 0; n < n_steps; ++n) {
    CUDA_TRY(cudaGraphLaunch(sg.exec, g->stream));
    g->launch_count += (long long)sg.kernels;  // every kernel node of the step
  }
  if (stats) return collect(g, stats);
  return BCM_OK;
}

extern "C" bcm_status bcm_profile(bcm_grid* g, int enable) {
  if (!g) return fail(BCM_E_INVALID, "grid is NULL");
  bcm_status st = drain_timer(g);
  if (st != BCM_OK) return st;
  g->timer.on = enable != 0;
  return BCM_OK;
}

extern "C" bcm_status bcm_profile_read(bcm_grid* g, double* total_ms, int64_t* launches,
                                       int64_t* launch_count, int reset) {
  if (!g) return fail(BCM_E_INVALID, "grid is NULL");
  bcm_status st = drain_timer(g);
  if (st != BCM_OK) return st;
  if ((st = graph_body_launches(g)) != BCM_OK) return st;
  for (int k = 0; k < BCM_NKERNELS; ++k) {
    if (total_ms) total_ms[k] = g->timer.total_ms[k];
    if (launches) launches[k] = g->timer.launches[k];
  }
  if (launch_count) *launch_count = g->launch_count;
  if (reset) {
    for (int k = 0; k < BCM_NKERNELS; ++k) {
      g->timer.total_ms[k] = 0.0;
      g->timer.launches[k] = 0;
    }
    g->launch_count = 0;
  }
  return BCM_OK;
}

extern "C" bcm_status bcm_set_solver(bcm_grid* g, double inner_rtol, int max_cycles,
                                     int check_every, double barrier_timeout_s, int recycle) {
  if (!g) return fail(BCM_E_INVALID, "grid is NULL");
  if (inner_rtol > 0) {
    if (!(inner_rtol < 1.0)) return fail(BCM_E_INVALID, "inner_rtol must be < 1");
    g->inner_rtol = inner_rtol;
  }
  if (max_cycles > 0) g->max_cycles = max_cycles;
  if (check_every > 0) g->check_every = check_every;
  if (barrier_timeout_s > 0) g->barrier_timeout_s = barrier_timeout_s;
  if (recycle >= 0) g->recycle = recycle ? 1 : 0;
  return BCM_OK;
}

extern "C" bcm_status bcm_get_solver(const bcm_grid* g, double* inner_rtol, int32_t* max_cycles,
                                     int32_t* check_every, double* barrier_timeout_s,
                                     int32_t* recycle) {
  if (!g) return fail(BCM_E_INVALID, "grid is NULL");
  if (inner_rtol) *inner_rtol = g->inner_rtol > 0 ? g->inner_rtol : 0.0;
  if (max_cycles) *max_cycles = g->max_cycles;
  if (check_every) *check_every = g->check_every;
  if (barrier_timeout_s) *barrier_timeout_s = g->barrier_timeout_s;
  if (recycle) *recycle = g->recycle;
  return BCM_OK;
}

extern "C" bcm_status bcm_set_launch(bcm_grid* g, int persistent, int slabs_a, int slabs_b) {
  if (!g) return fail(BCM_E_INVALID, "grid is NULL");
  auto ok = [&](int ns) { return ns == 1 || ns == 2 || ns == 4; };
  if (!ok(slabs_a) || !ok(slabs_b)) return fail(BCM_E_INVALID, "slabs per cube must be 1, 2 or 4");
  if (persistent && g->desc.n_sims > 256)
    return fail(BCM_E_BOUNDS, "the persistent PCG handles at most 256 sims per grid");
  if (g->B / slabs_a < 1 || g->B / slabs_b < 1 || (g->B * g->B / 4) * (g->B / slabs_b) < 1)
    return fail(BCM_E_INVALID, "slab too thin for this cube size");
  if (persistent < 0 || persistent > 5 || persistent == 4)
    return fail(BCM_E_INVALID, "persistent must be 0, 1, 2, 3 or 5");
  if (persistent == 5 && slabs_a != 1)
    return fail(BCM_E_INVALID, "the fused form takes whole cubes");
  if (persistent && g->B != 16 && slabs_a != 1)
    return fail(BCM_E_INVALID, "persistent slabs need 16^3 cubes");
  g->ctx.persistent = persistent ? 1 : 0;
  g->ctx.single_pass = persistent == 2 ? 1 : 0;
  g->ctx.resident = persistent == 3 ? 1 : 0;
  g->ctx.fused = persistent == 5 ? 1 : 0;
  if (persistent) {
    g->ctx.slabs_p = slabs_a;
  } else {
    g->ctx.slabs_a = slabs_a;
    g->ctx.slabs_b = slabs_b;
  }
  return BCM_OK;
}

extern "C" bcm_status bcm_set_stencil_slabs(bcm_grid* g, int slabs) {
  if (!g) return fail(BCM_E_INVALID, "grid is NULL");
  if (slabs != 0 && slabs != 1 && slabs != 2 && slabs != 4)
    return fail(BCM_E_INVALID, "stencil slabs must be 0, 1, 2 or 4");
  g->ctx.slabs_m = g->B == 16 ? slabs : 0;
  return BCM_OK;
}

extern "C" bcm_status bcm_get_stencil_slabs(const bcm_grid* g, int32_t* slabs) {
  if (!g || !slabs) return fail(BCM_E_INVALID, "NULL argument");
  *slabs = g->ctx.slabs_m;
  return BCM_OK;
}

extern "C" bcm_status bcm_solve_pressure(bcm_grid* g, double rtol, int max_iter, bcm_stats* stats) {
  if (!g) return fail(BCM_E_INVALID, "grid is NULL");
  if (!(rtol > 0) || max_iter < 1) return fail(BCM_E_INVALID, "need rtol > 0, max_iter >= 1");
  NvtxRange r("bcm_solve_pressure");
  RUN(BCM_K_MISC, launch_bmean(g->ctx));
  bcm_status st = solve(g, rtol, max_iter);
  if (st != BCM_OK) return st;
  if (stats) return collect(g, stats);
  return BCM_OK;
}

extern "C" bcm_status bcm_fill_halo(bcm_grid* g, int field, int kind, double* dev_out) {
  if (!g || !dev_out) return fail(BCM_E_INVALID, "NULL argument");
  if (kind < 0 || kind > 3) return fail(BCM_E_INVALID, "kind must be 0..3");
  void* ptr;
  size_t cnt;
  int32_t eb;
  bcm_status st = bcm_field(g, field, &ptr, &cnt, &eb);
  if (st != BCM_OK) return st;
  if (field == BCM_UB) return fail(BCM_E_INVALID, "BCM_UB is not a cell field");
  RUN(BCM_K_MISC, launch_fill_halo(g->ctx, ptr, eb == 8, kind, dev_out));
  return BCM_OK;
}

extern "C" bcm_status bcm_set_momentum_scheme(bcm_grid* g, int scheme, double cn_rtol,
                                              int cn_max_iter) {
  if (!g) return fail(BCM_E_INVALID, "grid is NULL");
  if (scheme != BCM_SCHEME_AB2_CENTRAL && scheme != BCM_SCHEME_QUICK_CN)
    return fail(BCM_E_INVALID, "unknown momentum scheme %d", scheme);
  if (!(cn_rtol >= 0) || cn_max_iter < 0) return fail(BCM_E_INVALID, "cn_rtol, cn_max_iter >= 0");
  Ctx& x = g->ctx;
  if (scheme == BCM_SCHEME_AB2_CENTRAL && x.scheme == BCM_SCHEME_QUICK_CN) {
    // N^{n-1} was not kept under Crank-Nicolson: the next AB2 step starts with Euler
    const int one = 1;
    for (int s = 0; s < g->desc.n_sims; ++s)
      CUDA_TRY(cudaMemcpyAsync(g->ws + g->L.ss + sizeof(SimState) * s + offsetof(SimState, ab2_restart),
                               &one, sizeof(int), cudaMemcpyHostToDevice, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
  }
  x.scheme = scheme;
  x.cn_rtol = cn_rtol > 0 ? cn_rtol : (g->f64 ? 1e-10 : 2e-8);
  x.cn_max = cn_max_iter > 0 ? cn_max_iter : 50;
  g->gen += 1;  // a captured step holds the old momentum launches
  return BCM_OK;
}

// ---- wavelet compression of cell fields (bcm_wavelet.cu)

namespace {
// a cell field (4- or 8-byte elements) by id, for compression
bcm_status wavelet_field(bcm_grid* g, int field, void** ptr, int* f64) {
  size_t cnt = 0;
  int32_t eb = 0;
  bcm_status st = bcm_field(g, field, ptr, &cnt, &eb);
  if (st != BCM_OK) return st;
  if (cnt != g->n_cells || (eb != 4 && eb != 8))
    return fail(BCM_E_INVALID, "field %d is not a 4- or 8-byte cell field", field);
  *f64 = eb == 8;
  return BCM_OK;
}
// scratch while no step runs: codes in the PCG residual, per-cube tables in q
struct WavScratch {
  uint32_t *zc, *nbits, *k, *off;
  int* err;
};
WavScratch wavelet_scratch(bcm_grid* g) {
  WavScratch s;
  s.zc = (uint32_t*)g->ctx.f.r;
  uint32_t* q = (uint32_t*)g->ctx.f.q;
  const size_t nc = (size_t)g->desc.n_cubes;
  s.nbits = q;
  s.k = q + nc;
  s.off = q + 2 * nc;
  s.err = (int*)(g->ws + g->L.err) + 8;
  return s;
}
}  // namespace

extern "C" size_t bcm_compress_bound(const bcm_grid* g) {
  if (!g) return 0;
  const size_t nc = (size_t)g->desc.n_cubes, B3 = (size_t)g->B * g->B * g->B;
  return 4 * (8 + nc + nc * (1 + (48 * B3 + 31) / 32));
}

extern "C" bcm_status bcm_compress_field(bcm_grid* g, int field, double step, void* dev_stream,
                                         size_t capacity, size_t* stream_bytes) {
  if (!g || !dev_stream || !stream_bytes) return fail(BCM_E_INVALID, "NULL argument");
  if (!(step > 0) || !std::isfinite(step)) return fail(BCM_E_INVALID, "step must be > 0");
  if ((uintptr_t)dev_stream % 4) return fail(BCM_E_INVALID, "stream must be 4-byte aligned");
  void* ptr = nullptr;
  int f64 = 0;
  bcm_status st = wavelet_field(g, field, &ptr, &f64);
  if (st != BCM_OK) return st;
  const WavScratch s = wavelet_scratch(g);
  const size_t nc = (size_t)g->desc.n_cubes;
  CUDA_TRY(cudaMemsetAsync(s.err, 0, sizeof(int), g->stream));
  RUN(BCM_K_MISC, launch_wavelet_analyze(g->ctx, ptr, f64, step, s.zc, s.nbits, s.k, s.off,
                                         s.err));
  g->launch_count += 1;
  uint32_t total = 0;
  int err = 0;
  CUDA_TRY(cudaMemcpyAsync(&total, s.off + nc, sizeof(uint32_t), cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaMemcpyAsync(&err, s.err, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (err) return fail(BCM_E_BOUNDS, "step too small: a quantized coefficient exceeds 2^30");
  const size_t bytes = 4 * (size_t)total;
  if (bytes > capacity)
    return fail(BCM_E_INVALID, "stream capacity %zu < %zu bytes", capacity, bytes);
  CUDA_TRY(cudaMemsetAsync(dev_stream, 0, bytes, g->stream));
  RUN(BCM_K_MISC, launch_wavelet_encode(g->ctx, s.zc, s.nbits, s.k, s.off, step,
                                        (uint32_t*)dev_stream));
  *stream_bytes = bytes;
  return BCM_OK;
}

extern "C" bcm_status bcm_decompress_field(bcm_grid* g, int field, const void* dev_stream,
                                           size_t bytes) {
  if (!g || !dev_stream) return fail(BCM_E_INVALID, "NULL argument");
  if ((uintptr_t)dev_stream % 4 || bytes % 4) return fail(BCM_E_INVALID, "stream not word-sized");
  void* ptr = nullptr;
  int f64 = 0;
  bcm_status st = wavelet_field(g, field, &ptr, &f64);
  if (st != BCM_OK) return st;
  const size_t words = bytes / 4, nc = (size_t)g->desc.n_cubes;
  if (words < 8 + nc) return fail(BCM_E_INVALID, "stream shorter than its header");
  // the header and the record-size table: the decoder stages the largest record
  std::vector<uint32_t> head(8 + nc);
  CUDA_TRY(cudaMemcpyAsync(head.data(), dev_stream, head.size() * 4, cudaMemcpyDeviceToHost,
                           g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  uint32_t max_payload = 0;
  for (size_t c = 0; c < nc; ++c) max_payload = std::max(max_payload, head[8 + c] ? head[8 + c] - 1 : 0u);
  double step;
  memcpy(&step, head.data() + 6, sizeof step);
  if (head[0] != 0x57434d42u || head[1] != 1u || head[2] != (uint32_t)g->B ||
      head[3] != (uint32_t)nc || !(step > 0))
    return fail(BCM_E_INVALID, "not a wavelet stream of this grid");
  const WavScratch s = wavelet_scratch(g);
  CUDA_TRY(cudaMemsetAsync(s.err, 0, sizeof(int), g->stream));
  RUN(BCM_K_MISC, launch_wavelet_decode(g->ctx, ptr, f64, (const uint32_t*)dev_stream, words,
                                        max_payload, step, s.off, s.err));
  g->launch_count += 1;
  int err = 0;
  CUDA_TRY(cudaMemcpyAsync(&err, s.err, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (err) return fail(BCM_E_INVALID, "malformed cube record in the stream");
  return BCM_OK;
}

// ---- Lagrangian-particle immersed boundary (bcm_ib.cu)

namespace {

struct PartLayout {
  size_t X, F, sim, body, dV, cube, start, ids, count, lat, meta, err, total;
};

// Layout of the caller's particle workspace, and the cube lattice of every sim
// (cube id by cube coordinates, -1 where the sim has no cube).
PartLayout part_plan(const bcm_grid* g, int n, std::vector<int>* lat, std::vector<int>* meta) {
  PartLayout P{};
  const int B = g->B, nc = g->desc.n_cubes, ns = g->desc.n_sims;
  std::vector<int> m(4 * (size_t)ns);
  size_t nl = 0;
  for (int s = 0; s < ns; ++s) {
    m[4 * s] = (int)nl;
    size_t cells = 1;
    for (int e = 0; e < 3; ++e) {
      m[4 * s + 1 + e] = (g->T.sp[s].extent[e] + B - 1) / B;
      cells *= (size_t)m[4 * s + 1 + e];
    }
    nl += cells;
  }
  if (lat) {
    lat->assign(nl ? nl : 1, -1);
    for (int c = 0; c < nc; ++c) {
      const int s = g->T.sim[c];
      const int* ms = &m[4 * (size_t)s];
      const int cx = g->T.ijk[3 * c] / B, cy = g->T.ijk[3 * c + 1] / B, cz = g->T.ijk[3 * c + 2] / B;
      (*lat)[ms[0] + ((size_t)cz * ms[2] + cy) * ms[1] + cx] = c;
    }
  }
  if (meta) *meta = m;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + (bytes ? bytes : 1));
    return o;
  };
  const size_t nn = (size_t)(n > 0 ? n : 0);
  P.X = take(24 * nn);
  P.F = take(24 * nn);
  P.sim = take(4 * nn);
  P.body = take(4 * nn);
  P.dV = take(8 * nn);
  P.cube = take(4 * nn);
  P.start = take(4 * ((size_t)nc + 1));
  P.ids = take(4 * nn);
  P.count = take(4 * (size_t)nc);
  P.lat = take(4 * (nl ? nl : 1));
  P.meta = take(16 * (size_t)ns);
  P.err = take(64);
  P.total = off;
  return P;
}

}  // namespace

extern "C" size_t bcm_particles_bytes(const bcm_grid* g, int32_t n_particles) {
  if (!g || n_particles < 0 || g->desc.max_level != 0) return 0;
  return part_plan(g, n_particles, nullptr, nullptr).total;
}

extern "C" bcm_status bcm_set_particles(bcm_grid* g, int32_t n, const double* xyz,
                                        const int32_t* sim, const int32_t* body,
                                        const double* dV, void* dev_workspace, size_t bytes) {
  if (!g) return fail(BCM_E_INVALID, "grid is NULL");
  if (g->desc.max_level != 0)
    return fail(BCM_E_INVALID, "Lagrangian particles need a single-level grid");
  if (n < 0) return fail(BCM_E_INVALID, "n_particles must be >= 0");
  Ctx& x = g->ctx;
  g->gen += 1;
  if (n == 0) {  // back to the solid-fraction IB
    x.part = PartDev{};
    RUN(BCM_K_SOLID_FRACTION, launch_solid_fraction(x, -1));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    return BCM_OK;
  }
  if (!xyz || !sim || !body || !dV || !dev_workspace)
    return fail(BCM_E_INVALID, "NULL particle array or workspace");
  if ((uintptr_t)dev_workspace % kAlign)
    return fail(BCM_E_INVALID, "particle workspace must be %zu-byte aligned", kAlign);
  std::vector<int> lat, meta;
  const PartLayout P = part_plan(g, n, &lat, &meta);
  if (bytes < P.total)
    return fail(BCM_E_INVALID, "particle workspace too small: %zu < %zu", bytes, P.total);
  for (int q = 0; q < n; ++q) {
    if (sim[q] < 0 || sim[q] >= g->desc.n_sims)
      return fail(BCM_E_INVALID, "particle %d: sim %d out of range", q, sim[q]);
    if (body[q] < 0 || body[q] >= kMaxBodies)
      return fail(BCM_E_INVALID, "particle %d: body %d out of range", q, body[q]);
    if (!(dV[q] > 0) || !std::isfinite(dV[q]))
      return fail(BCM_E_INVALID, "particle %d: dV must be > 0", q);
    for (int e = 0; e < 3; ++e)
      if (!std::isfinite(xyz[3 * q + e])) return fail(BCM_E_INVALID, "particle %d: position", q);
  }
  unsigned char* W = (unsigned char*)dev_workspace;
  cudaStream_t s = g->stream;
  CUDA_TRY(cudaMemsetAsync(W, 0, P.total, s));
  CUDA_TRY(cudaMemcpyAsync(W + P.X, xyz, 24 * (size_t)n, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(W + P.sim, sim, 4 * (size_t)n, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(W + P.body, body, 4 * (size_t)n, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(W + P.dV, dV, 8 * (size_t)n, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(W + P.lat, lat.data(), 4 * lat.size(), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(W + P.meta, meta.data(), 4 * meta.size(), cudaMemcpyHostToDevice, s));
  PartDev D{};
  D.n = n;
  D.X = (double*)(W + P.X);
  D.F = (double*)(W + P.F);
  D.sim = (const int*)(W + P.sim);
  D.body = (const int*)(W + P.body);
  D.dV = (const double*)(W + P.dV);
  D.cube = (int*)(W + P.cube);
  D.set_start = (int*)(W + P.start);
  D.set_ids = (int*)(W + P.ids);
  D.set_count = (int*)(W + P.count);
  D.lat = (const int*)(W + P.lat);
  D.lat_meta = (const int*)(W + P.meta);
  D.err = (int*)(W + P.err);
  x.part = D;
  // the solid fraction plays no part with particles
  CUDA_TRY(cudaMemsetAsync(g->ws + g->L.phi, 0, g->n_cells * (g->f64 ? 8 : 4), s));
  CUDA_TRY(cudaMemsetAsync(g->ws + g->L.near_, 0, (size_t)g->desc.n_cubes, s));
  RUN(BCM_K_IB, launch_ib_bin(x));
  g->launch_count += 2;
  int perr = 0;
  CUDA_TRY(cudaMemcpyAsync(&perr, D.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (perr) {
    x.part = PartDev{};
    RUN(BCM_K_SOLID_FRACTION, launch_solid_fraction(x, -1));
    return fail(BCM_E_BOUNDS, "a Lagrangian particle lies outside every cube");
  }
  return BCM_OK;
}

extern "C" bcm_status bcm_get_particles(bcm_grid* g, double* xyz, double* force, int32_t* cube) {
  if (!g) return fail(BCM_E_INVALID, "grid is NULL");
  const PartDev& D = g->ctx.part;
  const size_t n = (size_t)(D.n > 0 ? D.n : 0);
  if (n == 0) return BCM_OK;
  if (xyz) CUDA_TRY(cudaMemcpyAsync(xyz, D.X, 24 * n, cudaMemcpyDeviceToHost, g->stream));
  if (force) CUDA_TRY(cudaMemcpyAsync(force, D.F, 24 * n, cudaMemcpyDeviceToHost, g->stream));
  if (cube) CUDA_TRY(cudaMemcpyAsync(cube, D.cube, 4 * n, cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return BCM_OK;
}

extern "C" bcm_status bcm_particle_sets(bcm_grid* g, int32_t* start, int32_t* ids) {
  if (!g || !start || !ids) return fail(BCM_E_INVALID, "NULL argument");
  const PartDev& D = g->ctx.part;
  if (D.n <= 0) return fail(BCM_E_INVALID, "no particles set");
  CUDA_TRY(cudaMemcpyAsync(start, D.set_start, 4 * ((size_t)g->desc.n_cubes + 1),
                           cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaMemcpyAsync(ids, D.set_ids, 4 * (size_t)D.n, cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return BCM_OK;
}

extern "C" bcm_status bcm_ib_interpolate(bcm_grid* g, const double* dev_f, double* dev_out) {
  if (!g || !dev_f || !dev_out) return fail(BCM_E_INVALID, "NULL argument");
  if (g->ctx.part.n <= 0) return fail(BCM_E_INVALID, "no particles set");
  RUN(BCM_K_MISC, launch_ib_interpolate(g->ctx, dev_f, dev_out));
  return BCM_OK;
}

extern "C" bcm_status bcm_ib_spread(bcm_grid* g, const double* dev_F, double* dev_out) {
  if (!g || !dev_F || !dev_out) return fail(BCM_E_INVALID, "NULL argument");
  if (g->ctx.part.n <= 0) return fail(BCM_E_INVALID, "no particles set");
  RUN(BCM_K_MISC, launch_ib_spread(g->ctx, dev_F, dev_out));
  return BCM_OK;
}

extern "C" bcm_status bcm_set_preconditioner(bcm_grid* g, int kind) {
  if (!g) return fail(BCM_E_INVALID, "grid is NULL");
  if (kind != BCM_PRECOND_JACOBI && kind != BCM_PRECOND_MULTIGRID)
    return fail(BCM_E_INVALID, "unknown preconditioner %d", kind);
  if (kind == BCM_PRECOND_MULTIGRID && !g->mg_ok)
    return fail(BCM_E_INVALID, "no multigrid hierarchy for this grid (too many aggregate levels)");
  g->ctx.use_mg = kind == BCM_PRECOND_MULTIGRID ? 1 : 0;
  return BCM_OK;
}

extern "C" bcm_status bcm_apply_preconditioner(bcm_grid* g, const double* r, double* z) {
  if (!g || !r || !z) return fail(BCM_E_INVALID, "NULL argument");
  if (!g->solve64 || !g->mg_ok)
    return fail(BCM_E_INVALID, "the preconditioner test path needs an FP64 grid with a multigrid hierarchy");
  const Ctx& x = g->ctx;
  const size_t bytes = g->n_cells * sizeof(double);
  CUDA_TRY(cudaMemcpyAsync(x.f.r, r, bytes, cudaMemcpyDeviceToDevice, g->stream));
  SolveParams prm{};
  RUN(BCM_K_MG, launch_mg_vcycle(x, prm, 2));
  CUDA_TRY(cudaMemcpyAsync(z, x.mg.y[0], bytes, cudaMemcpyDeviceToDevice, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return BCM_OK;
}

extern "C" bcm_status bcm_apply_poisson(bcm_grid* g, const double* x, double* y) {
  if (!g || !x || !y) return fail(BCM_E_INVALID, "NULL argument");
  RUN(BCM_K_MISC, launch_apply_poisson(g->ctx, x, y));
  return BCM_OK;
}
