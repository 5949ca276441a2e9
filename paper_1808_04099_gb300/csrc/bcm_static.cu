// bcm_static.cu -- a pressure solve that allocates no memory at all.
//
// Some callers cannot allocate device memory when they need a solve: a host
// application whose GPU memory is fully reserved up front by its own pool or budget
// (a cudaMalloc would fail or break that budget), or a plugin that is not allowed to
// touch the allocator of the process it runs in.  For them
// bcm_solve_pressure_static runs the FP64 Jacobi-PCG of bcm_solve_pressure with all
// of its working memory (the CG vectors, the per-sim solver state and the block
// counters) in one fixed array that lives in this library's device image.  The
// caller passes only the right-hand side and the pressure (its start value and the
// result); the grid's read-only tables are used as they are.
//
// The array is kStaticBytes (32 MiB) on every GPU that loads the library, held until
// the process exits.  All calls share it: calls that overlap on the GPU (different
// streams, or different host threads on the same device) race and corrupt each other.
// The solve runs in FP64 whatever the grid's precision (the grid's tables and
// per-sim constants are precision independent; its FP32 fields are not touched).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/bcm.h"
#include "bcm_internal.cuh"
#include "bcm_kernels.h"

namespace bcm {
const Ctx* grid_ctx(const bcm_grid* g);
int grid_two_level(const bcm_grid* g);
int grid_device(const bcm_grid* g);
cudaStream_t grid_stream(const bcm_grid* g);
bcm_status grid_fail(bcm_status st, const char* msg);
}  // namespace bcm

using namespace bcm;

namespace {

constexpr size_t kStaticBytes = 32u << 20;
constexpr int kMaxDevices = 64;

// The fixed working memory.  In host code this name is only a stand-in for the
// device symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {nullptr};

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// Device address of the array for `device` (made current by the caller); looked up
// once per device.
bcm_status scratch_for(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices)
    return grid_fail(BCM_E_INVALID, "device ordinal out of range for the static solve");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return grid_fail(BCM_E_CUDA, "cudaGetSymbolAddress of the static solver memory failed");
    g_scratch_ptr[device] = (unsigned char*)p;
  }
  *out = g_scratch_ptr[device];
  return BCM_OK;
}

#define STATIC_TRY(expr)                                                  \
  do {                                                                    \
    cudaError_t e_ = (expr);                                              \
    if (e_ != cudaSuccess) return grid_fail(BCM_E_CUDA, cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

extern "C" bcm_status bcm_solve_pressure_static(bcm_grid* grid, const double* dev_b,
                                                double* dev_p, double rtol, int max_iter,
                                                bcm_stats* stats) {
  if (!grid || !dev_b || !dev_p) return grid_fail(BCM_E_INVALID, "NULL argument");
  if (!(rtol > 0) || max_iter < 1) return grid_fail(BCM_E_INVALID, "need rtol > 0, max_iter >= 1");
  if (grid_two_level(grid))
    return grid_fail(BCM_E_INVALID, "the static solve supports single-level grids");
  const Ctx& base = *grid_ctx(grid);
  const int B = base.B;
  const size_t n = (size_t)base.g.n_cubes * B * B * B;
  const int nsim = base.g.n_sims;
  // layout inside the fixed array: r, p0, p1, q (FP64), SimState[nsim], tickets, flags, guard
  const size_t vec = up256(n * sizeof(double));
  const size_t off_ss = 4 * vec;
  const size_t off_cnt = off_ss + up256(sizeof(SimState) * (size_t)nsim);
  const size_t off_flags = off_cnt + up256(sizeof(unsigned int) * kTicketWords);
  const size_t off_guard = off_flags + 256;
  const size_t need = off_guard + 256;
  if (need > kStaticBytes) {
    char msg[200];
    snprintf(msg, sizeof msg,
             "grid needs %zu bytes of solver memory; the static solve holds at most %zu "
             "(about %zu cells)", need, kStaticBytes, kStaticBytes / 32);
    return grid_fail(BCM_E_BOUNDS, msg);
  }
  int cur = -1;
  STATIC_TRY(cudaGetDevice(&cur));
  if (cur != grid_device(grid))
    return grid_fail(BCM_E_INVALID, "make the grid's device current before the static solve");
  unsigned char* S = nullptr;
  bcm_status st = scratch_for(cur, &S);
  if (st != BCM_OK) return st;

  Ctx x = base;
  x.f64 = 1;  // FP64 vectors and two launches per iteration, as bcm_solve_pressure in FP64
  x.solve64 = 1;
  x.persistent = 0;
  x.f.b = const_cast<double*>(dev_b);
  x.f.p = dev_p;
  x.f.r = S;
  x.f.p0 = S + vec;
  x.f.p1 = S + 2 * vec;
  x.f.q = S + 3 * vec;
  x.g.ss = (SimState*)(S + off_ss);
  x.g.counter = (unsigned int*)(S + off_cnt);
  x.g.flags = (int*)(S + off_flags);
  x.f.guard = (unsigned int*)(S + off_guard);
  cudaStream_t s = grid_stream(grid);
  // the array keeps the previous call's contents: solver state, counters and flags
  // must start at zero
  STATIC_TRY(cudaMemsetAsync(S + off_ss, 0, need - off_ss, s));

  SolveParams prm{};
  prm.rtol = rtol;
  prm.inner_rtol = 1e-5;
  prm.max_iter = max_iter;
  prm.inner_max_iter = max_iter;
  prm.max_cycles = 1;
  prm.mixed = 0;
  prm.guard = x.f.guard;
  STATIC_TRY(launch_solve_begin(x));
  STATIC_TRY(launch_bmean(x));
  STATIC_TRY(launch_residual(x, prm));
  int done = 0, it = 0;
  while (true) {
    STATIC_TRY(cudaMemcpyAsync(&done, x.g.flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    STATIC_TRY(cudaStreamSynchronize(s));
    if (done || it >= max_iter) break;
    for (int m = 0; m < 8 && it < max_iter; ++m, ++it) {
      STATIC_TRY(launch_cg_a(x, prm));
      STATIC_TRY(launch_cg_b(x, prm));
    }
  }
  bcm_status rc = BCM_OK;
  for (int q = 0; q < nsim; ++q) {  // one sim at a time through stack copies
    SimState t, own;
    STATIC_TRY(cudaMemcpyAsync(&t, x.g.ss + q, sizeof(SimState), cudaMemcpyDeviceToHost, s));
    // the step count is the grid's own (the scratch state starts every call at zero)
    STATIC_TRY(cudaMemcpyAsync(&own, base.g.ss + q, sizeof(SimState), cudaMemcpyDeviceToHost, s));
    STATIC_TRY(cudaStreamSynchronize(s));
    if (stats) {
      memset(&stats[q], 0, sizeof(bcm_stats));
      stats[q].cg_iters = t.total_iters;
      stats[q].steps = own.step;
      stats[q].converged = t.converged;
      stats[q].rel_resid = t.bb > 0 ? sqrt(t.rr64 / t.bb) : 0.0;
      stats[q].pcg_form = PCG_TWO_LAUNCH;
    }
    if (t.nonfinite) rc = BCM_E_NONFINITE;
    else if (!t.converged && rc == BCM_OK) rc = BCM_E_NOT_CONVERGED;
  }
  if (rc == BCM_E_NONFINITE) return grid_fail(rc, "non-finite residual");
  if (rc == BCM_E_NOT_CONVERGED) return grid_fail(rc, "pressure solve did not reach rtol");
  return BCM_OK;
}
