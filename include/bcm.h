/*
 * bcm.h -- C ABI of the GB300 (sm_103a) Building Cube Method time-step library.
 *
 * The library advances incompressible-flow simulations on block-structured
 * Cartesian grids of equal cubes (arXiv:1808.04099, section "Building Cube
 * Method") by the fractional-step method of section "Numerical algorithm":
 * momentum sub-step (Eq. substep1, explicit here), immersed-boundary forcing,
 * pressure Poisson equation (Eq. poisson) and projection.  Every step of that
 * path runs in this library's CUDA kernels; nothing falls back to the CPU.
 *
 * Conventions for every entry point
 *   - Plain C types only.  "dev" pointers are CUDA device pointers on the device
 *     that was current at bcm_create_grid; "host" pointers are host memory.
 *   - All device work is issued on the stream given to bcm_create_grid and is
 *     asynchronous unless the call returns host results (bcm_step / bcm_solve_pressure
 *     with a non-NULL stats pointer synchronise that stream).
 *   - Errors are returned as bcm_status; nothing throws or aborts across the ABI.
 *     bcm_last_error() gives a message for the calling thread's last failure.
 *   - Memory: the caller owns the device workspace (bcm_workspace_bytes) and every
 *     pointer it passes; the library keeps only small host tables and never calls
 *     cudaMalloc.  Field views returned by bcm_field point into the workspace.
 *   - rho = 1 throughout (kinematic pressure).
 *
 * Field layout (every cell field): cube-major, x fastest inside a cube:
 *   index = cube * B^3 + (k * B + j) * B + i,  B = cells_per_edge.
 * Outflow face values (BCM_UB): [n_slots][3][B][B]; one slot per (cube, face)
 * pair on an OUTFLOW domain face, in cube order then face order (-x,+x,-y,+y,-z,+z);
 * inside a face patch the lower-numbered tangential axis is fastest.
 */
#ifndef BCM_H
#define BCM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bcm_grid bcm_grid; /* opaque; created by bcm_create_grid */

typedef enum {
    BCM_OK = 0,
    BCM_E_INVALID = -1,       /* bad argument or inconsistent grid description */
    BCM_E_CUDA = -2,          /* a CUDA runtime call failed (message has the code) */
    BCM_E_NOT_CONVERGED = -3, /* a pressure solve hit max_iter; fields stay valid */
    BCM_E_NONFINITE = -4,     /* NaN or Inf found in a residual */
    BCM_E_TIMEOUT = -5,       /* a bounded device wait (grid barrier) ran out */
    BCM_E_BOUNDS = -6         /* a size exceeds a documented maximum */
} bcm_status;

/* Precision of a grid.  BCM_PREC_F64: FP64 state, sweeps and pressure solve.
 * BCM_PREC_F32_REFINE: FP32 state and sweeps; the pressure solve is an FP32 inner PCG
 * inside FP64 defect correction (FP64 residual, pressure and divergence check).
 * BCM_PREC_F64_REFINE: FP64 state and momentum/projection sweeps with the pressure
 * solve of BCM_PREC_F32_REFINE: the FP32 Poisson sweeps without the rounding of the
 * state to FP32 every step (which a flow that amplifies perturbations, like the
 * sphere wake at Re 300, turns into 1e-4 differences over a few hundred steps). */
enum { BCM_PREC_F64 = 0, BCM_PREC_F32_REFINE = 1, BCM_PREC_F64_REFINE = 2 };

/* Domain-face boundary conditions (face order -x,+x,-y,+y,-z,+z). */
enum {
    BCM_BC_WALL = 0,     /* no-slip wall moving with sim_bc_vel (a lid) */
    BCM_BC_INFLOW = 1,   /* prescribed velocity sim_bc_vel x inflow profile */
    BCM_BC_SLIP = 2,     /* free slip */
    BCM_BC_OUTFLOW = 3,  /* convective outflow (speed sim_uconv), pressure 0 */
    BCM_BC_PERIODIC = 4  /* periodic; the opposite face must also be periodic */
};

enum { BCM_BODY_NONE = 0, BCM_BODY_SPHERE = 1, BCM_BODY_ELLIPSOID = 2 };

/* Field ids for bcm_field. */
enum {
    BCM_U = 0, BCM_V = 1, BCM_W = 2, /* cell velocity (state, storage type of the mode) */
    BCM_P = 3,                       /* pressure (always FP64) */
    BCM_PHI = 4,                     /* solid fraction */
    BCM_NX = 5, BCM_NY = 6, BCM_NZ = 7, /* lagged convection N^{n-1} (state) */
    BCM_USTAR = 8, BCM_VSTAR = 9, BCM_WSTAR = 10, /* u* after IB forcing */
    BCM_RHS = 11,                    /* Poisson right-hand side b (FP64) */
    BCM_UB = 12,                     /* outflow face values (state) */
    BCM_NFIELDS = 13
};

/* Grid description.  All arrays are host memory, read during bcm_create_grid only.
 * Several independent simulations ("sims") may share one grid; their cubes are
 * contiguous ranges of the cube list.  Cube corners are in units of the finest cell
 * size h0 / 2^max_level; a level-l cube spans B * 2^(max_level-l) such units.
 * Face neighbours may differ by at most one level (ratio 2). */
typedef struct {
    int32_t n_sims;
    int32_t n_cubes;
    int32_t cells_per_edge;       /* B: 4, 8 or 16 */
    int32_t max_level;            /* 0 or 1 */
    int32_t precision;            /* BCM_PREC_* */
    int32_t lagged_bf16;          /* 1: BCM_PREC_F32_REFINE stores the lagged convection
                                     N^{n-1} (BCM_NX..NZ) as bfloat16; else 0 */
    const int32_t *sim_cube_offset; /* [n_sims+1] */
    const int32_t *cube_ijk;        /* [n_cubes*3] base corners */
    const int8_t *cube_level;       /* [n_cubes] */
    const int32_t *sim_extent;      /* [n_sims*3] domain size, finest-cell units */
    const double *sim_origin;       /* [n_sims*3] */
    const double *sim_h0;           /* [n_sims] level-0 cell size */
    const int32_t *sim_bc;          /* [n_sims*6] BCM_BC_* */
    const double *sim_bc_vel;       /* [n_sims*6*3] wall / inflow velocity per face */
    const double *sim_nu;           /* [n_sims] kinematic viscosity */
    const double *sim_dt;           /* [n_sims] time step (constant) */
    const double *sim_uconv;        /* [n_sims] convective outflow speed */
} bcm_grid_desc;

/* A rigid body moving with centre(t) = center + vel t and orientation
 * exp(t [omega]x) R(quat); quat = (w, x, y, z).  Sphere radius = axes[0]. */
typedef struct {
    int32_t kind;
    int32_t reserved;
    double center[3], axes[3], quat[4], omega[3], vel[3];
} bcm_body;

typedef struct {
    int32_t cg_iters;      /* PCG iterations of the last solve (mixed: inner, summed) */
    int32_t refine_cycles; /* FP64 defect-correction cycles (mixed mode; else 0) */
    int32_t steps;         /* steps taken so far */
    int32_t converged;     /* 1 if the last solve met rtol */
    double rel_resid;      /* ||rhs - K p|| / ||rhs|| at exit (FP64 residual in mixed mode) */
    double div_rel;        /* ||D U^{n+1}|| / ||D U*|| of the corrected face velocities */
    double drag[3];        /* force of the fluid on the bodies, last step */
    double umax;           /* max |u| after the last step */
    int32_t pcg_form;      /* PCG of the last solve: 0 two launches per iteration,
                              1 persistent streaming, 2 persistent single-reduction,
                              3 persistent with the state on chip, 4 multigrid-
                              preconditioned (two launches and a V-cycle), 5 persistent
                              fused (one grid barrier per iteration, bulk-copy staging) */
    int32_t cn_iters;      /* QUICK + Crank-Nicolson: iterations of the last momentum
                              sub-step (0 with Adams-Bashforth) */
} bcm_stats;

/* Bytes of device workspace the grid needs (fields, solver vectors, tables).
 * Returns 0 for an invalid description (see bcm_last_error). */
size_t bcm_workspace_bytes(const bcm_grid_desc *desc);

/* Build the grid: face adjacency (same level, 2:1, domain faces, periodic wrap),
 * boundary tables and per-sim parameters, written into dev_workspace (>= bytes of
 * bcm_workspace_bytes, 256-byte aligned).  Fields start at zero.  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  Paper: "Building Cube Method"
 * (cubes in linear arrays with corners, size and adjacency). */
bcm_status bcm_create_grid(const bcm_grid_desc *desc, void *dev_workspace, size_t bytes,
                           void *cuda_stream, bcm_grid **out);
bcm_status bcm_destroy_grid(bcm_grid *grid);

/* Device view of one field: *dev_ptr, element count and element size in bytes. */
bcm_status bcm_field(bcm_grid *grid, int field, void **dev_ptr, size_t *count,
                     int32_t *elem_bytes);

/* Set the bodies (up to 4) and the eight inflow-profile amplitudes (may be NULL) of
 * one sim, and recompute its solid fraction at the sim's current time.  The inflow
 * profile on INFLOW faces is 1 + sum_m a_m sin(k_m pi s/L_s) sin(l_m pi t/L_t) with
 * (k,l) = (1,1),(1,2),(2,1),(2,2),(1,3),(3,1),(2,3),(3,2) over the face's two
 * tangential coordinates.  The paper represents bodies by Lagrangian particles
 * ("Lagrangian-Eulerian approach"); here a per-cell solid fraction
 * phi = (1 - tanh(d / 1.5h)) / 2 of the signed distance d stands in for them. */
bcm_status bcm_set_geometry(bcm_grid *grid, int sim, const bcm_body *bodies, int n_bodies,
                            const double *inflow_modes);

/* Reset step counters (time = 0) of all sims; the next step starts AB2 with Euler. */
bcm_status bcm_reset_time(bcm_grid *grid);

/* The time-averaged force on the bodies of every sim: host out[3 * n_sims] gets, per
 * sim, the mean over the steps taken since the last reset of the per-step drag
 * (bcm_stats.drag; its x component averaged over N steps is the objective J of the
 * adjoint, bcm_adjoint_step).  reset != 0 then starts a new average (bcm_reset_time
 * does too).  Zeros before the first step.  BCM_E_INVALID for NULL arguments. */
bcm_status bcm_drag_mean(bcm_grid *grid, int reset, double *out);

/* Set the step counter of every sim (time = step * dt), e.g. when restarting from a
 * checkpoint; step 0 makes the next step the Euler start of AB2. */
bcm_status bcm_set_step(bcm_grid *grid, int step);

/* Advance every sim by n_steps fractional steps ("Numerical algorithm"):
 * solid fraction (moving bodies), momentum sub-step with halo staging, IB forcing,
 * Poisson right-hand side, Jacobi-PCG pressure solve to relative residual rtol
 * (FP64, or FP32 inner PCG inside FP64 defect correction), projection.
 * stats: host array [n_sims] or NULL (then nothing is synchronised). */
bcm_status bcm_step(bcm_grid *grid, int n_steps, double rtol, int max_iter, bcm_stats *stats);

/* bcm_step as a CUDA graph.  The first call (and any call whose rtol, max_iter or
 * solver settings differ from the captured ones) captures one step on a library
 * stream and instantiates it; every call then launches the graph n_steps times on
 * the grid's stream, with no host synchronisation unless stats is non-NULL.  The
 * captured step uses the persistent PCG (grids of at most 256 sims) and, in mixed
 * mode, a fixed budget of ceil(log rtol / log inner_rtol) + 4 defect-correction
 * cycles per solve (at most max_cycles; cycles after a sim has converged return at
 * once; a sim needing more is reported not converged).  With the multigrid
 * preconditioner the PCG iterations and the defect-correction cycles run as
 * conditional while nodes whose conditions the V-cycle's decisions and the FP64
 * residual set on the device (bounded by max_iter and max_cycles); the launch count
 * of bcm_profile_read includes the launches inside those loops. */
bcm_status bcm_step_graph(bcm_grid *grid, int n_steps, double rtol, int max_iter,
                          bcm_stats *stats);

/* Solver controls (defaults in brackets): inner_rtol, the relative reduction of the
 * FP32 inner PCG per defect-correction cycle in mixed mode [0.1 with recycle, 1e-4 with
 * the multigrid preconditioner, else 1e-5]; max_cycles, the
 * cap on FP64 residual evaluations per solve [30]; check_every, PCG iterations
 * between two reads of the device convergence flags by the host [8];
 * barrier_timeout_s, the longest wait of a block at a grid barrier of the
 * persistent PCG before the solve gives up with BCM_E_TIMEOUT [2 s]; recycle, in
 * mixed mode with the persistent PCG: 1 keeps the inner CG's search direction across
 * defect-correction cycles (the FP64 residual replaces the FP32 one: a reliable
 * update), 0 restarts the inner CG every cycle [1].  A value <= 0 keeps the current
 * setting (recycle: a value < 0). */
bcm_status bcm_set_solver(bcm_grid *grid, double inner_rtol, int max_cycles, int check_every,
                          double barrier_timeout_s, int recycle);

/* The current solver controls of bcm_set_solver (any pointer may be NULL); inner_rtol
 * is 0 while the automatic per-cycle reduction is in effect. */
bcm_status bcm_get_solver(const bcm_grid *grid, double *inner_rtol, int32_t *max_cycles,
                          int32_t *check_every, double *barrier_timeout_s, int32_t *recycle);

/* Launch shape of the PCG.  persistent = 5 (mixed mode on 16^3 cubes, grids of at most
 * 160 sims and 256 cubes per SM): one cooperative launch per solve, one block of 1024
 * threads (four x-adjacent cells of the cube in hand each) per SM,
 * one grid barrier per iteration (the beta of the next iteration follows from <q,z> and
 * <q,D^-1 q> of the same pass; q = K p is applied again rather than stored), each cube's
 * r, p, x and its neighbours' face planes staged by bulk asynchronous copies two cubes
 * ahead; grids it does not fit run persistent = 1.  persistent = 1: every PCG solve is one
 * cooperative launch whose blocks loop over the iterations with two grid-wide barriers
 * each, streaming the vectors through global memory (the mixed-mode default; in a
 * defect-correction cycle it also adds its correction to the FP64 pressure before it
 * returns, where the other forms launch BCM_K_ADD_CORRECTION);
 * persistent = 3: the same iteration with each cube's search direction kept in
 * shared memory, when every cube fits a co-resident block of at most two cubes (FP32
 * inner solve, 16^3 or 8^3 cubes, slabs_a = 1), else the streaming form; persistent = 2:
 * the single-reduction form of the iteration (Chronopoulos-Gear: one pass and one
 * barrier per iteration, three more vectors, the same iterates in exact arithmetic).
 * slabs_a = z-slabs per cube of the streaming work items (1, 2 or 4; 16^3 cubes only
 * for 2 and 4; slabs_a = 1 with 5).  persistent = 0: two launches per iteration (the FP64
 * default), one CTA
 * per z-slab, slabs_a / slabs_b slabs per cube for pass A / pass B.  Results do not
 * depend on the shape beyond rounding; bcm_stats.pcg_form says which form ran.
 * BCM_E_INVALID for other values. */
bcm_status bcm_set_launch(bcm_grid *grid, int persistent, int slabs_a, int slabs_b);

/* z-slabs per 16^3 cube of the momentum and Poisson right-hand-side kernels (one block
 * per slab, its tiles of u*, v*, w* with their halos in shared memory): 1, 2 or 4; 0
 * the default (2 in FP32, 4 in FP64).  Other cube sizes take whole cubes (the value is
 * ignored).  Results do not depend on it.  BCM_E_INVALID for other values. */
bcm_status bcm_set_stencil_slabs(bcm_grid *grid, int slabs);
bcm_status bcm_get_stencil_slabs(const bcm_grid *grid, int32_t *slabs);

/* Preconditioner of the pressure PCG.  BCM_PRECOND_JACOBI (the default): M = diag(K).
 * BCM_PRECOND_MULTIGRID: one symmetric V-cycle of a geometric multigrid per iteration
 * (the paper solves the pressure equation by multigrid on its cubes): every cube is
 * coarsened 2:1 down to one cell, then the cubes of each sim are aggregated 2x2x2 up
 * to one node; piecewise-constant transfers, Galerkin coarse operators, one damped
 * Jacobi sweep (omega = 0.8) before and after each coarse correction, four on the top
 * level; on a two-level grid the refined cubes of each level-0 position are aggregated
 * first (the per-cube levels keep the 2:1 flux form).  With multigrid the solve
 * runs two launches per iteration plus the V-cycle (no persistent form); in graph
 * steps its iteration and defect-correction loops are conditional graph nodes.  Results
 * agree with the Jacobi solve to the solver tolerance. */
enum { BCM_PRECOND_JACOBI = 0, BCM_PRECOND_MULTIGRID = 1 };
bcm_status bcm_set_preconditioner(bcm_grid *grid, int kind);

/* Solve the pressure Poisson equation (Eq. poisson) for the current BCM_RHS into
 * BCM_P (warm start from BCM_P).  stats as in bcm_step. */
bcm_status bcm_solve_pressure(bcm_grid *grid, double rtol, int max_iter, bcm_stats *stats);

/* Copy one cell field with its two-layer face halos, filled by the paper's halo
 * rules ("Building Cube Method", Fig. halo-hanging-node): same-level copy,
 * fine->coarse mean of the 2x2x2 fine cells, coarse->fine copy of the coarse cell,
 * and the domain boundary rules.  kind 0,1,2 = velocity component (field BCM_U,
 * BCM_V, BCM_W or the starred ones), 3 = pressure rules.  dev_out: FP64
 * [n_cubes][(B+4)^3], z slowest; cells that are not face halos are set to 0.
 * The field is converted to FP64. */
bcm_status bcm_fill_halo(bcm_grid *grid, int field, int kind, double *dev_out);

/* Pressure solve that allocates no memory, for callers that cannot allocate device
 * memory at the moment they solve: an application that reserves all GPU memory up
 * front for its own pool or budget, or a plugin that must not call the allocator of
 * the process it runs in.  There is no counterpart in the paper: it is the FP64
 * Jacobi-PCG of bcm_solve_pressure (two launches per iteration) with its working
 * memory (CG vectors, per-sim solver state, block counters) in one fixed 32 MiB array
 * inside the library's device image instead of the grid workspace.  It solves in FP64
 * on grids of either precision.  dev_b: right-hand side (FP64, grid layout, read);
 * dev_p: start value in, solution out (FP64, grid layout); the grid's own fields are
 * not touched.  The grid's device must be current.
 * Limits and sharing: grids needing more than 32 MiB (4 FP64 vectors, i.e. about
 * 1M cells, plus per-sim state) are rejected with BCM_E_BOUNDS; single-level grids
 * only (BCM_E_INVALID).  The array stays allocated on every GPU that loads the
 * library until the process exits, and every call reuses it: calls that overlap on
 * the GPU (other streams or host threads on the same device) race.  The first call on
 * each device looks up the array's device address.  Synchronises the grid's stream.
 * stats (host, [n_sims], or NULL): cg_iters, steps (the grid's step count), converged,
 * rel_resid and pcg_form are filled; div_rel, drag, umax and cn_iters are 0. */
bcm_status bcm_solve_pressure_static(bcm_grid *grid, const double *dev_b, double *dev_p,
                                     double rtol, int max_iter, bcm_stats *stats);

/* y = K x with K = -V A the flux-form pressure operator of Eq. poisson (FP64). */
bcm_status bcm_apply_poisson(bcm_grid *grid, const double *dev_x, double *dev_y);

/* z = M^-1 r, one multigrid V-cycle (the preconditioner of BCM_PRECOND_MULTIGRID), on
 * FP64 grids: a test path.  It uses the grid's PCG residual buffer as
 * scratch, so call it between solves.  BCM_E_INVALID for other grids. */
bcm_status bcm_apply_preconditioner(bcm_grid *grid, const double *dev_r, double *dev_z);

/* Discrete adjoint of the fractional step, for gradients of J = sum_n w_n F_x^n (F_x^n
 * the drag of step n) with respect to the eight inflow-profile amplitudes a_m and the
 * centre of a fixed sphere (body 0).  Every operator of the step is transposed exactly,
 * boundary ghosts included; the adjoint Poisson solve is the same Jacobi-PCG (K is
 * symmetric).  No counterpart in the paper, which has no adjoint; the step it reverses
 * is the paper's ("Numerical algorithm").  FP64 single-level grids whose sims have an
 * outflow face; bodies: fixed spheres.
 *   bcm_adjoint_bytes:  bytes of the adjoint workspace (caller-owned device memory).
 *   bcm_adjoint_init:   zero the adjoint state (lambda of the final state = 0).
 *   bcm_adjoint_step:   reverse one step n.  state[7] = device pointers to the forward
 *                       state at the start of step n: u, v, w, N^{n-1}_x, _y, _z (the
 *                       BCM_NX.. fields before the step) and the outflow face values;
 *                       first_step = 1 for step 0 (Euler start); drag_weight = w_n;
 *                       rtol / max_iter of the adjoint Poisson solve.  dev_dJ: FP64
 *                       device array [11] += dJ/d(a_1..a_8, c_x, c_y, c_z).
 * Call bcm_adjoint_step for n = N-1 down to 0 with the same workspace. */
size_t bcm_adjoint_bytes(const bcm_grid *grid);
bcm_status bcm_adjoint_init(bcm_grid *grid, void *dev_adj, size_t bytes);
bcm_status bcm_adjoint_step(bcm_grid *grid, void *dev_adj, size_t bytes, const void *const *state,
                            int first_step, double drag_weight, double rtol, int max_iter,
                            double *dev_dJ);

/* ---- Momentum scheme (Eq. substep1).  BCM_SCHEME_AB2_CENTRAL (default): explicit
 * Adams-Bashforth convection (central) and Euler diffusion.  BCM_SCHEME_QUICK_CN: the
 * paper's production scheme, QUICK convection (face values by quadratic upstream
 * interpolation 6/8 C + 3/8 D - 1/8 U on the central face velocities; two ghost layers)
 * and Crank-Nicolson for convection and diffusion,
 *   (u~ - u^n)/dt + (N(u~) + N(u^n))/2 = nu (L(u~) + L(u^n))/2,
 * solved per step by the iteration from the forward-Euler predictor u^(0) = 2 E - u^n,
 *   u^(k+1) = (E - dt/2 N(u^(k)) + dt nu/2 (sum of the 6 neighbours of u^(k))/h^2)
 *             / (1 + 3 dt nu/h^2),   E = u^n + dt (-N(u^n) + nu L(u^n))/2,
 * until ||u^(k+1) - u^(k)|| <= cn_rtol ||u^(k+1)|| per sim (all components), or the
 * update has reached the rounding floor (<= 64 unit roundoffs of ||u^(k+1)||) and stopped
 * shrinking (its square >= 0.99 of the previous one), or cn_max_iter iterations; ghosts
 * of u^(k) (velocities of t^{n+1}) follow the halo rules with the outflow values advanced
 * to t^{n+1}; those of u^n in E with the outflow values of t^n.  The mixed mode
 * iterates on the increment u^(k) - u^n in FP32.  cn_rtol = 0 / cn_max_iter = 0 select
 * the defaults (1e-10 FP64, 2e-8 mixed, i.e. down to the FP32 floor; 50).
 * Switching back to AB2 restarts it with an Euler step (N^{n-1} := N^n).  The adjoint
 * rejects grids on QUICK + Crank-Nicolson.  Errors: BCM_E_INVALID. */
enum { BCM_SCHEME_AB2_CENTRAL = 0, BCM_SCHEME_QUICK_CN = 1 };
bcm_status bcm_set_momentum_scheme(bcm_grid *grid, int scheme, double cn_rtol, int cn_max_iter);

/* ---- Wavelet compression of cell fields for checkpoints (section "Data compression":
 * a discrete wavelet transform per cube, one level of quantization, an encoder, one
 * stream that records the size of every cube's compressed record).
 * Transform: log2 B levels of a separable 3-D CDF 5/3 lifting transform of each cube's
 * B^3 values (d_i = x_{2i+1} - (x_{2i} + x_{2i+2})/2, s_i = x_{2i} + (d_{i-1} + d_i)/4,
 * symmetric at the ends, passes x, y, z per level on the low band, coefficients in place,
 * FP64 without contraction).  Quantizer q = rint(c / step).  Encoder in place of zlib:
 * Golomb-Rice on z = zigzag(q) with k = floor(log2(mean z)) per cube (at most 24); a
 * value with u = z >> k < 16 takes u one-bits, a zero-bit and the k low bits of z, else
 * 16 one-bits and the 32 bits of z; bits LSB-first in 32-bit little-endian words.
 * Stream (32-bit words): 0x57434D42 ("BCMW"), 1, B, n_cubes, 0, 0, step (FP64, 2 words),
 * the word count of every cube record, then the records (k | nbits << 5, then
 * ceil(nbits / 32) payload words).  The reconstruction error is at most
 * (1/2 + 7.3125 log2 B) step (the inverse lifting steps bound it).
 * field: BCM_U .. BCM_RHS except bfloat16 N fields.  The calls use the PCG scratch
 * vectors and must not overlap a step on the grid's stream (they are stream ordered).
 * bcm_compress_bound: bytes of the largest possible stream of this grid.
 * bcm_compress_field: writes the stream into dev_stream (4-byte aligned, capacity
 *   bytes) and *stream_bytes (host; synchronises).  Errors: BCM_E_INVALID (bad
 *   argument or field, capacity below the stream), BCM_E_BOUNDS (a coefficient / step
 *   beyond 2^30).
 * bcm_decompress_field: decodes a stream of this grid (same B and cube count) into the
 *   field (rounded to its storage type); bits of a record after its first B^3 codes
 *   are ignored.  Errors: BCM_E_INVALID (not such a stream, a malformed record such as
 *   one whose B^3 codes do not fit in its bit count: the field is then undefined).
 *   Synchronises (it reads the header and the record sizes to the host). */
size_t bcm_compress_bound(const bcm_grid *grid);
bcm_status bcm_compress_field(bcm_grid *grid, int field, double step, void *dev_stream,
                              size_t capacity, size_t *stream_bytes);
bcm_status bcm_decompress_field(bcm_grid *grid, int field, const void *dev_stream,
                                size_t bytes);

/* ---- Lagrangian-particle immersed boundary (section "Lagrangian Data Structure";
 * section "Lagrangian-Eulerian Interaction", Eqs. ddeltai and ddeltap with the smoothed
 * 3-point delta phi(r) = 3/4 - r^2 for |r| <= 1/2, (9/4 - 3|r| + r^2)/2 for
 * 1/2 < |r| <= 3/2, 0 beyond; the forcing sub-step and the position update of section
 * "Numerical algorithm"), single-level grids only.
 *
 * Particle q sits at xyz[3q..3q+2] (physical coordinates of its sim), belongs to sim
 * sim[q] and is moved by body body[q] of that sim (0 .. 3, as set by
 * bcm_set_geometry; a body slot without a body gives U_s = 0); dV[q] > 0 is its volume
 * weight (dc1 dc2 dc3 of Eq. ddeltap; one particle per surface cell: h^3).  With
 * particles set, every step replaces the solid-fraction forcing (the solid fraction is
 * zero) by
 *   U_q = sum over the 27 nearest cells of u~ phi(r_x) phi(r_y) phi(r_z)   (r = (x - X)/h)
 *   F_q = (U_s(X_q, t^n) - U_q) / dt                  (rho = 1)
 *   u*  = u~ + dt sum_q F_q phi phi phi dV_q / h^3
 * (cells outside the domain are left out of both sums), reports the force on the
 * bodies -sum_q F_q dV_q as the sim's drag, and after the step moves every particle by
 * X += dt U_s(X, t^{n+1}) with its body's rigid motion; particles are grouped into
 * per-cube sets that are rebuilt after every move.
 *
 * bcm_particles_bytes: device workspace bytes for n particles on this grid (0 on a
 *   two-level grid).
 * bcm_set_particles: copies the host arrays into the caller's device workspace
 *   (256-byte aligned, at least bcm_particles_bytes; it must outlive the
 *   particles: until bcm_set_particles(grid, 0, ...) or bcm_destroy_grid) and builds
 *   the sets.  n = 0 returns to the solid-fraction IB (other arguments ignored).
 *   Errors: BCM_E_INVALID (two-level grid, NULL array, sim or body out of range,
 *   dV <= 0, non-finite position, small or misaligned workspace), BCM_E_BOUNDS (a
 *   particle outside every cube; the grid returns to the solid-fraction IB).  Synchronises.
 * bcm_get_particles: host copies (each may be NULL) of the positions [n*3], the last
 *   step's force per particle [n*3] and the cube each particle lies in [n] (-1 outside).
 * bcm_particle_sets: host copies of the per-cube sets: the particles of cube c are
 *   ids[start[c] .. start[c+1]) (start: [n_cubes+1], ids: [n]; order within a set
 *   arbitrary).
 * bcm_ib_interpolate / bcm_ib_spread (test paths, FP64 device arrays, asynchronous):
 *   out[q] = sum_cells f phi phi phi;  out[cell] += sum_q F[q] phi phi phi dV_q / h^3.
 * A particle that leaves every cube carries no force from then on; bcm_step and
 * bcm_step_graph called with a stats pointer return BCM_E_BOUNDS once that happened.
 * The adjoint rejects grids with particles. */
size_t bcm_particles_bytes(const bcm_grid *grid, int32_t n_particles);
bcm_status bcm_set_particles(bcm_grid *grid, int32_t n_particles, const double *xyz,
                             const int32_t *sim, const int32_t *body, const double *dV,
                             void *dev_workspace, size_t bytes);
bcm_status bcm_get_particles(bcm_grid *grid, double *xyz, double *force, int32_t *cube);
bcm_status bcm_particle_sets(bcm_grid *grid, int32_t *start, int32_t *ids);
bcm_status bcm_ib_interpolate(bcm_grid *grid, const double *dev_f, double *dev_out);
bcm_status bcm_ib_spread(bcm_grid *grid, const double *dev_F, double *dev_out);

/* Kernel classes for bcm_profile_read. */
enum {
    BCM_K_SOLID_FRACTION = 0, /* solid fraction and body index per cell */
    BCM_K_MOMENTUM = 1,       /* halo staging + momentum sub-step + IB forcing */
    BCM_K_RHS = 2,            /* Poisson right-hand side */
    BCM_K_RESIDUAL = 3,       /* FP64 residual (PCG start / defect-correction cycle) */
    BCM_K_CG_A = 4,           /* PCG pass A: new direction, K p, <p, Kp> */
    BCM_K_CG_B = 5,           /* PCG pass B: iterate and residual update, <r,z>, <r,r> */
    BCM_K_ADD_CORRECTION = 6, /* mixed: x += e (forms other than persistent = 1) */
    BCM_K_CORRECT = 7,        /* projection + FP64 divergence check */
    BCM_K_MISC = 8,           /* bookkeeping and test-path kernels */
    BCM_K_PCG = 9,            /* persistent PCG: all iterations of one solve (with
                                 persistent = 1 also the cycle's x += e) */
    BCM_K_MG = 10,            /* multigrid V-cycle (BCM_PRECOND_MULTIGRID) */
    BCM_K_IB = 11,            /* Lagrangian particles: forcing, position update, sets */
    BCM_NKERNELS = 12
};

/* Timing of the library's own kernels: while enabled, every kernel the grid launches
 * is bracketed by two CUDA events on the grid's stream.  No device memory is used. */
bcm_status bcm_profile(bcm_grid *grid, int enable);

/* Per-class totals since the last reset: total_ms[BCM_NKERNELS] and
 * launches[BCM_NKERNELS] of timed launches (either may be NULL), and launch_count,
 * every kernel launch issued (timed or not).  Synchronises the grid's stream when
 * timed launches are pending.  reset != 0 clears all counters after reading. */
bcm_status bcm_profile_read(bcm_grid *grid, double *total_ms, int64_t *launches,
                            int64_t *launch_count, int reset);

/* Measured fused multiply-add rate of the current device in FLOP/s (2 per FMA),
 * FP64 (fp64 = 1) or FP32 (fp64 = 0): eight independent FMA chains per thread, eight
 * blocks of 256 threads per SM, about 20 ms per timed run, the best of three runs
 * timed by CUDA events on a stream of its own.  No counterpart in the paper: it is the
 * denominator of the FP64 kernels' arithmetic roofline.  Uses no device memory
 * beyond a 16-byte sink in the library image; synchronises its stream. */
bcm_status bcm_measure_fma_rate(int fp64, double *flops_per_s);

const char *bcm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
