/*
 * bcm_oracle.h -- plain, slow FP64 CPU oracle of the Building Cube Method time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark call this library.  It shares no code, header, table or
 * helper with the CUDA library: it builds its own cube adjacency from the raw
 * cube list, keeps a ghosted (B+2H)^3 copy of each cube as the paper's data
 * structure does, and applies every stencil as plain nested loops.
 *
 * What it follows (section / equation of arXiv:1808.04099):
 *   - cube mesh as linear arrays, equal cells per cube  ("Building Cube Method")
 *   - cell centres x_i = x_c + (i+1/2) dx             (Eq. cell-center)
 *   - halo filled from neighbouring cubes; fine->coarse by a weighted mean,
 *     coarse->fine by copying the coarse value      ("Building Cube Method", Fig. halo)
 *   - fractional step: momentum sub-step, IB forcing sub-step, projection with
 *     a pressure Poisson equation                    (Eq. substep1, Eq. poisson, "Numerical algorithm")
 *   - simplified rigidity constraint u = u_s inside the body ("Mathematical Framework")
 * Readings where the paper is silent or garbled are listed in the .c file header.
 *
 * Layout of every cell field: cube-major, cube c holds B^3 values, x fastest:
 *   idx = c*B^3 + (k*B + j)*B + i.
 * Ghosted arrays (orc_fill_ghosts) hold (B+2H)^3 values per cube with H = 2.
 * Outflow face values: [n_slots][3][B][B]; slot order = cube order, then face order.
 */
#ifndef BCM_ORACLE_H
#define BCM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_BODIES 4
#define ORC_BODY_STRIDE 17
#define ORC_NMODES 8

typedef struct orc_grid orc_grid;

typedef struct {
    int32_t cg_iters;     /* PCG iterations of the last solve */
    int32_t steps;        /* steps taken by this sim so far */
    double rel_resid;     /* ||rhs - K p|| / ||rhs|| (recurrence residual at exit) */
    double div_rel;       /* ||D U^{n+1}|| / ||D U*|| from the corrected face velocities */
    double drag[3];       /* force of the fluid on the bodies */
    double umax;          /* max |u| after the step */
} orc_stats;

/* Build the oracle's own copy of the grid.  Arrays as in the workload description:
 * sim_off[n_sims+1], ijk[n_cubes*3] (finest-cell units), level[n_cubes],
 * extent[n_sims*3], origin[n_sims*3], h0[n_sims], bc[n_sims*6],
 * bcvel[n_sims*18], nu, dt, uconv [n_sims], bodies[n_sims*4*17], modes[n_sims*8].
 * Returns NULL on an inconsistent grid (message in orc_error()). */
orc_grid *orc_create(int B, int max_level, int n_sims, int n_cubes, const int32_t *sim_off,
                     const int32_t *ijk, const int8_t *level, const int32_t *extent,
                     const double *origin, const double *h0, const int32_t *bc,
                     const double *bcvel, const double *nu, const double *dt,
                     const double *uconv, const double *bodies, const double *modes);
void orc_destroy(orc_grid *g);
const char *orc_error(void);
int orc_n_slots(const orc_grid *g);
int orc_threads(void);
int orc_set_threads(int n); /* threads of the parallel loops; returns the previous count */

/* Face adjacency: out[c*6+f] = same-level neighbour id, -1 domain boundary,
 * -2 coarser neighbour, -3 four finer neighbours. */
void orc_neighbors(const orc_grid *g, int32_t *out);

/* Ghost fill of one cell field.  kind 0,1,2 = velocity component x,y,z (uses ub
 * at outflow faces; may be NULL when there is none), 3 = pressure.
 * out: [n_cubes*(B+4)^3]; cells that are not face halos are left 0. */
void orc_fill_ghosts(const orc_grid *g, const double *f, int kind, const double *ub,
                     double *out);

/* Solid fraction phi and body velocity at per-sim times t[n_sims]. */
void orc_solid_fraction(const orc_grid *g, const double *t, double *phi, double *us,
                        double *vs, double *ws);

/* Explicit convection N(u) (component c) and Laplacian L(u_c); velocity ghosts from ub. */
void orc_convection_diffusion(const orc_grid *g, const double *u, const double *v,
                              const double *w, const double *ub, double *nx, double *ny,
                              double *nz, double *lx, double *ly, double *lz);

/* y = K x with K = -V A, the flux-form pressure operator (SPD / SPSD). */
void orc_apply_poisson(const orc_grid *g, const double *x, double *y);
/* diag(K) */
void orc_poisson_diag(const orc_grid *g, double *d);

/* Poisson right-hand side b = (rho/dt) D U* (face velocities from u*, BC at domain faces). */
void orc_rhs(const orc_grid *g, const double *us, const double *vs, const double *ws,
             const double *ub_new, double *b);

/* Solve A p = b for every sim (Jacobi PCG on K p = -V b, warm start p).
 * Returns 0, or -3 when some sim hit max_iter. */
int orc_solve_pressure(const orc_grid *g, const double *b, double *p, double rtol,
                       int max_iter, orc_stats *stats);

/* Advance every sim by nsteps time steps.  State arrays are updated in place:
 * u,v,w,p [n_cells]; nx,ny,nz lagged convection [n_cells]; ub [n_slots*3*B*B];
 * step[n_sims] step counters (0 = first step: Euler start of AB2).
 * Returns 0, or -3 when a pressure solve hit max_iter. */
int orc_step(const orc_grid *g, double *u, double *v, double *w, double *p, double *nx,
             double *ny, double *nz, double *ub, int32_t *step, int nsteps, double rtol,
             int max_iter, orc_stats *stats);

/* QUICK convection N(u) of every component (R20 in the .c file header); ghosts from ub. */
void orc_convection_quick(const orc_grid *g, const double *u, const double *v, const double *w,
                          const double *ub, double *nx, double *ny, double *nz);
/* Momentum scheme of the following steps: 0 AB2 + central (default), 1 QUICK +
 * Crank-Nicolson iterated to cn_rtol (at most cn_max iterations).  Returns 0, or -1. */
int orc_set_scheme(orc_grid *g, int scheme, double cn_rtol, int cn_max);

/* Lagrangian particles (R19 in the .c file header), single-level grids.
 * Particle q: position X[3q..3q+2], sim psim[q], body pbody[q] (0 .. ORC_MAX_BODIES-1 of
 * its sim), weight dV[q] (the particle's volume dc1 dc2 dc3 of Eq. ddeltap). */
double orc_delta3(double r);
/* out[q] = sum over cells of f * delta weight (Eq. ddeltai) */
void orc_ib_interpolate(const orc_grid *g, const double *f, int n, const double *X,
                        const int32_t *psim, double *out);
/* out[cell] += sum over particles of F[q] * delta weight * dV[q] / h^3 (Eq. ddeltap) */
void orc_ib_spread(const orc_grid *g, int n, const double *X, const int32_t *psim,
                   const double *F, const double *dV, double *out);
/* vel[3q..] = velocity of particle q's body at X and time t[psim[q]] */
void orc_ib_body_velocity(const orc_grid *g, int n, const double *X, const int32_t *psim,
                          const int32_t *pbody, const double *t, double *vel);
/* orc_step with the particle forcing in place of the solid fraction; X is advanced in
 * place; F[3q..] (may be NULL) receives the last step's force per particle.  Returns
 * -1 on a two-level grid. */
int orc_step_particles(const orc_grid *g, double *u, double *v, double *w, double *p,
                       double *nx, double *ny, double *nz, double *ub, int32_t *step,
                       int nsteps, double rtol, int max_iter, orc_stats *stats, int n_particles,
                       double *X, const int32_t *psim, const int32_t *pbody, const double *dV,
                       double *F);

/* Wavelet compression of cell fields (R21 in the .c file header). */
void orc_dwt3_forward(int B, double *x);
void orc_dwt3_inverse(int B, double *x);
long orc_wavelet_compress(int B, int n_cubes, const double *f, double step, uint32_t *out,
                          long capacity);
int orc_wavelet_decompress(const uint32_t *in, long words, double *f);

#ifdef __cplusplus
}
#endif
#endif
