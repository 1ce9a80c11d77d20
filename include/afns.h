/*
 * afns.h -- C-ABI of libafns: the per-Runge-Kutta-stage update of the compact
 * fourth-order positivity-preserving active flux (AF) method for the 1D/2D
 * compressible Navier-Stokes equations on Cartesian grids (Duan, Barsukow,
 * Klingenberg, arXiv 2609.29081), on one NVIDIA B300 GPU (sm_103a).
 *
 * The problem solved is Eq. (1) with the fluxes of Eq. (2), Newtonian stress and
 * Fourier heat flux of Eq. (3), nondimensional temperature T = p/rho,
 * kappa = gamma mu / ((gamma-1) Pr) and the ideal-gas law (Sec. 1). The degrees of
 * freedom are cell averages plus shared point values (Sec. 2.1, Sec. 2.2).
 *
 * Conventions for every call:
 *  - Every call returns af_status; nothing aborts, traps on the device or throws
 *    across this boundary. On failure af_last_error() describes the cause.
 *  - All device work is issued on the CUDA stream given to af_create (NULL = the
 *    legacy default stream). Calls that return host data synchronise that stream.
 *  - A context is not thread-safe; use one context per host thread.
 *
 * DoF layout of af_set_state / af_get_state ("site arrays", conservative
 * variables, component-major, x index fastest, FP64):
 *   2D: site[0] = avg [4][n2  ][n1  ]  cell averages U-bar_{ij}
 *       site[1] = xe  [4][n2  ][n1+1]  x-edge points U_{i+1/2,j}
 *       site[2] = ye  [4][n2+1][n1  ]  y-edge points U_{i,j+1/2}
 *       site[3] = vx  [4][n2+1][n1+1]  vertex points U_{i+1/2,j+1/2}
 *   1D: site[0] = avg [3][n1], site[1] = pt [3][n1+1]; site[2], site[3] unused.
 *   Components: (rho, rho u, [rho v,] E). Face index i of xe/vx/pt lies at
 *   x = lo[0] + i dx. On a periodic side the last face row/column duplicates
 *   the first: af_set_state requires them equal, af_get_state writes them equal.
 */
#ifndef AFNS_H
#define AFNS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct afns_ctx afns_ctx; /* opaque */

typedef enum {
    AF_OK = 0,
    AF_EINVAL = 1,  /* bad argument or inadmissible state (rho <= 0, p <= 0, NaN) */
    AF_ENOMEM = 2,  /* device or host allocation failed / workspace too small */
    AF_ECUDA = 3,   /* a CUDA call failed */
    AF_ENOTPP = 4,  /* max_halvings exceeded in the restart of Remark 3.2 */
    AF_ESTATE = 5   /* call out of order (e.g. step before set_state) */
} af_status;

typedef enum {
    AF_BC_PERIODIC = 0,
    AF_BC_WALL = 1,        /* no-slip adiabatic wall */
    AF_BC_SYMMETRY = 2,    /* slip wall / symmetry plane */
    AF_BC_TRANSMISSIVE = 3, /* zero-gradient outflow */
    AF_BC_EXACT = 4,        /* 1D: ghost data from the exact moving viscous shock of Sec. 4
                               (Becker's solution, parameters ex_M0 / ex_uinf of af_opts)
                               at each stage's time */
    AF_BC_MOVING_WALL = 5   /* 2D: no-slip adiabatic wall moving tangentially with speed
                               af_bc.wall_speed[side] (the lid of the Sec. 4 cavity): ghost
                               velocities mirror about the wall velocity, wall point values
                               take it after every stage */
} af_bc_kind;

typedef enum { AF_FP64 = 0, AF_MIXED = 1 } af_precision;
typedef enum { AF_LIM_NONE = 0, AF_LIM_PP = 1, AF_LIM_S_PP = 2 } af_limiter;
/* Manufactured source of the 2D Taylor-Green vortex (Sec. 4): with
 * a = exp(-2 mu t), b = cos 2x + cos 2y, rho = 1, (u, v) = a (sin x cos y,
 * -cos x sin y) and p = p0/(gamma-1) + a^2 b/4 solve Eqs. (1)-(3) plus the energy
 * source S_E = (p_t + u p_x + v p_y)/(gamma-1) - 4 mu a^2 cos^2 x cos^2 y
 * - kappa Lap p. Point values get S_E at the node and the stage time, cell
 * averages its 5 x 5 Gauss-Legendre cell average. 2D only. */
typedef enum { AF_SRC_NONE = 0, AF_SRC_TAYLOR_GREEN = 1 } af_source;

typedef struct {
    int dim;        /* 1 or 2 */
    int n[2];       /* cells per direction (n[1] ignored in 1D); each >= 4 */
    double lo[2];   /* domain [lo, hi] per direction */
    double hi[2];
} af_grid;

typedef struct {
    int side[4];    /* af_bc_kind of x-lo, x-hi, y-lo, y-hi; a periodic side needs a periodic partner */
    double wall_speed[4]; /* AF_BC_MOVING_WALL sides: tangential wall velocity (the x-velocity of
                             a y-side, the y-velocity of an x-side); ignored on other kinds */
} af_bc;

typedef struct {
    int precision;     /* af_precision (AF_MIXED: FP32 stencils, FP64 positivity islands) */
    int limiter;       /* af_limiter; AF_LIM_S_PP is the paper's scheme */
    double c_s;        /* smoothness-limiter strength C_s (Sec. 3.2); paper: 1 */
    double cfl_c;      /* inviscid CFL number C^c of Eq. (13); paper: 1.04/d */
    double cfl_v;      /* viscous CFL number C^v of Eq. (13); default 0.33 in 1D (the
                          paper's), 0.13 in 2D: the von Neumann limit of the 2D viscous
                          operator under SSP-RK54 is 0.1307 where heat conduction
                          dominates the bound, so the paper's 0.33/2 is unstable there */
    double eps;        /* positivity floor cap epsilon (Sec. 3.3); paper: 1e-13 */
    int max_halvings;  /* restarts allowed per step (Remark 3.2); default 30 */
    int tile_x;        /* 2D tile width in cells: 16 (default) or 32 (AF_MIXED only) */
    int tile_y;        /* 2D tile height in cells: 8 (default) or 16 */
    int source;        /* af_source: manufactured source term added to every stage */
    double src_p0;     /* p0 of the Taylor-Green source (paper: 100) */
    double ex_M0;      /* AF_BC_EXACT: upstream Mach number of the Becker shock (default 3) */
    double ex_uinf;    /* AF_BC_EXACT: translation velocity of the shock (default 0.2) */
    int threads;       /* threads per CTA of the 2D stage kernel: 128 (default) or 256 (a
                          32x16 tile always runs 512); af_tune may change tile_x / tile_y /
                          threads */
    int kappa_off;     /* 1: no heat conduction, kappa = 0 exactly (the Sec. 4 first problem
                          of Stokes), and no conduction term in the CFL bound of Eq. (13);
                          single-problem contexts (af_create); default 0 */
} af_opts;

/* Fill *o with the paper's defaults for a problem of dimension dim (except C^v
 * in 2D, see cfl_v). */
af_status af_opts_default(int dim, af_opts *o);

/* Bytes of device workspace af_create needs for this grid and these options. */
af_status af_workspace_bytes(const af_grid *grid, const af_opts *opts, size_t *bytes);

/*
 * Create a solver context.
 *  grid, bc: problem geometry (Sec. 2.1 / Sec. 2.2); gamma > 1, mu >= 0, Pr > 0.
 *  opts: NULL = af_opts_default(grid->dim).
 *  cuda_stream: a cudaStream_t (or NULL) on which all work is issued.
 *  workspace: device memory of at least af_workspace_bytes() bytes, 256-byte
 *    aligned, owned by the caller and kept alive until af_destroy; NULL lets the
 *    library allocate (and free) its own with cudaMalloc.
 */
af_status af_create(const af_grid *grid, double gamma, double mu, double Pr, const af_bc *bc,
                    const af_opts *opts, void *cuda_stream, void *workspace, size_t workspace_bytes,
                    afns_ctx **out);
af_status af_destroy(afns_ctx *ctx);

/*
 * Copy the DoFs in (layout above). on_device: 1 = the site pointers are device
 * memory, 0 = host memory. The library copies; the caller keeps ownership.
 * Validates that every DoF is finite with rho > 0 and p > 0 (Def. 3.1, the
 * method starts from G) and that periodic duplicates match (AF_EINVAL otherwise).
 */
af_status af_set_state(afns_ctx *ctx, const double *const site[4], int on_device, double t);
af_status af_get_state(afns_ctx *ctx, double *const site[4], int on_device, double *t);

/*
 * FP32 variants for AF_MIXED contexts (AF_EINVAL on an FP64 context): the same
 * site layout with float elements, copied straight into / out of the FP32 state,
 * half the bytes of the FP64 calls. af_set_state_f32 starts the compensation
 * words of the cell averages at zero and validates like af_set_state;
 * af_get_state_f32 returns every value rounded to FP32 (for a cell average, the
 * rounding of its compensated value hi + lo). Host arrays go through the
 * context's staging area as one contiguous copy per site; device arrays are read
 * or written in place. Both calls synchronise the context's stream.
 */
af_status af_set_state_f32(afns_ctx *ctx, const float *const site[4], int on_device, double t);
af_status af_get_state_f32(afns_ctx *ctx, float *const site[4], int on_device, double *t);

/* Largest stable step of Eq. (13) on the current cell averages. */
af_status af_dt_max(afns_ctx *ctx, double *dt);

/*
 * One SSP-RK54 step (Sec. 2.3) of size dt; dt <= 0 takes the CFL step of
 * Eq. (13). If a low-order state the limiters evaluate is not admissible, the
 * step is recomputed from the start with dt/2 (Remark 3.2), at most
 * max_halvings times (AF_ENOTPP, state left at the step's start).
 * *dt_taken (may be NULL) receives the accepted step, *halvings the restarts.
 */
af_status af_step(afns_ctx *ctx, double dt, double *dt_taken, int *halvings);

/* Advance to t_end with CFL steps (last step clipped); counts may be NULL. */
af_status af_advance(afns_ctx *ctx, double t_end, int *steps, int *restarts);

/*
 * The limited semi-discrete residual L(u) of every DoF for a forward-Euler
 * stage of size dt (dt enters the limiters through mu_l = dt/dx_l, Sec. 3), in
 * the DoF layout above. This is one RK stage's right-hand side, exported for
 * parity checks. *notpp (may be NULL) receives 1 when a low-order state was
 * inadmissible.
 */
af_status af_residual(afns_ctx *ctx, double dt, double *const L[4], int on_device, int *notpp);

/*
 * Per-face limiter values of the last af_residual call: theta_s (Sec. 3.2) and
 * theta^rho theta^p (Sec. 3.3). Layout: x-faces [n2][n1+1], then (2D) y-faces
 * [n2+1][n1]. Host pointers; either may be NULL.
 */
af_status af_get_limiter(afns_ctx *ctx, double *theta_s, double *theta_pp);

/*
 * Autotuner of the 2D stage kernel launch (tiles of 16x8, 16x16, 32x8 or 32x16
 * cells, 256 or 128 threads per CTA, 512 for 32x16; 32-wide tiles only in
 * AF_MIXED): times each candidate
 * on residual evaluations of the current state (the state is not changed) and
 * keeps the fastest for the following steps. Results do not depend on the
 * choice. Needs a state (AF_ESTATE otherwise). Outputs may be NULL.
 */
af_status af_tune(afns_ctx *ctx, int *tile_x, int *tile_y, int *threads);

/*
 * Test hook of the bounded tile-load wait (the paper has no counterpart). The 2D
 * stage kernel loads each tile with TMA copies that complete an mbarrier armed
 * with the copies' byte count; every thread waits on it for at most 2 s of the
 * GPU's global timer, after which the kernel flags the step and the call that
 * reads it (af_step, af_advance, af_residual, af_dt_max) returns AF_ECUDA with a
 * message, leaving the context usable. extra_bytes > 0 arms the barrier with that
 * many bytes more than the copies deliver, so every wait runs out; 0 restores
 * normal operation. extra_bytes must be a multiple of 16. Meant for tests on
 * small grids: each CTA then spends 2 s.
 */
af_status af_debug_tile_wait(afns_ctx *ctx, int extra_bytes);

/* Number of cells n1*n2 and of faces (sizes of the arrays above). */
af_status af_sizes(const afns_ctx *ctx, size_t *cells, size_t *faces, size_t *site_elems4);

/*
 * Profiling. af_set_profiling(ctx, 1) resets the counters and, from then on,
 * brackets every fused stage-kernel launch with CUDA events on the context's
 * stream; af_get_profile returns the summed stage-kernel time (ms, harvested at
 * each step's restart-flag read), the number of stage-kernel launches and the
 * number of all kernel launches issued by the library since the reset.
 * Not part of the method (no counterpart in the paper).
 */
af_status af_set_profiling(afns_ctx *ctx, int on);
af_status af_get_profile(afns_ctx *ctx, double *stage_ms, long long *stage_launches, long long *launches);

/* Description of the context's last failure; af_last_error(NULL) describes why
 * the calling thread's last af_create refused its arguments. */
const char *af_last_error(const afns_ctx *ctx);

/*
 * Allocation-free CFL step (the paper has no counterpart of this call).
 *
 * af_dt_max_noalloc computes the time step of Eq. (13) for a 2D FP64 state that
 * the caller already holds on the device, without allocating any device memory.
 * It serves callers that cannot call cudaMalloc: code whose device memory is all
 * owned by a host framework's pool allocator, or that runs where an allocation
 * (with the device-wide synchronisation it can imply) is not allowed.
 *  grid, gamma, mu, Pr: as for af_create (grid->dim must be 2).
 *  opts: NULL = af_opts_default(2); only cfl_c, cfl_v and kappa_off are used
 *    (kappa_off = 1 drops the conduction term from the bound, as af_create does).
 *  avg_dev: device pointer to the cell averages in the layout of site[0] of
 *    af_set_state, avg[4][n2][n1]; the caller owns it.
 *  dt_dev: device pointer that receives one double; the caller owns it. If any
 *    cell average is non-finite or has rho <= 0 or p <= 0 (outside the set where
 *    Eq. (13) is defined), *dt_dev receives NaN: the call does not wait for the
 *    GPU, so it cannot return AF_EINVAL for the values themselves.
 *  cuda_stream: the two kernels of the call are issued there, asynchronously;
 *    nothing is synchronised (read dt_dev after the stream has reached it).
 * Returns AF_EINVAL for a bad argument or an oversized grid (nothing launched),
 * AF_ECUDA if the address lookup or a launch of this call failed.
 * Scratch: one file-scope device array inside the library, two doubles per chunk
 * of AF_NOALLOC_CHUNK cells for at most AF_NOALLOC_MAX_CHUNKS chunks (256 KiB).
 * Every GPU that loads the library holds it until the process exits. Grids with
 * more than AF_NOALLOC_CHUNK * AF_NOALLOC_MAX_CHUNKS cells (67,108,864) are
 * rejected with AF_EINVAL before anything is launched. The first call on a device
 * (and the first after the device's context was reset) looks up the array's
 * device address for that device and context; make that first call before any
 * stream capture. Every call writes each slot it later reads, so nothing needs
 * clearing between calls; but all calls share the one array, so calls that
 * overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.
 */
/*
 * Measured FMA throughput of the current device (the paper has no counterpart):
 * the ALU roofline denominator of the stage kernels. precision AF_MIXED times
 * FP32 FMA chains, AF_FP64 FP64 FMA chains (8 independent chains per thread,
 * 8 CTAs of 256 threads per SM, one warm-up launch, then one launch timed with
 * CUDA events on a stream of its own). *tflops receives 2 x FMAs / second / 1e12.
 * Allocates and frees a small device buffer; synchronises its own stream.
 * Returns AF_EINVAL for a bad argument, AF_ECUDA if a CUDA call failed.
 */
af_status af_alu_peak(int precision, double *tflops);

#define AF_NOALLOC_CHUNK 4096
#define AF_NOALLOC_MAX_CHUNKS 16384
af_status af_dt_max_noalloc(const af_grid *grid, double gamma, double mu, double Pr, const af_opts *opts,
                            const double *avg_dev, double *dt_dev, void *cuda_stream);

/* ------------------------------------------------------------------------- */
/* Batched problems: many independent 2D problems of uneven grid sizes and     */
/* gas parameters advanced together, one persistent stage kernel per RK stage  */
/* over a (problem, tile) work list. Every problem keeps its own CFL step      */
/* (Eq. (13)) and its own restart (Remark 3.2): a rejected step keeps u^n and  */
/* is recomputed with dt/2 in the next batch step while the other problems     */
/* move on. A batch step never waits for the host, so it is captured once in a */
/* CUDA graph and replayed. Problems are 2D; precision and limiter come from    */
/* opts (NULL = paper defaults with AF_MIXED); no manufactured source.          */
/* ------------------------------------------------------------------------- */
typedef struct afb_ctx afb_ctx;

af_status afb_workspace_bytes(int nprob, const af_grid *grids, const af_opts *opts, size_t *bytes);
/* grids, gamma, mu, Pr, bcs: arrays of nprob entries. Workspace as in af_create. */
af_status afb_create(int nprob, const af_grid *grids, const double *gamma, const double *mu, const double *Pr,
                     const af_bc *bcs, const af_opts *opts, void *cuda_stream, void *workspace,
                     size_t workspace_bytes, afb_ctx **out);
af_status afb_destroy(afb_ctx *ctx);
/* Per-problem state in the 2D site layout of af_set_state (validated likewise). */
af_status afb_set_state(afb_ctx *ctx, int i, const double *const site[4], int on_device, double t);
af_status afb_get_state(afb_ctx *ctx, int i, double *const site[4], int on_device, double *t);
/* Autotuner: times the candidate tile shapes, CTA sizes and work-list orders on
 * the current states (restored afterwards) and keeps the fastest. */
af_status afb_tune(afb_ctx *ctx, int *tile_x, int *tile_y, int *threads, int *schedule);
/* Issue nsteps batch steps (asynchronous; use_graph = replay the captured step). */
af_status afb_step_all(afb_ctx *ctx, int nsteps, int use_graph);
/* Per-problem counters: accepted steps, rejected (restarted) steps, failure flag, time. */
af_status afb_stats(afb_ctx *ctx, int i, int *accepted, int *restarts, int *failed, double *t);
/* Wait for the batch; *launches_per_step = kernels issued per batch step. */
af_status afb_sync(afb_ctx *ctx, long long *launches_per_step);
const char *afb_last_error(const afb_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
