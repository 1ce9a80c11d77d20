/*
 * afns_oracle.h -- plain, slow, scalar FP64 CPU oracle of the compact fourth-order
 * positivity-preserving active flux (AF) method for the 1D/2D compressible
 * Navier-Stokes equations (Duan, Barsukow, Klingenberg, arXiv 2609.29081).
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference leg of bench.py may load this library. It shares no code, header,
 * table or helper with the CUDA library (libafns); neither includes the other.
 *
 * Packed state layout (conservative variables, component-major, row-major with
 * the x index fastest):
 *   2D (4 components rho, rho*u, rho*v, E):
 *     avg  [4][n2  ][n1  ]   cell averages                      (Sec. 2.2)
 *     xe   [4][n2  ][n1+1]   x-edge point values U_{i+1/2,j}    (Sec. 2.2)
 *     ye   [4][n2+1][n1  ]   y-edge point values U_{i,j+1/2}
 *     vx   [4][n2+1][n1+1]   vertex point values U_{i+1/2,j+1/2}
 *   1D (3 components rho, rho*u, E):
 *     avg  [3][n1], pt [3][n1+1]                                 (Sec. 2.1)
 *   Index i of xe/vx is the face at x = lo1 + i*dx; index j of ye/vx is the face
 *   at y = lo2 + j*dy. On periodic sides the last face duplicates the first.
 *
 * Per-face limiter outputs (theta_s, theta_pp = theta^rho*theta^p) are packed as
 *   x-faces [n2][n1+1] then (2D only) y-faces [n2+1][n1].
 */
#ifndef AFNS_ORACLE_H
#define AFNS_ORACLE_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_BC_PERIODIC 0
#define ORC_BC_WALL 1          /* no-slip adiabatic wall */
#define ORC_BC_SYMMETRY 2      /* slip (reflective) wall */
#define ORC_BC_TRANSMISSIVE 3  /* zero-gradient outflow */

#define ORC_LIM_NONE 0  /* pure high-order fluxes, no point limiter */
#define ORC_LIM_PP 1    /* positivity limiting only (theta_s = 1) */
#define ORC_LIM_S_PP 2  /* smoothness indicator, then positivity limiting */

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOTPP 4

typedef struct {
    int dim;            /* 1 or 2 */
    int n1, n2;         /* cells per direction; n2 is ignored in 1D */
    double lo1, hi1, lo2, hi2;
    double gamma, mu, Pr;
    int bc[4];          /* x-lo, x-hi, y-lo, y-hi (ORC_BC_*) */
    int limiter;        /* ORC_LIM_* */
    double c_s;         /* smoothness limiter strength C_s */
    double cfl_c;       /* inviscid CFL number C^c */
    double cfl_v;       /* viscous CFL number C^v */
    double eps;         /* cap of the positivity floors epsilon (1e-13 in Sec. 3.3) */
    int source;         /* ORC_SRC_*: manufactured source term added to L */
    double src_p0;      /* p0 of the Taylor-Green source (Sec. 4: 100) */
    double time;        /* time of the state given to orc_residual / orc_step */
    double ex_M0;       /* Becker shock (ORC_BC_EXACT sides): upstream Mach number M0 */
    double ex_uinf;     /* Becker shock: translation velocity u_inf */
    double wall_speed[4]; /* ORC_BC_MOVING sides: tangential wall velocity (x-velocity of a
                             y-side, y-velocity of an x-side) */
} orc_problem;

#define ORC_BC_EXACT 4  /* 1D: ghost cells and points from the exact Becker shock at the stage time */
#define ORC_BC_MOVING 5 /* 2D: no-slip adiabatic wall moving tangentially with wall_speed[side] */

#define ORC_SRC_NONE 0
#define ORC_SRC_TAYLOR_GREEN 1  /* energy source of the 2D manufactured Taylor-Green vortex (Sec. 4) */

/* Fill the paper's defaults for everything but the grid, gas and BCs. */
void orc_defaults(orc_problem *P);

size_t orc_state_len(const orc_problem *P);
size_t orc_face_len(const orc_problem *P);

/* L(u): limited semi-discrete residual of every DoF (same packed layout as the
 * state) for one forward-Euler stage of size dt (dt enters the limiter through
 * mu_l = dt/dx_l, Sec. 3). theta_s / theta_pp may be NULL. *notpp is set to 1 when
 * a low-order state the limiter evaluates lies outside G (Remark 3.2). */
int orc_residual(const orc_problem *P, const double *state, double dt, double *L,
                 double *theta_s, double *theta_pp, int *notpp);

/* CFL time step of Eq. (13) on the cell averages. */
double orc_dt_max(const orc_problem *P, const double *state);

/* Low-order point update (Sec. 3.4, reading R7) of lattice node (a0, a1) (a1 = 0
 * in 1D; even lattice indices are point nodes), as the limiter would form it for
 * step dt; UL receives dim + 2 conservative values. */
void orc_point_low_order(const orc_problem *P, const double *state, double dt, int a0, int a1, double *UL);

/* Low-order LLF total flux of Eq. (19) of face (f0, f1) in direction l, the face
 * between cells f - e_l and f (f1 = 0 in 1D); FL receives dim + 2 values. */
void orc_face_low_order(const orc_problem *P, const double *state, int l, int f0, int f1, double *FL);

/* One SSP-RK54 step of size dt with the halving restart of Remark 3.2. */
int orc_step(const orc_problem *P, double *state, double dt, int max_halvings,
             double *dt_taken, int *halvings);

/* Advance from t to t_end with CFL steps; the last step is clipped to t_end. */
int orc_advance(const orc_problem *P, double *state, double t, double t_end,
                int max_halvings, int max_steps, int *steps, int *restarts);

/* Building blocks, exported for the unit pins in tests/. */
void orc_rk_table(double alpha[5][5], double beta[5][5]);
void orc_op_dplus(const double *z5, double dx, double *out);
void orc_op_dminus(const double *z5, double dx, double *out);
void orc_op_dcentral(const double *z5, double dx, double *out);
void orc_op_bmatrix(double *b25);
/* D^2(K,Z) for scalar K and Z on the 5 lattice nodes a-2..a+2 (Eq. 9). */
void orc_op_d2_scalar(const double *k5, const double *z5, double dx, double *out);
/* Physics of one state (dim 1: 3 comps, dim 2: 4 comps). grad = dZ/dx_l, l-major. */
void orc_inviscid_flux(const orc_problem *P, const double *U, int l, double *F);
void orc_viscous_flux(const orc_problem *P, const double *U, const double *grad, int l, double *F);
double orc_visc_bound(const orc_problem *P, const double *U, const double *grad, int l);
double orc_pressure(const orc_problem *P, const double *U);
double orc_wave_speed(const orc_problem *P, const double *U, int l);
double orc_theta(double zL, double zH, double eps);

#ifdef __cplusplus
}
#endif
#endif
