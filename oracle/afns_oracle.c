/*
 * afns_oracle.c -- plain, slow, scalar FP64 CPU oracle of the compact fourth-order
 * positivity-preserving active flux (AF) method for compressible Navier-Stokes
 * (Duan, Barsukow, Klingenberg, arXiv 2609.29081).
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference leg of bench.py may load this code. It shares nothing with libafns.
 *
 * The code follows the paper's steps in the paper's order and notation, written
 * for a reader checking it against the paper, not for speed: every quantity is
 * evaluated on a "half lattice" of spacing dx_l/2 that holds the point values
 * (even indices) and the reconstructed cell centres (odd indices), so each
 * operator of Sec. 2 is a 5-node stencil along one lattice line.
 *
 * Readings of points the paper leaves open (each is also listed in the design
 * notes of the repository):
 *  R1  SSP-RK54 (Sec. 2.3) uses the Spiteri-Ruuth SSPRK(5,4) Shu-Osher coefficients.
 *  R2  The limiter of every RK stage uses the full step dt in mu_l = dt/dx_l.
 *  R3  The 2D FVS viscosity alpha at node zeta in direction l is the maximum of
 *      rho_l = |u_l| + c over the 5 lattice nodes of the l-line through zeta.
 *  R4  The tangential gradient in F^v at edge/vertex nodes is D_c along the
 *      lattice line through the node.
 *  R5  S_i (Sec. 3.1) is the second-order central difference of Z(U-bar) in every
 *      direction; the Ducros div/curl use the same differences of u-bar.
 *  R6  epsilon = min(1e-13, z^L) per state; the cell-centre scaling limiter
 *      (Remark 3.1) blends toward the cell average by Theta on rho, then on p.
 *  R7  The low-order point update (Sec. 3.4) is first-order LLF on the half
 *      lattice (spacing dx_l/2) with the total flux of Eq. (19) between lattice
 *      neighbours and S from central differences on the lattice; it is evaluated
 *      only where the high-order point update leaves G_eps.
 *  R8  Restart (Remark 3.2) when any evaluated low-order state has rho <= 0,
 *      p <= 0 or is not finite.
 *  R9  Ghost layers: periodic wrap; walls mirror about the boundary node with the
 *      momentum signs flipped (no-slip: both, symmetry: normal), transmissive is
 *      the unflipped mirror. After every RK stage the wall point values get zero
 *      (normal) momentum with their internal energy kept.
 *  R15 Exact boundary data (1D viscous shock, Sec. 4): the ghost cell averages
 *      (5-point Gauss-Legendre) and ghost point values come from the exact Becker
 *      solution at the stage's time; the boundary point values themselves evolve
 *      with the scheme like every other point.
 *  R14 CFL numbers of Eq. (13): C^c = 1.04/d as printed; C^v = 0.33 in 1D as
 *      printed, but 0.13 in 2D. The von Neumann limit of the 2D viscous
 *      operator of Eq. (12) under SSP-RK54 is 0.1307 where heat conduction
 *      dominates the bound (its largest eigenvalue is 40.8 / dx^2 against
 *      2 x 16 / dx^2 for two 1D operators: the Simpson centres and edge
 *      averages couple the directions), so the printed 0.33/2 lets such flows
 *      grow a high-frequency mode. The 1D limit of 0.333 is the printed one
 *      (both pinned in the tests).
 */
#include "afns_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXC 4 /* at most 4 conservative components (2D) */

/* Operation-count hooks. Here they do nothing. The op-counting build
 * (opcount.cpp, the same source compiled as C++ with a counting scalar type)
 * defines ORC_PHASE(k) to attribute the operations that follow to step k of a
 * stage, and ORC_PURE(id, a, na, b, nb, i, j) to mark the rest of a function as
 * a pure evaluation keyed by its inputs (arrays a[na], b[nb], integers i, j),
 * so that a repeated evaluation with the same inputs is counted apart. */
#ifndef ORC_PHASE
#define ORC_PHASE(k) ((void)0)
#endif
#ifndef ORC_PURE
#define ORC_PURE(id, a, na, b, nb, i, j) ((void)0)
#endif

/* ------------------------------------------------------------------------- */
/* Physics: Sec. 1 Eqs. (1)-(3), Sec. 2.1 Eqs. (4)-(5), Sec. 2.2 K matrices.   */
/* Component layout: U = (rho, rho*u_1..rho*u_d, E).                          */
/* ------------------------------------------------------------------------- */

static double kappa_of(const orc_problem *P)
{
    /* Sec. 1: kappa = gamma*mu / ((gamma-1) Pr) */
    return P->gamma * P->mu / ((P->gamma - 1.0) * P->Pr);
}

double orc_pressure(const orc_problem *P, const double *U)
{
    ORC_PURE(1, U, P->dim + 2, (const double *)0, 0, 0, 0);
    /* Def. 3.1, Eq. (14): p = (gamma-1) (E - |rho u|^2 / (2 rho)) */
    int d = P->dim;
    double m2 = 0.0;
    for (int k = 0; k < d; ++k) m2 += U[1 + k] * U[1 + k];
    return (P->gamma - 1.0) * (U[d + 1] - m2 / (2.0 * U[0]));
}

/* W = (rho, u_1..u_d, p) (Eq. (5) and Sec. 2.2) */
static void primitive(const orc_problem *P, const double *U, double *W)
{
    ORC_PURE(2, U, P->dim + 2, (const double *)0, 0, 0, 0);
    int d = P->dim;
    W[0] = U[0];
    for (int k = 0; k < d; ++k) W[1 + k] = U[1 + k] / U[0];
    W[d + 1] = orc_pressure(P, U);
}

/* Z = (0, u_1..u_d, T) with T = p/rho (Eq. (5), Sec. 1 nondimensional form) */
static void zvars(const orc_problem *P, const double *W, double *Z)
{
    ORC_PURE(3, W, P->dim + 2, (const double *)0, 0, 0, 0);
    int d = P->dim;
    Z[0] = 0.0;
    for (int k = 0; k < d; ++k) Z[1 + k] = W[1 + k];
    Z[d + 1] = W[d + 1] / W[0];
}

void orc_inviscid_flux(const orc_problem *P, const double *U, int l, double *F)
{
    ORC_PURE(4, U, P->dim + 2, (const double *)0, 0, l, 0);
    /* Eq. (2): F^c_l = (rho u_l, rho u u_l + p e_l, (E + p) u_l) */
    int d = P->dim;
    double W[MAXC];
    primitive(P, U, W);
    double ul = W[1 + l], p = W[d + 1];
    F[0] = U[0] * ul;
    for (int k = 0; k < d; ++k) F[1 + k] = U[1 + k] * ul + (k == l ? p : 0.0);
    F[d + 1] = (U[d + 1] + p) * ul;
}

/* K_lm(W) of Sec. 2.1 (1D, 3x3) and Sec. 2.2 (2D, four 4x4 matrices). */
static void kmatrix(const orc_problem *P, const double *W, int l, int m, double K[MAXC][MAXC])
{
    double mu = P->mu, ka = kappa_of(P);
    for (int r = 0; r < MAXC; ++r)
        for (int c = 0; c < MAXC; ++c) K[r][c] = 0.0;
    if (P->dim == 1) {
        double u = W[1];
        K[1][1] = 4.0 / 3.0 * mu;
        K[2][1] = 4.0 / 3.0 * mu * u;
        K[2][2] = ka;
        return;
    }
    double u = W[1], v = W[2];
    if (l == 0 && m == 0) {
        K[1][1] = 4.0 / 3.0 * mu;
        K[2][2] = mu;
        K[3][1] = 4.0 / 3.0 * mu * u;
        K[3][2] = mu * v;
        K[3][3] = ka;
    } else if (l == 1 && m == 1) {
        K[1][1] = mu;
        K[2][2] = 4.0 / 3.0 * mu;
        K[3][1] = mu * u;
        K[3][2] = 4.0 / 3.0 * mu * v;
        K[3][3] = ka;
    } else if (l == 0 && m == 1) {
        K[1][2] = -2.0 / 3.0 * mu;
        K[2][1] = mu;
        K[3][1] = mu * v;
        K[3][2] = -2.0 / 3.0 * mu * u;
    } else { /* l == 1 && m == 0 */
        K[1][2] = mu;
        K[2][1] = -2.0 / 3.0 * mu;
        K[3][1] = -2.0 / 3.0 * mu * v;
        K[3][2] = mu * u;
    }
}

/* out = K_lm(W) z (matrix-vector product, nc components) */
static void kapply(const orc_problem *P, const double *W, int l, int m, const double *z, double *out)
{
    ORC_PURE(5, W, P->dim + 2, z, P->dim + 2, l, m);
    double K[MAXC][MAXC];
    int nc = P->dim + 2;
    kmatrix(P, W, l, m, K);
    for (int r = 0; r < nc; ++r) {
        double s = 0.0;
        for (int c = 0; c < nc; ++c) s += K[r][c] * z[c];
        out[r] = s;
    }
}

void orc_viscous_flux(const orc_problem *P, const double *U, const double *grad, int l, double *F)
{
    ORC_PURE(6, U, P->dim + 2, grad, P->dim * (P->dim + 2), l, 0);
    /* Sec. 2.2: F^v_l = sum_m K_lm(W) dZ/dx_m (Sec. 2.1 in 1D: K(W) Z_x) */
    int nc = P->dim + 2;
    double W[MAXC], t[MAXC];
    primitive(P, U, W);
    for (int r = 0; r < nc; ++r) F[r] = 0.0;
    for (int m = 0; m < P->dim; ++m) {
        kapply(P, W, l, m, grad + m * nc, t);
        for (int r = 0; r < nc; ++r) F[r] += t[r];
    }
}

double orc_wave_speed(const orc_problem *P, const double *U, int l)
{
    ORC_PURE(7, U, P->dim + 2, (const double *)0, 0, l, 0);
    /* Lemma 3.1 / Sec. 2.3: rho_l = |u_l| + c, c = sqrt(gamma p / rho) */
    double W[MAXC];
    primitive(P, U, W);
    double c = sqrt(P->gamma * W[P->dim + 1] / W[0]);
    return fabs(W[1 + l]) + c;
}

static double visc_eigen(const orc_problem *P, const double *U)
{
    /* Sec. 2.3: rho~ = max{4 mu / (3 rho), gamma mu / (Pr rho)} */
    double a = 4.0 * P->mu / (3.0 * U[0]);
    double b = P->gamma * P->mu / (P->Pr * U[0]);
    return a > b ? a : b;
}

double orc_visc_bound(const orc_problem *P, const double *U, const double *grad, int l)
{
    ORC_PURE(8, U, P->dim + 2, grad, P->dim * (P->dim + 2), l, 0);
    /* Lemma 3.2: b_l = (sqrt(rho^2 q_l^2 + 2 rho^2 e |tau_l|^2) + rho |q_l|) / (2 rho^2 e),
     * with tau from Eq. (3) and q = -kappa grad T.  grad[m*nc + k] = d Z_k / d x_m. */
    int d = P->dim, nc = d + 2;
    double W[MAXC];
    primitive(P, U, W);
    double rho = W[0], p = W[d + 1];
    double e = p / ((P->gamma - 1.0) * rho);
    double divu = 0.0;
    for (int m = 0; m < d; ++m) divu += grad[m * nc + 1 + m];
    /* tau_l = tau e_l, components k: tau_{k l} = mu (d_l u_k + d_k u_l - 2/3 div u delta_kl) */
    double tau2 = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = P->mu * (grad[l * nc + 1 + k] + grad[k * nc + 1 + l] - (k == l ? 2.0 / 3.0 * divu : 0.0));
        tau2 += t * t;
    }
    double q = -kappa_of(P) * grad[l * nc + d + 1];
    return (sqrt(rho * rho * q * q + 2.0 * rho * rho * e * tau2) + rho * fabs(q)) / (2.0 * rho * rho * e);
}

/* Admissible set G of Def. 3.1 (finite, rho > 0, p > 0). */
static int in_G(const orc_problem *P, const double *U)
{
    int nc = P->dim + 2;
    for (int c = 0; c < nc; ++c)
        if (!isfinite(U[c])) return 0;
    if (!(U[0] > 0.0)) return 0;
    double p = orc_pressure(P, U);
    return isfinite(p) && p > 0.0;
}

/* Sec. 3.3: Theta(zL, zH, eps) = (zL - eps)/(zL - zH) if zH < eps, else 1 */
double orc_theta(double zL, double zH, double eps)
{
    if (zH < eps) return (zL - eps) / (zL - zH);
    return 1.0;
}

/* ------------------------------------------------------------------------- */
/* Difference operators of Sec. 2.1 on 5 lattice values z[0..4] = nodes      */
/* a-2..a+2 of one lattice line (lattice spacing dx/2).                      */
/* ------------------------------------------------------------------------- */

void orc_op_dplus(const double *z, double dx, double *out)
{
    /* Eq. (7a) */
    *out = (z[0] - 6.0 * z[1] + 3.0 * z[2] + 2.0 * z[3]) / (3.0 * dx);
}

void orc_op_dminus(const double *z, double dx, double *out)
{
    /* Eq. (7b) */
    *out = (-2.0 * z[1] - 3.0 * z[2] + 6.0 * z[3] - z[4]) / (3.0 * dx);
}

void orc_op_dcentral(const double *z, double dx, double *out)
{
    /* Eq. (8) */
    *out = (z[0] - 8.0 * z[1] + 8.0 * z[3] - z[4]) / (6.0 * dx);
}

void orc_op_bmatrix(double *b)
{
    /* Eq. (10): B = [[0,0],[0,M]] - [[M,0],[0,0]], rows/columns ordered -2..2 */
    static const double M[4][4] = {
        {1.0 / 8.0, -1.0 / 6.0, 1.0 / 24.0, 0.0},
        {-1.0 / 6.0, -3.0 / 8.0, 2.0 / 3.0, -1.0 / 8.0},
        {1.0 / 8.0, -2.0 / 3.0, 3.0 / 8.0, 1.0 / 6.0},
        {0.0, -1.0 / 24.0, 1.0 / 6.0, -1.0 / 8.0},
    };
    for (int r = 0; r < 5; ++r)
        for (int c = 0; c < 5; ++c) {
            double v = 0.0;
            if (r >= 1 && c >= 1) v += M[r - 1][c - 1];
            if (r <= 3 && c <= 3) v -= M[r][c];
            b[r * 5 + c] = v;
        }
}

void orc_op_d2_scalar(const double *k5, const double *z5, double dx, double *out)
{
    /* Eq. (9) with scalar K: (4/dx^2) sum_{m,n} b_mn K_{a+m} Z_{a+n} */
    double b[25], s = 0.0;
    orc_op_bmatrix(b);
    for (int m = 0; m < 5; ++m)
        for (int n = 0; n < 5; ++n) s += b[m * 5 + n] * k5[m] * z5[n];
    *out = 4.0 / (dx * dx) * s;
}

/* ------------------------------------------------------------------------- */
/* SSP-RK54 (Sec. 2.3), Shu-Osher form u(i) = sum_k alpha_ik u(k) +           */
/* beta_ik dt L(u(k)), u(0) = u^n, u(5) = u^{n+1}. Reading R1.               */
/* ------------------------------------------------------------------------- */

void orc_rk_table(double a[5][5], double b[5][5])
{
    memset(a, 0, sizeof(double) * 25);
    memset(b, 0, sizeof(double) * 25);
    a[0][0] = 1.0;
    b[0][0] = 0.391752226571890;
    a[1][0] = 0.444370493651235;
    a[1][1] = 0.555629506348765;
    b[1][1] = 0.368410593050371;
    a[2][0] = 0.620101851488403;
    a[2][2] = 0.379898148511597;
    b[2][2] = 0.251891774271694;
    a[3][0] = 0.178079954393132;
    a[3][3] = 0.821920045606868;
    b[3][3] = 0.544974750228521;
    a[4][2] = 0.517231671970585;
    a[4][3] = 0.096059710526147;
    b[4][3] = 0.063692468666290;
    a[4][4] = 0.386708617503269;
    b[4][4] = 0.226007483236906;
}

/* ------------------------------------------------------------------------- */
/* Grid: half lattice with 2 ghost nodes and cell averages with 2 ghost cells */
/* ------------------------------------------------------------------------- */

typedef struct {
    const orc_problem *P;
    int d, nc;
    int n[2];
    double h[2];   /* dx_l */
    int na[2];     /* lattice extents (2n+5 used, 1 unused) */
    int nca[2];    /* cell extents (n+4 used, 1 unused) */
    int off[2];    /* ghost depth per direction (2 used, 0 unused) */
    double *U;     /* [nc][na1][na0]: point values and reconstructed centres */
    double *W;     /* primitive variables at lattice nodes */
    double *Z;     /* Z variables at lattice nodes */
    double *A;     /* [nc][nca1][nca0]: cell averages */
} grid_t;

static size_t lat_idx(const grid_t *g, int c, int a0, int a1)
{
    return ((size_t)c * g->na[1] + (size_t)(a1 + g->off[1])) * g->na[0] + (size_t)(a0 + g->off[0]);
}

static size_t cell_idx(const grid_t *g, int c, int i0, int i1)
{
    return ((size_t)c * g->nca[1] + (size_t)(i1 + g->off[1])) * g->nca[0] + (size_t)(i0 + g->off[0]);
}

static void lat_get(const grid_t *g, const double *arr, int a0, int a1, double *v)
{
    for (int c = 0; c < g->nc; ++c) v[c] = arr[lat_idx(g, c, a0, a1)];
}

static void lat_set(grid_t *g, double *arr, int a0, int a1, const double *v)
{
    for (int c = 0; c < g->nc; ++c) arr[lat_idx(g, c, a0, a1)] = v[c];
}

static void cell_get(const grid_t *g, int i0, int i1, double *v)
{
    for (int c = 0; c < g->nc; ++c) v[c] = g->A[cell_idx(g, c, i0, i1)];
}

static void cell_set(grid_t *g, int i0, int i1, const double *v)
{
    for (int c = 0; c < g->nc; ++c) g->A[cell_idx(g, c, i0, i1)] = v[c];
}

static int is_centre(const grid_t *g, int a0, int a1)
{
    if (g->d == 1) return (a0 & 1) != 0;
    return (a0 & 1) && (a1 & 1);
}

static void grid_init(grid_t *g, const orc_problem *P)
{
    memset(g, 0, sizeof(*g));
    g->P = P;
    g->d = P->dim;
    g->nc = P->dim + 2;
    g->n[0] = P->n1;
    g->n[1] = P->dim == 2 ? P->n2 : 1;
    g->h[0] = (P->hi1 - P->lo1) / P->n1;
    g->h[1] = P->dim == 2 ? (P->hi2 - P->lo2) / P->n2 : 1.0;
    for (int l = 0; l < 2; ++l) {
        int used = l < g->d;
        g->off[l] = used ? 2 : 0;
        g->na[l] = used ? 2 * g->n[l] + 5 : 1;
        g->nca[l] = used ? g->n[l] + 4 : 1;
    }
    size_t nl = (size_t)g->nc * g->na[0] * g->na[1];
    size_t ncl = (size_t)g->nc * g->nca[0] * g->nca[1];
    g->U = (double *)calloc(nl, sizeof(double));
    g->W = (double *)calloc(nl, sizeof(double));
    g->Z = (double *)calloc(nl, sizeof(double));
    g->A = (double *)calloc(ncl, sizeof(double));
}

static void grid_free(grid_t *g)
{
    free(g->U);
    free(g->W);
    free(g->Z);
    free(g->A);
}

/* ------------------------------------------------------------------------- */
/* Packed public layout <-> grid                                             */
/* ------------------------------------------------------------------------- */

size_t orc_state_len(const orc_problem *P)
{
    size_t n1 = P->n1;
    if (P->dim == 1) return 3 * (n1 + n1 + 1);
    size_t n2 = P->n2;
    return 4 * (n1 * n2 + (n1 + 1) * n2 + n1 * (n2 + 1) + (n1 + 1) * (n2 + 1));
}

size_t orc_face_len(const orc_problem *P)
{
    size_t n1 = P->n1;
    if (P->dim == 1) return n1 + 1;
    size_t n2 = P->n2;
    return (n1 + 1) * n2 + n1 * (n2 + 1);
}

/* Offset of point node (a0,a1) (not a centre) in the packed array, component c. */
static size_t packed_point(const orc_problem *P, int c, int a0, int a1)
{
    size_t n1 = P->n1;
    if (P->dim == 1) return 3 * n1 + (size_t)c * (n1 + 1) + (size_t)(a0 / 2);
    size_t n2 = P->n2;
    size_t o_xe = 4 * n1 * n2;
    size_t o_ye = o_xe + 4 * (n1 + 1) * n2;
    size_t o_vx = o_ye + 4 * n1 * (n2 + 1);
    int e0 = (a0 & 1) == 0, e1 = (a1 & 1) == 0;
    if (e0 && !e1) return o_xe + ((size_t)c * n2 + (size_t)(a1 / 2)) * (n1 + 1) + (size_t)(a0 / 2);
    if (!e0 && e1) return o_ye + ((size_t)c * (n2 + 1) + (size_t)(a1 / 2)) * n1 + (size_t)(a0 / 2);
    return o_vx + ((size_t)c * (n2 + 1) + (size_t)(a1 / 2)) * (n1 + 1) + (size_t)(a0 / 2);
}

static size_t packed_cell(const orc_problem *P, int c, int i0, int i1)
{
    size_t n1 = P->n1;
    if (P->dim == 1) return (size_t)c * n1 + (size_t)i0;
    return ((size_t)c * P->n2 + (size_t)i1) * n1 + (size_t)i0;
}

/* Loop helpers over the interior DoFs: points a_l in [0, 2 n_l], cells i_l in [0, n_l). */
static int amax(const grid_t *g, int l) { return l < g->d ? 2 * g->n[l] : 0; }
static int imax(const grid_t *g, int l) { return l < g->d ? g->n[l] : 1; }

static void unpack(grid_t *g, const double *s)
{
    const orc_problem *P = g->P;
    for (int i1 = 0; i1 < imax(g, 1); ++i1)
        for (int i0 = 0; i0 < imax(g, 0); ++i0)
            for (int c = 0; c < g->nc; ++c) g->A[cell_idx(g, c, i0, i1)] = s[packed_cell(P, c, i0, i1)];
    for (int a1 = 0; a1 <= amax(g, 1); ++a1)
        for (int a0 = 0; a0 <= amax(g, 0); ++a0) {
            if (is_centre(g, a0, a1)) continue;
            for (int c = 0; c < g->nc; ++c) g->U[lat_idx(g, c, a0, a1)] = s[packed_point(P, c, a0, a1)];
        }
}

/* ------------------------------------------------------------------------- */
/* Boundary conditions (reading R9)                                          */
/* ------------------------------------------------------------------------- */

/* Lattice coordinate of the interior image of a (possibly ghost) coordinate a
 * in direction l; *sgn receives the momentum signs of the mirror. */
static int image(const grid_t *g, int l, int a, double *sgn)
{
    const orc_problem *P = g->P;
    int n2x = 2 * g->n[l];
    for (int c = 0; c < g->nc; ++c) sgn[c] = 1.0;
    int side;
    if (a < 0)
        side = 2 * l;
    else if (a > n2x)
        side = 2 * l + 1;
    else
        return a;
    int kind = P->bc[side];
    if (kind == ORC_BC_PERIODIC) return ((a % n2x) + n2x) % n2x;
    if (kind == ORC_BC_WALL || kind == ORC_BC_MOVING)
        for (int k = 0; k < g->d; ++k) sgn[1 + k] = -1.0;
    if (kind == ORC_BC_SYMMETRY) sgn[1 + l] = -1.0;
    return side & 1 ? 2 * n2x - a : -a;
}

/* Reading R17: a moving no-slip wall mirrors the velocity about the wall velocity,
 * u_ghost = 2 U_w - u_image (tangential), -u_image (normal), with the internal
 * energy of the image kept; v holds the image state with both momenta already
 * negated by image(). Applied to point values and cell averages alike. */
static void moving_wall_ghost(const grid_t *g, int l, int a, double *v)
{
    const orc_problem *P = g->P;
    if (g->d != 2 || (a >= 0 && a <= 2 * g->n[l])) return;
    int side = a < 0 ? 2 * l : 2 * l + 1;
    if (P->bc[side] != ORC_BC_MOVING) return;
    int t = 1 + (1 - l);  /* tangential momentum component */
    double m2_old = v[1] * v[1] + v[2] * v[2];
    v[t] += 2.0 * v[0] * P->wall_speed[side];
    double m2_new = v[1] * v[1] + v[2] * v[2];
    v[3] += (m2_new - m2_old) / (2.0 * v[0]);
}

static void fill_ghosts(grid_t *g)
{
    double v[MAXC], sg[MAXC];
    int lo[2], hi[2];
    for (int l = 0; l < 2; ++l) {
        lo[l] = l < g->d ? -2 : 0;
        hi[l] = l < g->d ? 2 * g->n[l] + 2 : 0;
    }
    /* direction 0 first on interior rows, then direction 1 on all columns. */
    for (int l = 0; l < g->d; ++l) {
        int per = g->P->bc[2 * l] == ORC_BC_PERIODIC;
        /* point nodes */
        int mlo = (l == 0) ? 0 : lo[0], mhi = (l == 0) ? amax(g, 1) : hi[0];
        if (g->d == 1) mlo = mhi = 0;
        for (int am = mlo; am <= mhi; ++am)
            for (int al = lo[l]; al <= hi[l]; ++al) {
                int ghost = al < 0 || al > 2 * g->n[l] || (per && al == 2 * g->n[l]);
                if (!ghost) continue;
                int a0 = l == 0 ? al : am, a1 = l == 0 ? am : al;
                if (is_centre(g, a0, a1)) continue;
                int src = image(g, l, al, sg);
                if (per && al == 2 * g->n[l]) src = 0;
                int s0 = l == 0 ? src : am, s1 = l == 0 ? am : src;
                lat_get(g, g->U, s0, s1, v);
                for (int c = 0; c < g->nc; ++c) v[c] *= sg[c];
                moving_wall_ghost(g, l, al, v);
                lat_set(g, g->U, a0, a1, v);
            }
        /* cells: ghost i in {-2,-1} and {n, n+1}; image through the lattice centre 2i+1 */
        int clo = (l == 0) ? 0 : -2, chi = (l == 0) ? imax(g, 1) - 1 : g->n[0] + 1;
        if (g->d == 1) clo = chi = 0;
        for (int im = clo; im <= chi; ++im)
            for (int il = -2; il <= g->n[l] + 1; ++il) {
                if (il >= 0 && il < g->n[l]) continue;
                int src = (image(g, l, 2 * il + 1, sg) - 1) / 2;
                int i0 = l == 0 ? il : im, i1 = l == 0 ? im : il;
                int s0 = l == 0 ? src : im, s1 = l == 0 ? im : src;
                cell_get(g, s0, s1, v);
                for (int c = 0; c < g->nc; ++c) v[c] *= sg[c];
                moving_wall_ghost(g, l, 2 * il + 1, v);
                cell_set(g, i0, i1, v);
            }
    }
}

/* ------------------------------------------------------------------------- */
/* Exact moving viscous shock (Sec. 4, 1D viscous shock wave; Becker's         */
/* solution): rho_L = w_L = m0 = 1, w_R / w_L = ((gamma-1) + 2/M0^2)/(gamma+1),  */
/* w0 = sqrt(w_L w_R); the relative velocity w(xi), xi = x - u_inf t, solves      */
/* xi = 2 mu gamma / ((gamma+1) m0 Pr) [w_L/(w_L-w_R) log((w_L-w)/(w_L-w0))     */
/*       - w_R/(w_L-w_R) log((w-w_R)/(w0-w_R))],                                */
/* rho = m0/w, u = u_inf + w, p = (gamma-1) rho e,                               */
/* e = ((gamma+1)/(gamma-1) w0^2 - w^2)/(2 gamma).                               */
/* ------------------------------------------------------------------------- */

static double becker_xi(const orc_problem *P, double w)
{
    double g = P->gamma, wL = 1.0, m0 = 1.0;
    double wR = wL * ((g - 1.0) + 2.0 / (P->ex_M0 * P->ex_M0)) / (g + 1.0), w0 = sqrt(wL * wR);
    double k = 2.0 * P->mu * g / ((g + 1.0) * m0 * P->Pr);
    return k * (wL / (wL - wR) * log((wL - w) / (wL - w0)) - wR / (wL - wR) * log((w - wR) / (w0 - wR)));
}

/* Primitive (rho, u, p) of the exact solution at (x, t): xi(w) decreases from
 * +inf (w -> w_R) to -inf (w -> w_L); bisection to the spacing of doubles. */
static void becker_prim(const orc_problem *P, double x, double t, double *rho, double *u, double *p)
{
    double g = P->gamma, wL = 1.0, m0 = 1.0;
    double wR = wL * ((g - 1.0) + 2.0 / (P->ex_M0 * P->ex_M0)) / (g + 1.0), w0 = sqrt(wL * wR);
    double xi = x - P->ex_uinf * t, lo = wR, hi = wL;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (becker_xi(P, mid) > xi) lo = mid;
        else hi = mid;
    }
    double w = 0.5 * (lo + hi);
    double e = ((g + 1.0) / (g - 1.0) * w0 * w0 - w * w) / (2.0 * g);
    *rho = m0 / w;
    *u = P->ex_uinf + w;
    *p = (g - 1.0) * (*rho) * e;
}

static void becker_cons(const orc_problem *P, double x, double t, double *U)
{
    double rho, u, p;
    becker_prim(P, x, t, &rho, &u, &p);
    U[0] = rho;
    U[1] = rho * u;
    U[2] = p / (P->gamma - 1.0) + 0.5 * rho * u * u;
}

/* 1D sides of kind ORC_BC_EXACT: ghost point and ghost cells from the exact
 * solution at time t (reading R15). */
static void exact_ghosts(grid_t *g, double t)
{
    const orc_problem *P = g->P;
    if (g->d != 1) return;
    static const double gx[5] = {-0.9061798459386640, -0.5384693101056831, 0.0, 0.5384693101056831,
                                 0.9061798459386640};
    static const double gw[5] = {0.2369268850561891, 0.4786286704993665, 0.5688888888888889, 0.4786286704993665,
                                 0.2369268850561891};
    double h = g->h[0];
    for (int side = 0; side < 2; ++side) {
        if (P->bc[side] != ORC_BC_EXACT) continue;
        double U[MAXC];
        int a = side ? 2 * g->n[0] + 2 : -2;
        becker_cons(P, P->lo1 + 0.5 * a * h, t, U);
        lat_set(g, g->U, a, 0, U);
        int c0 = side ? g->n[0] : -2;
        for (int i = c0; i < c0 + 2; ++i) {
            double A[MAXC] = {0, 0, 0, 0};
            for (int q = 0; q < 5; ++q) {
                becker_cons(P, P->lo1 + (i + 0.5 + 0.5 * gx[q]) * h, t, U);
                for (int c = 0; c < g->nc; ++c) A[c] += 0.5 * gw[q] * U[c];
            }
            cell_set(g, i, 0, A);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Cell centres: Simpson inversion (Sec. 2.1 / Sec. 2.2) and the scaling     */
/* limiter toward the cell average (Remark 3.1, reading R6).                 */
/* ------------------------------------------------------------------------- */

static void scale_toward(const orc_problem *P, const double *Ubar, double *Uc)
{
    int nc = P->dim + 2;
    double eps = P->eps;
    double rL = Ubar[0], rH = Uc[0];
    double er = rL < eps ? rL : eps;
    double th_r = orc_theta(rL, rH, er);
    double Ur[MAXC];
    for (int c = 0; c < nc; ++c) Ur[c] = (1.0 - th_r) * Ubar[c] + th_r * Uc[c];
    double pL = orc_pressure(P, Ubar), pH = orc_pressure(P, Ur);
    double ep = pL < eps ? pL : eps;
    double th_p = orc_theta(pL, pH, ep);
    double th = th_r * th_p;
    for (int c = 0; c < nc; ++c) Uc[c] = (1.0 - th) * Ubar[c] + th * Uc[c];
}

static void centres(grid_t *g)
{
    const orc_problem *P = g->P;
    double Ub[MAXC], Uc[MAXC];
    int i1lo = g->d == 2 ? -1 : 0, i1hi = g->d == 2 ? g->n[1] : 0;
    for (int i1 = i1lo; i1 <= i1hi; ++i1)
        for (int i0 = -1; i0 <= g->n[0]; ++i0) {
            int a0 = 2 * i0 + 1, a1 = g->d == 2 ? 2 * i1 + 1 : 0;
            cell_get(g, i0, i1, Ub);
            for (int c = 0; c < g->nc; ++c) {
                if (g->d == 1) {
                    /* U_i = (6 Ubar_i - (U_{i-1/2} + U_{i+1/2})) / 4 */
                    double zl = g->U[lat_idx(g, c, a0 - 1, 0)], zr = g->U[lat_idx(g, c, a0 + 1, 0)];
                    Uc[c] = (6.0 * Ub[c] - (zl + zr)) / 4.0;
                } else {
                    /* z_ij = (36 zbar - 4 (4 edge values) - (4 vertex values)) / 16 */
                    double edges = g->U[lat_idx(g, c, a0 - 1, a1)] + g->U[lat_idx(g, c, a0 + 1, a1)] +
                                   g->U[lat_idx(g, c, a0, a1 - 1)] + g->U[lat_idx(g, c, a0, a1 + 1)];
                    double verts = g->U[lat_idx(g, c, a0 - 1, a1 - 1)] + g->U[lat_idx(g, c, a0 + 1, a1 - 1)] +
                                   g->U[lat_idx(g, c, a0 - 1, a1 + 1)] + g->U[lat_idx(g, c, a0 + 1, a1 + 1)];
                    Uc[c] = (36.0 * Ub[c] - 4.0 * edges - verts) / 16.0;
                }
            }
            if (P->limiter != ORC_LIM_NONE) {
                double pc = orc_pressure(P, Uc);
                if (!(Uc[0] >= P->eps) || !(pc >= P->eps)) scale_toward(P, Ub, Uc);
            }
            lat_set(g, g->U, a0, a1, Uc);
        }
}

static void node_prims(grid_t *g)
{
    double U[MAXC], W[MAXC], Z[MAXC];
    for (int a1 = 0; a1 < g->na[1]; ++a1)
        for (int a0 = 0; a0 < g->na[0]; ++a0) {
            int b0 = a0 - g->off[0], b1 = a1 - g->off[1];
            lat_get(g, g->U, b0, b1, U);
            primitive(g->P, U, W);
            zvars(g->P, W, Z);
            lat_set(g, g->W, b0, b1, W);
            lat_set(g, g->Z, b0, b1, Z);
        }
}

/* ------------------------------------------------------------------------- */
/* Lattice line access                                                       */
/* ------------------------------------------------------------------------- */

static void step_node(int l, int k, int a0, int a1, int *b0, int *b1)
{
    *b0 = a0 + (l == 0 ? k : 0);
    *b1 = a1 + (l == 1 ? k : 0);
}

/* D_c along direction m of Z at node (a0,a1) (Eq. (8) on the lattice line) */
static void grad_Z(const grid_t *g, int m, int a0, int a1, double *dz)
{
    ORC_PURE(9, (const double *)0, 0, (const double *)0, 0, m, a0 * 65536 + a1);
    for (int c = 0; c < g->nc; ++c) {
        double z5[5];
        for (int k = -2; k <= 2; ++k) {
            int b0, b1;
            step_node(m, k, a0, a1, &b0, &b1);
            z5[k + 2] = g->Z[lat_idx(g, c, b0, b1)];
        }
        orc_op_dcentral(z5, g->h[m], &dz[c]);
    }
}

/* ------------------------------------------------------------------------- */
/* Point-value residual: Eq. (6b) in 1D, point part of Eq. (12) in 2D        */
/* ------------------------------------------------------------------------- */

static void point_residual(const grid_t *g, int a0, int a1, double *R)
{
    const orc_problem *P = g->P;
    int nc = g->nc, d = g->d;
    for (int c = 0; c < nc; ++c) R[c] = 0.0;
    for (int l = 0; l < d; ++l) {
        double dx = g->h[l];
        double U5[5][MAXC], W5[5][MAXC], Z5[5][MAXC], F5[5][MAXC];
        double alpha = 0.0;
        for (int k = -2; k <= 2; ++k) {
            int b0, b1;
            step_node(l, k, a0, a1, &b0, &b1);
            lat_get(g, g->U, b0, b1, U5[k + 2]);
            lat_get(g, g->W, b0, b1, W5[k + 2]);
            lat_get(g, g->Z, b0, b1, Z5[k + 2]);
            orc_inviscid_flux(P, U5[k + 2], l, F5[k + 2]);
            /* Sec. 2.1: alpha = max of the spectral radius over the 5 stencil nodes (R3) */
            double r = orc_wave_speed(P, U5[k + 2], l);
            if (r > alpha) alpha = r;
        }
        /* inviscid: D_+ (F^{c,+}) + D_- (F^{c,-}), F^{c,+-} = (F^c +- alpha U)/2 */
        for (int c = 0; c < nc; ++c) {
            double fp[5], fm[5], dp, dm;
            for (int k = 0; k < 5; ++k) {
                fp[k] = 0.5 * (F5[k][c] + alpha * U5[k][c]);
                fm[k] = 0.5 * (F5[k][c] - alpha * U5[k][c]);
            }
            orc_op_dplus(fp, dx, &dp);
            orc_op_dminus(fm, dx, &dm);
            R[c] -= dp + dm;
        }
        /* viscous, same direction: D^{(l),2}(K_ll, Z), Eq. (9) with matrix K:
         * sum_m sum_n b_mn K(W_m) Z_n, with K(W_m) taken out of the sum over n */
        {
            double b[25], s[MAXC] = {0, 0, 0, 0};
            orc_op_bmatrix(b);
            for (int m = 0; m < 5; ++m) {
                double y[MAXC] = {0, 0, 0, 0}, t[MAXC];
                for (int n = 0; n < 5; ++n)
                    for (int c = 0; c < nc; ++c) y[c] += b[m * 5 + n] * Z5[n][c];
                kapply(P, W5[m], l, l, y, t);
                for (int c = 0; c < nc; ++c) s[c] += t[c];
            }
            for (int c = 0; c < nc; ++c) R[c] += 4.0 / (dx * dx) * s[c];
        }
        /* viscous, mixed: D_c^{(l)} (K_lm D_c^{(m)} Z), m != l (Sec. 2.2) */
        for (int m = 0; m < d; ++m) {
            if (m == l) continue;
            double G5[5][MAXC];
            for (int k = -2; k <= 2; ++k) {
                int b0, b1;
                double dz[MAXC];
                step_node(l, k, a0, a1, &b0, &b1);
                grad_Z(g, m, b0, b1, dz);
                kapply(P, W5[k + 2], l, m, dz, G5[k + 2]);
            }
            for (int c = 0; c < nc; ++c) {
                double z5[5], dc;
                for (int k = 0; k < 5; ++k) z5[k] = G5[k][c];
                orc_op_dcentral(z5, dx, &dc);
                R[c] += dc;
            }
        }
    }
}

/* Total high-order flux F^c_l - F^v_l at a lattice node (Eqs. (6a),(6c), (12)). */
static void node_total_flux(const grid_t *g, int l, int a0, int a1, double *F)
{
    const orc_problem *P = g->P;
    double U[MAXC], grad[2 * MAXC], Fv[MAXC];
    lat_get(g, g->U, a0, a1, U);
    for (int m = 0; m < g->d; ++m) grad_Z(g, m, a0, a1, grad + m * g->nc);
    orc_inviscid_flux(P, U, l, F);
    orc_viscous_flux(P, U, grad, l, Fv);
    for (int c = 0; c < g->nc; ++c) F[c] -= Fv[c];
}

/* ------------------------------------------------------------------------- */
/* Low-order quantities per cell (Sec. 3.1) and the smoothness sensor        */
/* (Sec. 3.2), on cells [-1, n_l] in every used direction.                   */
/* ------------------------------------------------------------------------- */

typedef struct {
    double F[2][MAXC]; /* total low-order flux F_{l,i} = F^c_l(Ubar) - F^v_l(Ubar, S) */
    double rho_l[2];   /* spectral radius rho_l(Ubar) */
    double b_l[2];     /* viscous bound b_l(Ubar, S) */
    double phi1, phi2; /* Jameson and modified Ducros sensors */
} cellq_t;

static void cell_step(int l, int k, int i0, int i1, int *j0, int *j1)
{
    *j0 = i0 + (l == 0 ? k : 0);
    *j1 = i1 + (l == 1 ? k : 0);
}

static void cell_quantities(const grid_t *g, int i0, int i1, cellq_t *q)
{
    const orc_problem *P = g->P;
    int d = g->d, nc = g->nc;
    double U[MAXC], S[2 * MAXC];
    cell_get(g, i0, i1, U);
    /* S_i: central difference of Z(Ubar) (R5) */
    for (int m = 0; m < d; ++m) {
        double Up[MAXC], Um[MAXC], Wp[MAXC], Wm[MAXC], Zp[MAXC], Zm[MAXC];
        int p0, p1, m0, m1;
        cell_step(m, 1, i0, i1, &p0, &p1);
        cell_step(m, -1, i0, i1, &m0, &m1);
        cell_get(g, p0, p1, Up);
        cell_get(g, m0, m1, Um);
        primitive(P, Up, Wp);
        primitive(P, Um, Wm);
        zvars(P, Wp, Zp);
        zvars(P, Wm, Zm);
        for (int c = 0; c < nc; ++c) S[m * nc + c] = (Zp[c] - Zm[c]) / (2.0 * g->h[m]);
    }
    for (int l = 0; l < d; ++l) {
        double Fc[MAXC], Fv[MAXC];
        orc_inviscid_flux(P, U, l, Fc);
        orc_viscous_flux(P, U, S, l, Fv);
        for (int c = 0; c < nc; ++c) q->F[l][c] = Fc[c] - Fv[c];
        q->rho_l[l] = orc_wave_speed(P, U, l);
        q->b_l[l] = orc_visc_bound(P, U, S, l);
    }
    /* Sec. 3.2 sensors from cell-average pressure and velocity */
    double phi1 = 0.0, divu = 0.0, curl = 0.0;
    double pc = orc_pressure(P, U);
    for (int m = 0; m < d; ++m) {
        double Up[MAXC], Um[MAXC];
        int p0, p1, m0, m1;
        cell_step(m, 1, i0, i1, &p0, &p1);
        cell_step(m, -1, i0, i1, &m0, &m1);
        cell_get(g, p0, p1, Up);
        cell_get(g, m0, m1, Um);
        double pp = orc_pressure(P, Up), pm = orc_pressure(P, Um);
        double r = fabs(pp - 2.0 * pc + pm) / fabs(pp + 2.0 * pc + pm);
        if (r > phi1) phi1 = r;
        divu += (Up[1 + m] / Up[0] - Um[1 + m] / Um[0]) / (2.0 * g->h[m]);
        if (d == 2) {
            /* curl = d v / dx - d u / dy */
            if (m == 0) curl += (Up[2] / Up[0] - Um[2] / Um[0]) / (2.0 * g->h[0]);
            if (m == 1) curl -= (Up[1] / Up[0] - Um[1] / Um[0]) / (2.0 * g->h[1]);
        }
    }
    double phi2 = -divu / sqrt(divu * divu + curl * curl + 1e-13);
    q->phi1 = phi1;
    q->phi2 = phi2 > 0.0 ? phi2 : 0.0;
}

/* ------------------------------------------------------------------------- */
/* Low-order point update on the half lattice (Sec. 3.4, reading R7)         */
/* ------------------------------------------------------------------------- */

static void lattice_S(const grid_t *g, int a0, int a1, double *S)
{
    /* central differences of Z on the lattice, spacing dx_m/2 */
    for (int m = 0; m < g->d; ++m) {
        int p0, p1, q0, q1;
        step_node(m, 1, a0, a1, &p0, &p1);
        step_node(m, -1, a0, a1, &q0, &q1);
        for (int c = 0; c < g->nc; ++c)
            S[m * g->nc + c] = (g->Z[lat_idx(g, c, p0, p1)] - g->Z[lat_idx(g, c, q0, q1)]) / g->h[m];
    }
}

/* Eq. (19) between lattice neighbours A (left) and B (right) in direction l. */
static void lattice_llf(const grid_t *g, int l, int A0, int A1, int B0, int B1, double *Fh)
{
    const orc_problem *P = g->P;
    int nc = g->nc;
    double UA[MAXC], UB[MAXC], SA[2 * MAXC], SB[2 * MAXC], FA[MAXC], FB[MAXC], t[MAXC];
    lat_get(g, g->U, A0, A1, UA);
    lat_get(g, g->U, B0, B1, UB);
    lattice_S(g, A0, A1, SA);
    lattice_S(g, B0, B1, SB);
    orc_inviscid_flux(P, UA, l, FA);
    orc_viscous_flux(P, UA, SA, l, t);
    for (int c = 0; c < nc; ++c) FA[c] -= t[c];
    orc_inviscid_flux(P, UB, l, FB);
    orc_viscous_flux(P, UB, SB, l, t);
    for (int c = 0; c < nc; ++c) FB[c] -= t[c];
    double al = fmax(orc_wave_speed(P, UA, l), orc_wave_speed(P, UB, l));
    double be = fmax(orc_visc_bound(P, UA, SA, l), orc_visc_bound(P, UB, SB, l));
    double lam = al + be;
    for (int c = 0; c < nc; ++c) Fh[c] = 0.5 * (FA[c] + FB[c]) - 0.5 * lam * (UB[c] - UA[c]);
}

static void point_low_order(const grid_t *g, int a0, int a1, double dt, double *UL)
{
    int nc = g->nc;
    double U[MAXC];
    lat_get(g, g->U, a0, a1, U);
    for (int c = 0; c < nc; ++c) UL[c] = U[c];
    for (int l = 0; l < g->d; ++l) {
        double Fr[MAXC], Fl[MAXC];
        int p0, p1, q0, q1;
        step_node(l, 1, a0, a1, &p0, &p1);
        step_node(l, -1, a0, a1, &q0, &q1);
        lattice_llf(g, l, a0, a1, p0, p1, Fr);
        lattice_llf(g, l, q0, q1, a0, a1, Fl);
        double r = dt / (0.5 * g->h[l]);
        for (int c = 0; c < nc; ++c) UL[c] -= r * (Fr[c] - Fl[c]);
    }
}

/* ------------------------------------------------------------------------- */
/* The residual L(u) of one stage                                            */
/* ------------------------------------------------------------------------- */

/* ------------------------------------------------------------------------- */
/* Manufactured source (Sec. 4, 2D manufactured Taylor-Green vortex): with     */
/* a = exp(-2 mu t), b = cos 2x + cos 2y, u = a sin x cos y, v = -a cos x sin y, */
/* rho = 1 and p = p0/(gamma-1) + a^2 b/4, only the energy equation needs      */
/* S_E = (p_t + u p_x + v p_y)/(gamma-1) - 4 mu a^2 cos^2 x cos^2 y - kappa Lap p */
/* with p_t = -mu a^2 b, p_x = -a^2 sin(2x)/2, p_y = -a^2 sin(2y)/2,           */
/* Lap p = -a^2 b. Point values get S at the node, cell averages the 5 x 5     */
/* Gauss-Legendre average of S over the cell.                                  */
/* ------------------------------------------------------------------------- */

static double tg_energy_source(const orc_problem *P, double x, double y, double t)
{
    double a = exp(-2.0 * P->mu * t), a2 = a * a;
    double b = cos(2.0 * x) + cos(2.0 * y);
    double u = a * sin(x) * cos(y), v = -a * cos(x) * sin(y);
    double pt = -P->mu * a2 * b, px = -a2 * sin(2.0 * x) / 2.0, py = -a2 * sin(2.0 * y) / 2.0;
    double lap = -a2 * b;
    double cx = cos(x), cy = cos(y);
    return (pt + u * px + v * py) / (P->gamma - 1.0) - 4.0 * P->mu * a2 * cx * cx * cy * cy - kappa_of(P) * lap;
}

static void source_point(const orc_problem *P, double x, double y, double t, double *S)
{
    for (int c = 0; c < MAXC; ++c) S[c] = 0.0;
    if (P->source == ORC_SRC_TAYLOR_GREEN && P->dim == 2) S[3] = tg_energy_source(P, x, y, t);
}

static void source_cell(const orc_problem *P, double x0, double y0, double hx, double hy, double t, double *S)
{
    /* 5-point Gauss-Legendre nodes and weights on [-1, 1] */
    static const double gx[5] = {-0.9061798459386640, -0.5384693101056831, 0.0, 0.5384693101056831,
                                 0.9061798459386640};
    static const double gw[5] = {0.2369268850561891, 0.4786286704993665, 0.5688888888888889, 0.4786286704993665,
                                 0.2369268850561891};
    for (int c = 0; c < MAXC; ++c) S[c] = 0.0;
    if (P->source == ORC_SRC_NONE || P->dim != 2) return;
    for (int q1 = 0; q1 < 5; ++q1)
        for (int q0 = 0; q0 < 5; ++q0) {
            double Sq[MAXC];
            source_point(P, x0 + 0.5 * hx * (1.0 + gx[q0]), y0 + 0.5 * hy * (1.0 + gx[q1]), t, Sq);
            for (int c = 0; c < MAXC; ++c) S[c] += 0.25 * gw[q0] * gw[q1] * Sq[c];
        }
}

/* Eq. (19): the LLF total flux of the face between cells L and R in direction l,
 * from their total fluxes, wave speeds rho_l and viscous bounds b_l (Lemma 3.2). */
static void face_llf(int nc, int l, const cellq_t *qL, const cellq_t *qR, const double *UbL, const double *UbR,
                     double *FL)
{
    double al = fmax(qL->rho_l[l], qR->rho_l[l]);
    double be = fmax(qL->b_l[l], qR->b_l[l]);
    double lam = al + be;
    for (int c = 0; c < nc; ++c) FL[c] = 0.5 * (qL->F[l][c] + qR->F[l][c]) - 0.5 * lam * (UbR[c] - UbL[c]);
}

/* The low-order face flux of Eq. (19) of face (f0, f1) in direction l (between
 * cells f - e_l and f), exposed so that tests can pin it. */
void orc_face_low_order(const orc_problem *P, const double *state, int l, int f0, int f1, double *FL)
{
    grid_t G, *g = &G;
    grid_init(g, P);
    unpack(g, state);
    fill_ghosts(g);
    exact_ghosts(g, P->time);
    int L0, L1;
    cell_step(l, -1, f0, f1, &L0, &L1);
    cellq_t qL, qR;
    cell_quantities(g, L0, L1, &qL);
    cell_quantities(g, f0, f1, &qR);
    double UbL[MAXC], UbR[MAXC];
    cell_get(g, L0, L1, UbL);
    cell_get(g, f0, f1, UbR);
    face_llf(g->nc, l, &qL, &qR, UbL, UbR, FL);
    grid_free(g);
}

/* The low-order point update of lattice node (a0, a1) (reading R7), exposed so
 * that tests can pin it: the lattice is prepared exactly as for a residual
 * (ghosts, centres, node primitives), then point_low_order. */
void orc_point_low_order(const orc_problem *P, const double *state, double dt, int a0, int a1, double *UL)
{
    grid_t G, *g = &G;
    grid_init(g, P);
    unpack(g, state);
    fill_ghosts(g);
    exact_ghosts(g, P->time);
    centres(g);
    node_prims(g);
    point_low_order(g, a0, a1, dt, UL);
    grid_free(g);
}

int orc_residual(const orc_problem *P, const double *state, double dt, double *L, double *theta_s,
                 double *theta_pp, int *notpp)
{
    grid_t G, *g = &G;
    int bad = 0;
    grid_init(g, P);
    int d = g->d, nc = g->nc;
    unpack(g, state);
    ORC_PHASE(0); /* ghost fill */
    fill_ghosts(g);
    exact_ghosts(g, P->time);
    ORC_PHASE(1); /* cell centres and centre scaling limiter */
    centres(g);
    ORC_PHASE(2); /* node primitives W, Z */
    node_prims(g);
    ORC_PHASE(5); /* low-order cell quantities and smoothness sensors */

    /* cell quantities on cells [-1, n_l] */
    int ce0 = g->n[0] + 2, ce1 = d == 2 ? g->n[1] + 2 : 1;
    cellq_t *cq = (cellq_t *)calloc((size_t)ce0 * ce1, sizeof(cellq_t));
#define CQ(i0, i1) cq[(size_t)((i1) + (d == 2 ? 1 : 0)) * ce0 + (size_t)((i0) + 1)]
    for (int i1 = (d == 2 ? -1 : 0); i1 <= (d == 2 ? g->n[1] : 0); ++i1)
        for (int i0 = -1; i0 <= g->n[0]; ++i0) cell_quantities(g, i0, i1, &CQ(i0, i1));

    /* limited face fluxes; face f of direction l lies between cells f-1 and f */
    size_t nfx = (size_t)(g->n[0] + 1) * imax(g, 1);
    size_t nfy = d == 2 ? (size_t)g->n[0] * (g->n[1] + 1) : 0;
    double *Fx = (double *)calloc(nfx * nc, sizeof(double));
    double *Fy = d == 2 ? (double *)calloc(nfy * nc, sizeof(double)) : NULL;
    for (int l = 0; l < d; ++l) {
        int nf0 = l == 0 ? g->n[0] + 1 : g->n[0];
        int nf1 = d == 2 ? (l == 1 ? g->n[1] + 1 : g->n[1]) : 1;
        double *Fl = l == 0 ? Fx : Fy;
        double mu_l = dt / g->h[l];
        for (int f1 = 0; f1 < nf1; ++f1)
            for (int f0 = 0; f0 < nf0; ++f0) {
                size_t fid = (size_t)f1 * nf0 + f0;
                /* high-order total flux: Simpson average along the face (Sec. 2.2) */
                ORC_PHASE(4);
                double FH[MAXC] = {0, 0, 0, 0};
                if (d == 1) {
                    node_total_flux(g, 0, 2 * f0, 0, FH);
                } else {
                    static const double w[3] = {1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0};
                    for (int t = 0; t < 3; ++t) {
                        int a0 = l == 0 ? 2 * f0 : 2 * f0 + t;
                        int a1 = l == 0 ? 2 * f1 + t : 2 * f1;
                        double Fn[MAXC];
                        node_total_flux(g, l, a0, a1, Fn);
                        for (int c = 0; c < nc; ++c) FH[c] += w[t] * Fn[c];
                    }
                }
                double *out = Fl + fid * nc;
                double ts = 1.0, tpp = 1.0;
                if (P->limiter == ORC_LIM_NONE) {
                    for (int c = 0; c < nc; ++c) out[c] = FH[c];
                } else {
                    int L0, L1, R0, R1;
                    cell_step(l, -1, f0, f1, &L0, &L1);
                    R0 = f0;
                    R1 = f1;
                    const cellq_t *qL = &CQ(L0, L1), *qR = &CQ(R0, R1);
                    double UbL[MAXC], UbR[MAXC];
                    cell_get(g, L0, L1, UbL);
                    cell_get(g, R0, R1, UbR);
                    /* low-order LLF total flux, Eq. (19) */
                    ORC_PHASE(5);
                    double FL[MAXC], dF[MAXC], FLs[MAXC];
                    face_llf(nc, l, qL, qR, UbL, UbR, FL);
                    ORC_PHASE(6); /* monolithic limiter of the face */
                    /* smoothness-based blending, Sec. 3.2, Eq. (22) */
                    if (P->limiter == ORC_LIM_S_PP) {
                        double p1 = fmax(qL->phi1, qR->phi1), p2 = fmax(qL->phi2, qR->phi2);
                        ts = exp(-P->c_s * p1 * p2);
                    }
                    for (int c = 0; c < nc; ++c) {
                        FLs[c] = FL[c] + ts * (FH[c] - FL[c]);
                        dF[c] = FLs[c] - FL[c];
                    }
                    /* intermediate states, Eq. (20) and Sec. 3.3 (factor 2 d mu_l) */
                    double k = 2.0 * d * mu_l;
                    double ULp[MAXC], UHp[MAXC], ULm[MAXC], UHm[MAXC];
                    for (int c = 0; c < nc; ++c) {
                        ULp[c] = UbL[c] - k * (FL[c] - qL->F[l][c]);
                        UHp[c] = UbL[c] - k * (FLs[c] - qL->F[l][c]);
                        ULm[c] = UbR[c] - k * (qR->F[l][c] - FL[c]);
                        UHm[c] = UbR[c] - k * (qR->F[l][c] - FLs[c]);
                    }
                    if (!in_G(P, ULp) || !in_G(P, ULm)) bad = 1;
                    /* density: theta^rho, Sec. 3.3 */
                    double eRp = fmin(P->eps, ULp[0]), eRm = fmin(P->eps, ULm[0]);
                    double th_r = fmin(orc_theta(ULp[0], UHp[0], eRp), orc_theta(ULm[0], UHm[0], eRm));
                    double Urp[MAXC], Urm[MAXC];
                    for (int c = 0; c < nc; ++c) {
                        Urp[c] = (1.0 - th_r) * ULp[c] + th_r * UHp[c];
                        Urm[c] = (1.0 - th_r) * ULm[c] + th_r * UHm[c];
                    }
                    /* pressure: theta^p on the density-limited states (concavity of p) */
                    double pLp = orc_pressure(P, ULp), pLm = orc_pressure(P, ULm);
                    double ePp = fmin(P->eps, pLp), ePm = fmin(P->eps, pLm);
                    double th_p = fmin(orc_theta(pLp, orc_pressure(P, Urp), ePp),
                                       orc_theta(pLm, orc_pressure(P, Urm), ePm));
                    tpp = th_r * th_p;
                    for (int c = 0; c < nc; ++c) out[c] = FL[c] + tpp * dF[c];
                }
                if (theta_s || theta_pp) {
                    size_t o = (l == 0 ? 0 : nfx) + fid;
                    if (theta_s) theta_s[o] = ts;
                    if (theta_pp) theta_pp[o] = tpp;
                }
            }
    }

    /* cell-average residual: Eq. (6a) / Eq. (12) / Eq. (23) */
    ORC_PHASE(8);
    for (int i1 = 0; i1 < imax(g, 1); ++i1)
        for (int i0 = 0; i0 < g->n[0]; ++i0)
            for (int c = 0; c < nc; ++c) {
                double r = -(Fx[((size_t)i1 * (g->n[0] + 1) + i0 + 1) * nc + c] -
                             Fx[((size_t)i1 * (g->n[0] + 1) + i0) * nc + c]) / g->h[0];
                if (d == 2)
                    r -= (Fy[((size_t)(i1 + 1) * g->n[0] + i0) * nc + c] - Fy[((size_t)i1 * g->n[0] + i0) * nc + c]) /
                         g->h[1];
                L[packed_cell(P, c, i0, i1)] = r;
            }
    if (P->source != ORC_SRC_NONE)
        for (int i1 = 0; i1 < imax(g, 1); ++i1)
            for (int i0 = 0; i0 < g->n[0]; ++i0) {
                double S[MAXC];
                source_cell(P, P->lo1 + i0 * g->h[0], P->lo2 + i1 * g->h[1], g->h[0], g->h[1], P->time, S);
                for (int c = 0; c < nc; ++c) L[packed_cell(P, c, i0, i1)] += S[c];
            }

    /* point-value residual with the scaling limiter of Sec. 3.4 */
    for (int a1 = 0; a1 <= amax(g, 1); ++a1)
        for (int a0 = 0; a0 <= amax(g, 0); ++a0) {
            if (is_centre(g, a0, a1)) continue;
            double R[MAXC], U[MAXC], UH[MAXC];
            ORC_PHASE(3);
            point_residual(g, a0, a1, R);
            if (P->source != ORC_SRC_NONE) {
                double S[MAXC];
                source_point(P, P->lo1 + 0.5 * a0 * g->h[0], P->lo2 + 0.5 * a1 * g->h[1], P->time, S);
                for (int c = 0; c < nc; ++c) R[c] += S[c];
            }
            if (P->limiter != ORC_LIM_NONE) {
                ORC_PHASE(7); /* point scaling limiter */
                lat_get(g, g->U, a0, a1, U);
                for (int c = 0; c < nc; ++c) UH[c] = U[c] + dt * R[c];
                double pH = orc_pressure(P, UH);
                if (!(UH[0] >= P->eps) || !(pH >= P->eps)) {
                    double UL[MAXC], Ur[MAXC];
                    point_low_order(g, a0, a1, dt, UL);
                    if (!in_G(P, UL)) bad = 1;
                    double th_r = orc_theta(UL[0], UH[0], fmin(P->eps, UL[0]));
                    for (int c = 0; c < nc; ++c) Ur[c] = (1.0 - th_r) * UL[c] + th_r * UH[c];
                    double pL = orc_pressure(P, UL);
                    double th_p = orc_theta(pL, orc_pressure(P, Ur), fmin(P->eps, pL));
                    double th = th_r * th_p;
                    for (int c = 0; c < nc; ++c) R[c] = ((1.0 - th) * UL[c] + th * UH[c] - U[c]) / dt;
                }
            }
            for (int c = 0; c < nc; ++c) L[packed_point(P, c, a0, a1)] = R[c];
        }
#undef CQ
    free(cq);
    free(Fx);
    free(Fy);
    grid_free(g);
    if (notpp) *notpp = bad;
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Time step (Eq. (13)) and SSP-RK54 driver with restart (Remark 3.2)        */
/* ------------------------------------------------------------------------- */

void orc_defaults(orc_problem *P)
{
    P->ex_M0 = 3.0;
    P->ex_uinf = 0.2;
    for (int k = 0; k < 4; ++k) P->wall_speed[k] = 0.0;
    P->limiter = ORC_LIM_S_PP;
    P->source = ORC_SRC_NONE;
    P->src_p0 = 100.0;
    P->time = 0.0;
    P->c_s = 1.0;
    P->cfl_c = 1.04 / P->dim;
    P->cfl_v = P->dim == 1 ? 0.33 : 0.13;   /* reading R14 */
    P->eps = 1e-13;
}

double orc_dt_max(const orc_problem *P, const double *state)
{
    int d = P->dim, nc = d + 2;
    double h[2] = {(P->hi1 - P->lo1) / P->n1, d == 2 ? (P->hi2 - P->lo2) / P->n2 : 1.0};
    double m1 = 0.0, m2 = 0.0;
    int n2 = d == 2 ? P->n2 : 1;
    for (int i1 = 0; i1 < n2; ++i1)
        for (int i0 = 0; i0 < P->n1; ++i0) {
            double U[MAXC];
            for (int c = 0; c < nc; ++c) U[c] = state[packed_cell(P, c, i0, i1)];
            for (int l = 0; l < d; ++l) {
                double a = orc_wave_speed(P, U, l) / (P->cfl_c * h[l]);
                double b = visc_eigen(P, U) / (P->cfl_v * h[l] * h[l]);
                if (a > m1) m1 = a;
                if (b > m2) m2 = b;
            }
        }
    return 1.0 / (m1 + m2);
}

/* R9: wall point values get zero (normal) momentum, internal energy kept; R17:
 * on a moving wall the tangential momentum is rho U_w (sides in the order x-lo,
 * x-hi, y-lo, y-hi, so a corner takes the velocity of its y-side). */
static void wall_fix(const orc_problem *P, double *s)
{
    int d = P->dim, nc = d + 2;
    int n[2] = {P->n1, d == 2 ? P->n2 : 0};
    for (int side = 0; side < 2 * d; ++side) {
        int kind = P->bc[side];
        if (kind != ORC_BC_WALL && kind != ORC_BC_SYMMETRY && kind != ORC_BC_MOVING) continue;
        int l = side / 2, m = 1 - l;
        int al = (side & 1) ? 2 * n[l] : 0;
        int mhi = d == 2 ? 2 * n[m] : 0;
        for (int am = 0; am <= mhi; ++am) {
            int a0 = l == 0 ? al : am, a1 = l == 0 ? am : al;
            if (d == 2 && (a0 & 1) && (a1 & 1)) continue;
            double U[MAXC];
            size_t o[MAXC];
            for (int c = 0; c < nc; ++c) {
                o[c] = packed_point(P, c, a0, a1);
                U[c] = s[o[c]];
            }
            double ke_old = 0.0, ke_new = 0.0;
            for (int k = 0; k < d; ++k) ke_old += U[1 + k] * U[1 + k];
            for (int k = 0; k < d; ++k)
                if (kind != ORC_BC_SYMMETRY || k == l) U[1 + k] = 0.0;
            if (kind == ORC_BC_MOVING && d == 2) U[1 + m] = U[0] * P->wall_speed[side];
            for (int k = 0; k < d; ++k) ke_new += U[1 + k] * U[1 + k];
            U[d + 1] -= (ke_old - ke_new) / (2.0 * U[0]);
            for (int c = 0; c < nc; ++c) s[o[c]] = U[c];
        }
    }
}

int orc_step(const orc_problem *P, double *state, double dt, int max_halvings, double *dt_taken, int *halvings)
{
    size_t n = orc_state_len(P);
    double a[5][5], b[5][5];
    orc_rk_table(a, b);
    double *u[6], *Lk[5];
    for (int k = 0; k < 6; ++k) u[k] = (double *)malloc(n * sizeof(double));
    for (int k = 0; k < 5; ++k) Lk[k] = (double *)malloc(n * sizeof(double));
    /* time of stage state u(s) as a fraction of dt: c(u(s+1)) = sum_k a_sk c(u(k)) + b_sk */
    double cst[6] = {0.0};
    for (int s = 0; s < 5; ++s)
        for (int k = 0; k <= s; ++k) cst[s + 1] += a[s][k] * cst[k] + b[s][k];
    orc_problem Q = *P;
    int h = 0, rc = ORC_ENOTPP;
    for (;;) {
        int bad = 0;
        memcpy(u[0], state, n * sizeof(double));
        for (int s = 0; s < 5 && !bad; ++s) {
            int nb = 0;
            Q.time = P->time + cst[s] * dt;
            orc_residual(&Q, u[s], dt, Lk[s], NULL, NULL, &nb);
            if (nb) bad = 1;
            ORC_PHASE(10); /* SSP-RK54 combination */
            for (size_t x = 0; x < n; ++x) {
                double v = 0.0;
                for (int k = 0; k <= s; ++k) v += a[s][k] * u[k][x] + b[s][k] * dt * Lk[k][x];
                u[s + 1][x] = v;
            }
            wall_fix(P, u[s + 1]);
        }
        if (!bad) {
            memcpy(state, u[5], n * sizeof(double));
            rc = ORC_OK;
            break;
        }
        if (h >= max_halvings) break;
        dt *= 0.5;
        ++h;
    }
    if (dt_taken) *dt_taken = rc == ORC_OK ? dt : 0.0;
    if (halvings) *halvings = h;
    for (int k = 0; k < 6; ++k) free(u[k]);
    for (int k = 0; k < 5; ++k) free(Lk[k]);
    return rc;
}

int orc_advance(const orc_problem *P, double *state, double t, double t_end, int max_halvings, int max_steps,
                int *steps, int *restarts)
{
    int ns = 0, nr = 0, rc = ORC_OK;
    orc_problem Q = *P;
    while (t < t_end && (max_steps <= 0 || ns < max_steps)) {
        double dt = orc_dt_max(P, state);
        if (t + dt > t_end) dt = t_end - t;
        double taken;
        int h;
        Q.time = t;
        rc = orc_step(&Q, state, dt, max_halvings, &taken, &h);
        nr += h;
        if (rc != ORC_OK) break;
        t += taken;
        ++ns;
    }
    if (steps) *steps = ns;
    if (restarts) *restarts = nr;
    return rc;
}
