// stage2d.cuh -- fused 2D AF-NS Runge-Kutta stage kernel and its helpers.
//
// One CTA owns a TX x TY tile of cells. It stages the tile's half lattice
// (point values + reconstructed cell centres, two lattice nodes of halo) and the
// cell averages (two cells of halo) in shared memory, then computes in phases
// separated by barriers:
//   P0  load        point values and cell averages of the stage input
//   P1  centres +   Simpson inversion (Sec. 2.2) + scaling limiter (Remark 3.1),
//       primitives  and u, v, T, c at every lattice node
//   P3  gradients   D_c^(x) Z and D_c^(y) Z (Eq. (8)) at lattice nodes
//   P4  points +    point residual (Eq. (12)), point scaling limiter (Sec. 3.4),
//       faces (HO)  RK combination, store; high-order Simpson face fluxes
//   P5a cells (LO)  low-order cell quantities (Sec. 3.1, 3.2)
//   P5b faces       LLF flux (Eq. (19)), theta_s (Eq. (22)), theta^rho theta^p
//                   (Sec. 3.3), limited flux
//   P6  cells       cell residual (Eq. (23)), RK combination, store
// The lattice state, primitives and gradients are dead after P4, so the
// low-order cell records of P5a reuse their space; the shared memory of a 16x8
// FP32 tile (54 KB) then admits four CTAs per SM.
// Faces on tile borders are evaluated by both neighbouring tiles from identical
// inputs with identical code, so the two copies agree bit for bit and the update
// stays conservative to roundoff.
#pragma once

#include <cuda.h>   // CUtensorMap (the type only; no driver call is made from here)

#include "afns_dev.cuh"

namespace afns {

// The constants of the two terms of Eq. (13) per cell average: the spacings
// and CFL numbers folded in, so that a cell costs one reciprocal of rho. Formed
// once on the host and shared by every kernel that evaluates the bound (the
// CFL pass and the last stage of a step give the same step bit for bit).
struct CflConst {
    double g1, gamma, ix, iy, rvc;        // rvc = rho~ rho (Eq. (13)) x max_l 1 / (C^v dx_l^2)
    float g1f, gf, ixf, iyf, rvcf;
};
__host__ __device__ inline CflConst cfl_const(double gamma, double mu, double Pr, double cfl_c, double cfl_v,
                                              double dx, double dy)
{
    CflConst k;
    k.g1 = gamma - 1.0;
    k.gamma = gamma;
    k.ix = 1.0 / (cfl_c * dx);
    k.iy = 1.0 / (cfl_c * dy);
    const double vx = 1.0 / (cfl_v * dx * dx), vy = 1.0 / (cfl_v * dy * dy);
    const double a = 4.0 * mu / 3.0, b = gamma * mu / Pr;
    k.rvc = (a > b ? a : b) * (vx > vy ? vx : vy);
    k.g1f = (float)k.g1;
    k.gf = (float)gamma;
    k.ixf = (float)k.ix;
    k.iyf = (float)k.iy;
    k.rvcf = (float)k.rvc;
    return k;
}
// One cell average's terms, merged into the running maxima m1 (inviscid) and
// m2 (viscous); FP64 for the FP64 path, FP32 for the mixed path (the step size
// needs no more than FP32 accuracy). A NaN term is ignored, as by fmax.
__device__ __forceinline__ void cfl_terms(const CflConst &k, double rho, double mx, double my, double E, double &m1,
                                          double &m2)
{
    const double r = 1.0 / rho, uu = mx * r, vv = my * r;
    const double p = k.g1 * (E - 0.5 * (mx * uu + my * vv));
    const double c = sqrt(k.gamma * p * r);
    m1 = fmax(m1, fmax((fabs(uu) + c) * k.ix, (fabs(vv) + c) * k.iy));
    m2 = fmax(m2, k.rvc * r);
}
__device__ __forceinline__ void cfl_terms(const CflConst &k, float rho, float mx, float my, float E, float &m1,
                                          float &m2)
{
    const float r = 1.f / rho, uu = mx * r, vv = my * r;
    const float p = k.g1f * (E - 0.5f * (mx * uu + my * vv));
    const float c = sqrtf(k.gf * p * r);
    m1 = fmaxf(m1, fmaxf((fabsf(uu) + c) * k.ixf, (fabsf(vv) + c) * k.iyf));
    m2 = fmaxf(m2, k.rvcf * r);
}

struct StageArgs {
    Layout L;
    const void *uin;   // state being evaluated (ghosts filled)
    const void *u0;    // step start
    void *aux;         // u(2) / accumulator
    void *out;         // stage output (residual mode: L)
    Ctl *ctl;          // dt, notpp flag
    double *theta;     // optional per-face [theta_s | theta_pp] (2 * faces)
    StageCoef k;
    double gamma, mu, kappa, eps, c_s;
    int limiter;
    int source;        // 0: none, 1: Taylor-Green energy source (Sec. 4 example)
    double src_p0;
    const void *tconst;  // per-stage tile constants computed by k_tile_consts (or null)
    CflConst cfl;        // Eq. (13) constants (used when k.cfl_out)
    int extra_tx;        // test hook: bytes the tile-load barrier expects beyond the copies (0)
};

template <int TX, int TY>
struct Tile2 {
    static constexpr int LX = 2 * TX + 5;
    static constexpr int LY = 2 * TY + 5;
    static constexpr int NL = LX * LY;
    static constexpr int CX = TX + 4, CY = TY + 4, NCA = CX * CY;   // cells with 2 halo
    static constexpr int QX = TX + 2, QY = TY + 2, NCQ = QX * QY;   // cells with 1 halo
    static constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1);
    // x gradients exist on lattice columns [2, LX-3], y gradients on rows [2, LY-3]
    static constexpr int GXW = LX - 4, NGX = GXW * LY, NGY = LX * (LY - 4);
    // shared-memory offsets in units of V4 (one node / cell / face record)
    static constexpr int oU = 0;                 // NL  x (rho, rho u, rho v, E)
    static constexpr int oQ = oU + NL;           // NL  x (u, v, T, c)
    static constexpr int oGX = oQ + NL;          // NGX x d/dx (u, v, T, -)
    static constexpr int oGY = oGX + NGX;        // NGY x d/dy (u, v, T, -)
    static constexpr int oA = oGY + NGY;         // NCA x cell averages
    static constexpr int oFX = oA + NCA;         // NFX x x-face flux: high order, then limited
    static constexpr int oFY = oFX + NFX;        // NFY x y-face flux
    static constexpr int total = oFY + NFY;      // in V4 records
    // after P4: the 4 x NCQ records of low-order cell quantities over the lattice state
    static constexpr int oCQ = oU;
    static_assert(4 * NCQ <= NL, "low-order cell records fit in the lattice state");
    template <class R>
    static constexpr size_t bytes() { return (size_t)total * 4 * sizeof(R); }
    // Lattice records are stored row by row with every row de-interleaved: its HE
    // even columns first, then its odd ones. Items on every other column (edge
    // points, centres, face nodes) are then consecutive records, so the threads of
    // a warp that take consecutive such items touch consecutive records (no
    // shared-memory bank conflicts); lattice x-neighbours la +- 2 are records +- 1.
    static constexpr int HE = (LX + 1) / 2;
    __host__ __device__ static constexpr int col(int la) { return (la & 1) ? HE + (la >> 1) : (la >> 1); }
    __host__ __device__ static constexpr int node(int la, int lb) { return lb * LX + col(la); }
    // lattice column of position c of a de-interleaved row
    __host__ __device__ static constexpr int col_inv(int c) { return c < HE ? 2 * c : 2 * (c - HE) + 1; }
    // x gradients on columns [2, LX-3] of every row, de-interleaved likewise (the
    // GXE even columns first); y gradients on rows [2, LY-3], full rows
    static constexpr int GXE = (LX - 3) / 2;
    __host__ __device__ static constexpr int gxcol(int la) { return (la & 1) ? GXE + ((la - 3) >> 1) : ((la - 2) >> 1); }
    __host__ __device__ static constexpr int gxcol_inv(int c) { return c < GXE ? 2 + 2 * c : 3 + 2 * (c - GXE); }
    // index of the x / y gradient of lattice node (la, lb)
    __host__ __device__ static constexpr int gx(int la, int lb) { return lb * GXW + gxcol(la); }
    __host__ __device__ static constexpr int gy(int la, int lb) { return (lb - 2) * LX + col(la); }
};

// Four values of one lattice node, cell or face, stored together so that one
// vector instruction moves them (16-byte shared-memory accesses in FP32).
template <class R>
struct alignas(4 * sizeof(R)) V4 {
    R x, y, z, w;
};

// Per-tile constants in the compute precision, derived once per tile by one
// thread (the mixed path then runs no FP64 instruction outside its islands).
template <class R>
struct TileConst {
    R gam, gm1, mu, ka, dx, dy, dt, eps, cs;
    R kkx, kky;          // 2 d dt / dx_l with d = 2 (Sec. 3.3 intermediate states)
    R w;                 // weight of L in the stage output (cl dt, or 1 in residual mode)
    R a0, a1, a2, b1, b2, bldt;
    // float-float weights of the compensated cell-average update (mixed path)
    ff fa0, fa1, fa2, fwx, fwy, fb1, fb2, fbx, fby;
    R idx, idy;
    int ua0, ua2;        // the combination reads u^n / the auxiliary state
    R i6[2];             // 1 / (6 dx_l): D_c and the FVS stencils
    R i3h2[2];           // 1 / (3 dx_l^2): (4 / dx_l^2) times the 1/12 of the column sums
    R f4h2[2];           // 4 / dx_l^2: prefactor of Eq. (9)
    R i2[2];             // 1 / (2 dx_l): central differences of the cell averages
};

// No divisions: the grid reciprocals come from the layout (host-computed), dt
// enters by multiplication.
template <class R>
__device__ __forceinline__ void tile_const_init(TileConst<R> &t, const StageArgs &A, double dt)
{
    const Layout &L = A.L;
    t.gam = (R)A.gamma;
    t.gm1 = (R)(A.gamma - 1.0);
    t.mu = (R)A.mu;
    t.ka = (R)A.kappa;
    t.dx = (R)L.dx;
    t.dy = (R)L.dy;
    t.dt = (R)dt;
    t.eps = (R)A.eps;
    t.cs = (R)A.c_s;
    t.kkx = (R)(4.0 * dt * L.idx[0]);
    t.kky = (R)(4.0 * dt * L.idx[1]);
    t.w = (R)(A.k.residual ? 1.0 : A.k.cl * dt);
    t.a0 = (R)A.k.a0;
    t.a1 = (R)A.k.a1;
    t.a2 = (R)A.k.a2;
    t.b1 = (R)A.k.b1;
    t.b2 = (R)A.k.b2;
    t.bldt = (R)(A.k.bl * dt);
    t.fa0 = ff_from(A.k.a0);
    t.fa1 = ff_from(A.k.a1);
    t.fa2 = ff_from(A.k.a2);
    t.fwx = ff_from(A.k.cl * dt * L.idx[0]);
    t.fwy = ff_from(A.k.cl * dt * L.idx[1]);
    t.fb1 = ff_from(A.k.b1);
    t.fb2 = ff_from(A.k.b2);
    t.fbx = ff_from(A.k.bl * dt * L.idx[0]);
    t.fby = ff_from(A.k.bl * dt * L.idx[1]);
    t.idx = (R)L.idx[0];
    t.idy = (R)L.idx[1];
    t.ua0 = A.k.a0 != 0.0;
    t.ua2 = A.k.a2 != 0.0;
    for (int l = 0; l < 2; ++l) {
        t.i6[l] = (R)L.i6[l];
        t.i3h2[l] = (R)L.i3h2[l];
        t.f4h2[l] = (R)L.f4h2[l];
        t.i2[l] = (R)L.i2[l];
    }
}

// Manufactured energy source of the 2D Taylor-Green vortex (Sec. 4 example),
// FP64: a = exp(-2 mu t), b = cos 2x + cos 2y, u = a sin x cos y,
// v = -a cos x sin y, p = p0/(gamma-1) + a^2 b/4 (rho = 1);
// S_E = (p_t + u p_x + v p_y)/(gamma-1) - 4 mu a^2 cos^2 x cos^2 y - kappa Lap p,
// p_t = -mu a^2 b, p_x = -a^2 sin(2x)/2, p_y = -a^2 sin(2y)/2, Lap p = -a^2 b.
__device__ inline double tg_energy_source(double mu, double kappa, double gamma, double x, double y, double t)
{
    const double a = exp(-2.0 * mu * t), a2 = a * a;
    const double b = cos(2.0 * x) + cos(2.0 * y);
    const double sx = sin(x), cx = cos(x), sy = sin(y), cy = cos(y);
    const double u = a * sx * cy, v = -a * cx * sy;
    const double pt = -mu * a2 * b, px = -a2 * sin(2.0 * x) / 2.0, py = -a2 * sin(2.0 * y) / 2.0;
    return (pt + u * px + v * py) / (gamma - 1.0) - 4.0 * mu * a2 * cx * cx * cy * cy + kappa * a2 * b;
}

// The source at lattice node (a, b) (spacing half a cell) and its 5 x 5
// Gauss-Legendre average over cell (i, j), at time t, for a grid with origin
// (x0, y0) and spacing (hx, hy).
static __device__ __forceinline__ double tg_point_source(double mu, double kappa, double gamma, double x0, double y0,
                                                      double hx, double hy, int a, int b, double t)
{
    return tg_energy_source(mu, kappa, gamma, x0 + 0.5 * a * hx, y0 + 0.5 * b * hy, t);
}
static __device__ __forceinline__ double tg_cell_source(double mu, double kappa, double gamma, double x0, double y0,
                                                     double hx, double hy, int i, int j, double t)
{
    const double gx[5] = {-0.9061798459386640, -0.5384693101056831, 0.0, 0.5384693101056831, 0.9061798459386640};
    const double gw[5] = {0.2369268850561891, 0.4786286704993665, 0.5688888888888889, 0.4786286704993665,
                          0.2369268850561891};
    const double xc = x0 + i * hx, yc = y0 + j * hy;
    double s = 0.0;
    for (int q1 = 0; q1 < 5; ++q1)
        for (int q0 = 0; q0 < 5; ++q0)
            s += 0.25 * gw[q0] * gw[q1] *
                 tg_energy_source(mu, kappa, gamma, xc + 0.5 * hx * (1.0 + gx[q0]), yc + 0.5 * hy * (1.0 + gx[q1]), t);
    return s;
}

// Records of the low-order cell quantities (4 arrays of NCQ records, one per field):
// [0] total flux F_x, [1] total flux F_y, [2] (rho_x, rho_y, b_x, b_y), [3] (phi1, phi2, -, -)
enum { CQ_FX = 0, CQ_FY = 1, CQ_RB = 2, CQ_PH = 3 };

// D_c weights (x 1/(6 dx)) and fourth-difference weights of (D_+ - D_-)/2 (x 1/(6 dx))
__device__ __constant__ static const double kDC[5] = {1.0, -8.0, 0.0, 8.0, -1.0};
__device__ __constant__ static const double kD4[5] = {1.0, -4.0, 6.0, -4.0, 1.0};
// M of Eq. (10) (rows p, columns q)
__device__ __constant__ static const double kM[4][4] = {
    {1.0 / 8.0, -1.0 / 6.0, 1.0 / 24.0, 0.0},
    {-1.0 / 6.0, -3.0 / 8.0, 2.0 / 3.0, -1.0 / 8.0},
    {1.0 / 8.0, -2.0 / 3.0, 3.0 / 8.0, 1.0 / 6.0},
    {0.0, -1.0 / 24.0, 1.0 / 6.0, -1.0 / 8.0},
};

// B of Eq. (10) written out (rows m = -2..2, columns n = -2..2), from
// B = [[0,0],[0,M]] - [[M,0],[0,0]].
__device__ __constant__ static const double kB[5][5] = {
    {-1.0 / 8.0, 1.0 / 6.0, -1.0 / 24.0, 0.0, 0.0},
    {1.0 / 6.0, 1.0 / 2.0, -5.0 / 6.0, 1.0 / 6.0, 0.0},
    {-1.0 / 8.0, 1.0 / 2.0, -3.0 / 4.0, 1.0 / 2.0, -1.0 / 8.0},
    {0.0, 1.0 / 6.0, -5.0 / 6.0, 1.0 / 2.0, 1.0 / 6.0},
    {0.0, 0.0, -1.0 / 24.0, 1.0 / 6.0, -1.0 / 8.0},
};
// Column sums of B times 12: the textbook 5-point second difference.
__device__ __constant__ static const double kD2[5] = {-1.0, 16.0, -30.0, 16.0, -1.0};

template <class S>
__device__ __forceinline__ double ld(const void *base, long long off)
{
    return (double)((const S *)base)[off];
}

// Conservative -> primitive helpers in precision R
template <class R>
__device__ __forceinline__ R pressure2(R rho, R mx, R my, R E, R gm1)
{
    return gm1 * (E - (mx * mx + my * my) / (R(2) * rho));
}

// Gate of the FP64 islands: is a state V, computed in precision R from terms of
// magnitude at most mag[c] per component, certainly at or above eps in density and
// pressure? In FP64 this is the exact test. In FP32 the test keeps margins far
// above the rounding error of the terms (density 1e-2 of its term magnitude,
// pressure 1e-3 of its term magnitude), so "true" implies the FP64 answer; a
// "false" only sends the state to the FP64 island, which decides exactly.
// Reciprocal, square root, reciprocal square root and exponential of the
// compute precision. FP32: the hardware approximations (PTX rcp/sqrt/rsqrt
// .approx.ftz, __expf), within about 2 ulp: their values feed FP32 stencils and
// screens whose own rounding is larger, and every positivity decision that they
// could tip is re-taken in FP64. FP64: correctly rounded division and square
// root; the reciprocal square root from the math library's rsqrt (1 ulp), one
// operation instead of a square root and a division.
template <class R>
__device__ __forceinline__ R frcp(R x)
{
    if constexpr (sizeof(R) == 4) {
        float y;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    } else {
        return 1.0 / x;
    }
}
template <class R>
__device__ __forceinline__ R fsqrt(R x)
{
    if constexpr (sizeof(R) == 4) {
        float y;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    } else {
        return sqrt(x);
    }
}
template <class R>
__device__ __forceinline__ R frsqrt(R x)
{
    if constexpr (sizeof(R) == 4) {
        float y;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    } else {
        return rsqrt(x);
    }
}
template <class R>
__device__ __forceinline__ R fexp(R x)
{
    if constexpr (sizeof(R) == 4) return __expf(x);
    else return exp(x);
}

template <class R>
__device__ __forceinline__ bool surely_above(const R V[4], const R mag[4], R gm1, R eps)
{
    if constexpr (sizeof(R) == 8) {
        // the exact test without a division: for rho >= eps > 0,
        // p >= eps  <=>  (gamma-1) (2 rho E - |m|^2) >= 2 rho eps
        return V[0] >= eps && gm1 * (2.0 * V[0] * V[3] - (V[1] * V[1] + V[2] * V[2])) >= 2.0 * V[0] * eps;
    } else {
        if (!(V[0] > 1e-2f * mag[0] + eps)) return false;
        // a screen with percent-level margins: the fast reciprocal (2 ulp) suffices
        const float ir = __fdividef(1.f, V[0]);
        float ke = 0.5f * (V[1] * V[1] + V[2] * V[2]) * ir;
        float p = gm1 * (V[3] - ke);
        float m2 = mag[1] * mag[1] + mag[2] * mag[2];
        return p > 1e-3f * gm1 * (mag[3] + m2 * ir) + eps;
    }
}

// Is U admissible (finite, rho > 0, p > 0)? Evaluated in FP64.
// Check of an input DoF (finite, rho > 0, p > 0) without a division: for
// rho > 0 and gamma > 1, p > 0 exactly when 2 rho E > |m|^2.
__device__ __forceinline__ bool admissible_input2(const double *U)
{
    const bool fin = isfinite(U[0]) && isfinite(U[1]) && isfinite(U[2]) && isfinite(U[3]);
    return fin && U[0] > 0.0 && 2.0 * U[0] * U[3] > U[1] * U[1] + U[2] * U[2];
}

// The same check for FP32 values: decided in FP32 when 2 rho E and |m|^2 differ by
// more than 1e-5 relatively (their FP32 roundings are below 2e-7 relatively, so
// the order is certain), in FP64 otherwise and near the ends of the FP32 range.
__device__ __forceinline__ bool admissible_input2(const float *v)
{
    if (!(isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]) && isfinite(v[3]) && v[0] > 0.f)) return false;
    const float a = 2.f * v[0] * v[3], b = fmaf(v[1], v[1], v[2] * v[2]);
    if (a > 1e-30f && a < 1e30f && b < 1e30f) {
        if (a > b * 1.00001f) return true;
        if (a < b * 0.99999f) return false;
    }
    const double U[4] = {v[0], v[1], v[2], v[3]};
    return admissible_input2(U);
}

// Finite, rho >= eps and p >= eps (eps > 0), decided without a division.
__device__ __forceinline__ bool above_eps2(const double *U, double gm1, double eps)
{
    return isfinite(U[0] + U[1] + U[2] + U[3]) && U[0] >= eps &&
           gm1 * (2.0 * U[0] * U[3] - (U[1] * U[1] + U[2] * U[2])) >= 2.0 * U[0] * eps;
}

__device__ __forceinline__ bool admissible2(const double *U, double gm1)
{
    if (!(U[0] > 0.0)) return false;
    double p = gm1 * (U[3] - (U[1] * U[1] + U[2] * U[2]) / (2.0 * U[0]));
    bool fin = isfinite(U[0]) && isfinite(U[1]) && isfinite(U[2]) && isfinite(U[3]);
    return fin && p > 0.0;
}

// Monolithic positivity limiter of one face in FP64 (Sec. 3.3). Inputs: the total
// low-order fluxes F_{l,i} of the cells left (FLc) and right (FRc) of the face, their
// averages, the LLF speed lam of Eq. (19), theta_s and the high-order flux FH;
// kk = 2 d dt / dx_l. Returns the limited flux F^L + theta^rho theta^p theta_s (FH - F^L),
// theta^rho theta^p, and sets *bad when a low-order state U^{L,+-} leaves G.
__device__ __forceinline__ void face_pp_fp64(const double FLc[4], const double FRc[4], const double UbL[4],
                                             const double UbR[4], double lam, double ts, const double FH[4],
                                             double kk, double g1, double eps, double Fout[4], double *tpp,
                                             bool *bad)
{
    double FL[4], FLs[4], dF[4], ULp[4], UHp[4], ULm[4], UHm[4];
    for (int c = 0; c < 4; ++c) {
        FL[c] = 0.5 * (FLc[c] + FRc[c]) - 0.5 * lam * (UbR[c] - UbL[c]);
        FLs[c] = FL[c] + ts * (FH[c] - FL[c]);
        dF[c] = FLs[c] - FL[c];
        ULp[c] = UbL[c] - kk * (FL[c] - FLc[c]);
        UHp[c] = UbL[c] - kk * (FLs[c] - FLc[c]);
        ULm[c] = UbR[c] - kk * (FRc[c] - FL[c]);
        UHm[c] = UbR[c] - kk * (FRc[c] - FLs[c]);
    }
    // The common case first, without a division: both low-order and both
    // high-order states finite with density and pressure at or above eps (then
    // every Theta is 1 and no low-order state leaves G); the pressure test is
    // (gamma-1) (2 rho E - |m|^2) >= 2 rho eps for rho >= eps > 0.
    if (above_eps2(ULp, g1, eps) && above_eps2(ULm, g1, eps) && above_eps2(UHp, g1, eps) &&
        above_eps2(UHm, g1, eps)) {
        *tpp = 1.0;
        for (int c = 0; c < 4; ++c) Fout[c] = FL[c] + 1.0 * dF[c];
        return;
    }
    if (!admissible2(ULp, g1) || !admissible2(ULm, g1)) *bad = true;
    double thr = fmin(theta_fn(ULp[0], UHp[0], fmin(eps, ULp[0])), theta_fn(ULm[0], UHm[0], fmin(eps, ULm[0])));
    double Urp[4], Urm[4];
    for (int c = 0; c < 4; ++c) {
        Urp[c] = (1.0 - thr) * ULp[c] + thr * UHp[c];
        Urm[c] = (1.0 - thr) * ULm[c] + thr * UHm[c];
    }
    double pLp = g1 * (ULp[3] - (ULp[1] * ULp[1] + ULp[2] * ULp[2]) / (2.0 * ULp[0]));
    double pLm = g1 * (ULm[3] - (ULm[1] * ULm[1] + ULm[2] * ULm[2]) / (2.0 * ULm[0]));
    double prp = g1 * (Urp[3] - (Urp[1] * Urp[1] + Urp[2] * Urp[2]) / (2.0 * Urp[0]));
    double prm = g1 * (Urm[3] - (Urm[1] * Urm[1] + Urm[2] * Urm[2]) / (2.0 * Urm[0]));
    double thp = fmin(theta_fn(pLp, prp, fmin(eps, pLp)), theta_fn(pLm, prm, fmin(eps, pLm)));
    *tpp = thr * thp;
    for (int c = 0; c < 4; ++c) Fout[c] = FL[c] + *tpp * dF[c];
}

}  // namespace afns
