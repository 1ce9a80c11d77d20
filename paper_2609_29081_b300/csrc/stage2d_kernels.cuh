// stage2d_kernels.cuh -- 2D device code of libafns: ghost fill, fused RK stage,
// CFL reduction, state validation. The phase structure of the stage kernel is
// described in stage2d.cuh.
#pragma once

#include "stage2d.cuh"

namespace afns {

// ---------------------------------------------------------------------------
// Ghost fill: two ghost layers (periodic wrap, wall / symmetry / transmissive
// mirror, moving-wall shift), in one launch.
// ---------------------------------------------------------------------------
// Ghost value of (i, j) in direction l from its image (si, sj), which is read
// from buf: mirror signs, then the moving-wall shift of side `side`.
template <class S>
__device__ __forceinline__ void ghost_from_image(const Layout &L, const S *buf, int site, int si, int sj, int l,
                                                 int side, S v[4])
{
    const int kind = L.bc[2 * l + side];
    for (int c = 0; c < 4; ++c) {
        v[c] = buf[plane_of(L, site, c) + cell_off(L, si, sj)];
        if (mirror_sign(kind, l, c, 2) < 0) v[c] = -v[c];
    }
    moving_wall_ghost(L, 2 * l + side, v);
}

// Ghost fill in one launch, with the values of an x pass followed by a y pass:
// the x ghosts of the rows that are not y ghosts, and the y-ghost rows over all
// columns, where a column that is itself an x ghost takes the x transform of its
// x image (the value an x pass would have stored there), then the y transform.
template <class S>
__global__ void k_ghost2d_once(Layout L, S *buf)
{
    const int nx = 4 * (L.n2 + 1) * 5, ny = 4 * (L.n1 + 5) * 5;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nx + ny; t += gridDim.x * blockDim.x) {
        const bool xpass = t < nx;
        const int u = xpass ? t : t - nx, span = xpass ? (L.n2 + 1) : (L.n1 + 5);
        const int g = u % 5, r = (u / 5) % span, site = u / (5 * span);
        const bool ptx = site == 1 || site == 3, pty = site == 2 || site == 3;
        S v[4];
        int i, j;
        if (xpass) {
            j = r;
            if (j > L.n2 - 1 + (pty ? 1 : 0)) continue;
            int sdy;
            ghost_image(j, L.n2, pty, L.bc[2], L.bc[3], &sdy);
            if (sdy >= 0) continue;   // a y-ghost row: the y items write it
            i = g < 2 ? g - 2 : L.n1 + (g - 2);
            int side;
            const int si = ghost_image(i, L.n1, ptx, L.bc[0], L.bc[1], &side);
            if (side < 0) continue;
            ghost_from_image(L, buf, site, si, j, 0, side, v);
        } else {
            i = r - 2;
            j = g < 2 ? g - 2 : L.n2 + (g - 2);
            int side;
            const int sj = ghost_image(j, L.n2, pty, L.bc[2], L.bc[3], &side);
            if (side < 0) continue;
            int sdx;
            const int si = ghost_image(i, L.n1, ptx, L.bc[0], L.bc[1], &sdx);
            if (sdx < 0) {
                ghost_from_image(L, buf, site, i, sj, 1, side, v);
            } else {
                S w[4];
                ghost_from_image(L, buf, site, si, sj, 0, sdx, w);   // the x pass's value at (i, sj)
                const int kind = L.bc[2 + side];
                for (int c = 0; c < 4; ++c) v[c] = mirror_sign(kind, 1, c, 2) < 0 ? -w[c] : w[c];
                moving_wall_ghost(L, 2 + side, v);
            }
        }
        for (int c = 0; c < 4; ++c) buf[plane_of(L, site, c) + cell_off(L, i, j)] = v[c];
    }
}

template <class R>
__device__ __forceinline__ R comp(const V4<R> &v, int c)
{
    return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w;
}

// ---------------------------------------------------------------------------
// Point-value residual of Eq. (12) at lattice node n of the shared tile.
// sU: conservative, sQ: (u, v, T, c), sGX / sGY: D_c gradients of (v, u, T)
// (v first: the FP32 form below pairs them crosswise with (u, v)).
// ---------------------------------------------------------------------------
template <class R, int TX, int TY>
__device__ __forceinline__ void point_residual(const V4<R> *sm, int la, int lb, const TileConst<R> &tc, R res[4])
{
    using T = Tile2<TX, TY>;
    constexpr int LX = T::LX;
    const int n = T::node(la, lb);
    // the x-line la-2 .. la+2 in the de-interleaved rows: the same-parity
    // neighbours are records n -+ 1, the others sit in the row's other half
    const int row = lb * LX;
    const int xl[5] = {n - 1, row + T::col(la - 1), n, row + T::col(la + 1), n + 1};
    const V4<R> *sU = sm + T::oU, *sQ = sm + T::oQ, *sGX = sm + T::oGX, *sGY = sm + T::oGY;
    const R mu = tc.mu, ka = tc.ka;
    res[0] = res[1] = res[2] = res[3] = R(0);
    const R mu43 = R(4) / R(3) * mu, mu23 = R(2) / R(3) * mu;
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        V4<R> q[5], u[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int m = l == 0 ? xl[k] : n + (k - 2) * LX;
            q[k] = sQ[m];
            u[k] = sU[m];
        }
        // --- inviscid: D_+ F^+ + D_- F^- = [sum_k dc_k F_k + alpha sum_k d4_k U_k] / (6 h)
        // (alpha multiplies the fourth-difference sum once; dc_2 = 0 skips the
        // centre's flux)
        R al = R(0);
#pragma unroll
        for (int k = 0; k < 5; ++k) al = dmax(al, fabs(l == 0 ? q[k].x : q[k].y) + q[k].w);
        // F_l = u_l U + p (0, e_x, e_y, u_l) with the mass flux m_l kept exact:
        // sum_k dc_k F_k = (sum dc_k m_l, sum a_k m_x, sum a_k m_y, sum a_k E)
        //                + (0, P e_x, P e_y, sum a_k p_k),  a_k = dc_k u_l,k, P = sum dc_k p_k
        R f0 = 0, f1 = 0, f2 = 0, f3 = 0, h0 = 0, h1 = 0, h2 = 0, h3 = 0, sp = 0;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const R w4 = (R)kD4[k];
            h0 += w4 * u[k].x;
            h1 += w4 * u[k].y;
            h2 += w4 * u[k].z;
            h3 += w4 * u[k].w;
            if (kDC[k] == 0.0) continue;
            const R wc = (R)kDC[k];
            const R p = u[k].x * q[k].z;   // rho T
            const R a = wc * (l == 0 ? q[k].x : q[k].y);
            f0 += wc * (l == 0 ? u[k].y : u[k].z);
            f1 += a * u[k].y;
            f2 += a * u[k].z;
            f3 += a * (u[k].w + p);
            sp += wc * p;
        }
        if (l == 0)
            f1 += sp;
        else
            f2 += sp;
        const R inv6h = tc.i6[l];
        res[0] -= (f0 + al * h0) * inv6h;
        res[1] -= (f1 + al * h1) * inv6h;
        res[2] -= (f2 + al * h2) * inv6h;
        res[3] -= (f3 + al * h3) * inv6h;
        // --- viscous, same direction: D^{(l),2}(K_ll, Z) of Eq. (9), the K
        // coefficients applied once to the sums over the stencil; the energy
        // term's sum_m z_m (B z)_m is the quadratic form z^T B z, evaluated with
        // the upper triangle of B + B^T (12 nonzero products instead of 19 + 5)
        const R c1 = l == 0 ? mu43 : mu;   // K_ll entry on u
        const R c2 = l == 0 ? mu : mu43;   // K_ll entry on v
        R d2u = 0, d2v = 0, d2T = 0, equ = 0, eqv = 0;
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            d2u += (R)kD2[m] * q[m].x;
            d2v += (R)kD2[m] * q[m].y;
            d2T += (R)kD2[m] * q[m].z;
            R bu = 0, bv = 0;
#pragma unroll
            for (int nn = m; nn < 5; ++nn) {
                const double cmn = nn == m ? kB[m][m] : kB[m][nn] + kB[nn][m];
                if (cmn == 0.0) continue;
                bu += (R)cmn * q[nn].x;
                bv += (R)cmn * q[nn].y;
            }
            equ += q[m].x * bu;
            eqv += q[m].y * bv;
        }
        const R i3h2 = tc.i3h2[l];   // (4/dx^2)/12
        res[1] += c1 * d2u * i3h2;
        res[2] += c2 * d2v * i3h2;
        res[3] += ka * d2T * i3h2 + tc.f4h2[l] * (c1 * equ + c2 * eqv);
        // --- viscous, mixed: D_c^{(l)}(K_lm D_c^{(m)} Z), m != l, as sums of
        // dc_k (d u, d v) and of dc_k (u d v, v d u) that the K entries multiply once
        R su = 0, sv = 0, cuv = 0, cvu = 0;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            if (k == 2) continue;
            const R wc = (R)kDC[k];
            // y gradients at the x-neighbours (rows from 2), x gradients at the
            // y-neighbours; records hold (d v, d u, d T)
            const V4<R> g = l == 0 ? sGY[xl[k] - 2 * LX] : sGX[T::gx(la, lb) + (k - 2) * T::GXW];
            su += wc * g.y;
            sv += wc * g.x;
            cuv += wc * (q[k].x * g.x);   // u d v
            cvu += wc * (q[k].y * g.y);   // v d u
        }
        R g1, g2, g3;
        if (l == 0) {   // K_12 d_y Z: (-2/3 mu d_y v, mu d_y u, mu v d_y u - 2/3 mu u d_y v)
            g1 = -mu23 * sv;
            g2 = mu * su;
            g3 = mu * cvu - mu23 * cuv;
        } else {        // K_21 d_x Z: (mu d_x v, -2/3 mu d_x u, mu u d_x v - 2/3 mu v d_x u)
            g1 = mu * sv;
            g2 = -mu23 * su;
            g3 = mu * cuv - mu23 * cvu;
        }
        res[1] += g1 * inv6h;
        res[2] += g2 * inv6h;
        res[3] += g3 * inv6h;
    }
}

// Two-lane FP32 arithmetic (the packed FFMA2 / FADD2 / FMUL2 instructions of
// sm_100 and later): one instruction for a pair of independent FP32 operations.
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 xy2(const V4<float> &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 zw2(const V4<float> &v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }

// Float-float arithmetic of two components at once: the error-free sums and
// products of ff_quick / ff_two_sum / ff_add / ff_mul, lane by lane, with the
// same operations in the same order (so the same bits as the one-lane form).
struct ff2 {
    float2 h, l;
};
__device__ __forceinline__ ff2 ff2_quick(float2 a, float2 b)
{
    const float2 s = add2(a, b);
    return {s, sub2(b, sub2(s, a))};
}
__device__ __forceinline__ ff2 ff2_two_sum(float2 a, float2 b)
{
    const float2 s = add2(a, b), bb = sub2(s, a);
    return {s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}
__device__ __forceinline__ ff2 ff2_add(ff2 a, ff2 b)
{
    const ff2 s = ff2_two_sum(a.h, b.h);
    return ff2_quick(s.h, add2(add2(s.l, a.l), b.l));
}
// a weight (the same for both lanes) times a pair
__device__ __forceinline__ ff2 ff2_mul(ff a, ff2 b)
{
    const float2 ah = bc2(a.h), al = bc2(a.l);
    const float2 p = mul2(ah, b.h);
    float2 e = fma2(ah, b.h, neg2(p));
    e = fma2(ah, b.l, fma2(al, b.h, e));
    return ff2_quick(p, e);
}

// FP32 form of the point residual: the sums of the generic form above, carried
// in the component pairs (rho, m_x), (m_y, E), (u, v) and the gradient pairs
// (v, u) of the stored records, with the FVS flux sums regrouped as
//   sum_k dc_k F_k = sum_k (dc_k u_l,k) U_k + (0, P e_x, P e_y, sum_k dc_k u_l,k p_k),
//   P = sum_k dc_k p_k   (F_l = u_l U + p (0, e_x, e_y, u_l)),
// the fourth-difference dissipation as alpha * sum_k d4_k U_k, the cross
// viscous terms as sums of dc_k (d v, d u) and of dc_k (u d v, v d u) that the
// K coefficients multiply once, and the energy term of D^2 as
// c1 sum_m u_m (B u)_m + c2 sum_m v_m (B v)_m.
template <int TX, int TY>
__device__ __forceinline__ void point_residual_f32(const V4<float> *sm, int la, int lb, const TileConst<float> &tc,
                                                   float res[4])
{
    using T = Tile2<TX, TY>;
    constexpr int LX = T::LX;
    const int n = T::node(la, lb);
    const int row = lb * LX;
    const int xl[5] = {n - 1, row + T::col(la - 1), n, row + T::col(la + 1), n + 1};
    const V4<float> *sU = sm + T::oU, *sQ = sm + T::oQ, *sGX = sm + T::oGX, *sGY = sm + T::oGY;
    const float mu = tc.mu, ka = tc.ka;
    const float mu43 = 4.0f / 3.0f * mu, mu23 = 2.0f / 3.0f * mu;
    float2 r01 = bc2(0.0f), r23 = bc2(0.0f);   // inviscid part of (res0, res1), (res2, res3)
    float2 v12 = bc2(0.0f);                     // viscous part of (res1, res2)
    float v3 = 0.0f;                            // viscous part of res3
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        V4<float> q[5], u[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int m = l == 0 ? xl[k] : n + (k - 2) * LX;
            q[k] = sQ[m];
            u[k] = sU[m];
        }
        // --- inviscid
        float al = 0.0f;
#pragma unroll
        for (int k = 0; k < 5; ++k) al = fmaxf(al, fabsf(l == 0 ? q[k].x : q[k].y) + q[k].w);
        float2 a01 = bc2(0.0f), a23 = bc2(0.0f), d01 = bc2(0.0f), d23 = bc2(0.0f);
        float sp = 0.0f, spu = 0.0f;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            if (kDC[k] != 0.0) {
                const float wc = (float)kDC[k];
                const float ul = l == 0 ? q[k].x : q[k].y;
                const float p = u[k].x * q[k].z;   // rho T
                const float a = wc * ul;
                a01 = fma2(bc2(a), xy2(u[k]), a01);
                a23 = fma2(bc2(a), zw2(u[k]), a23);
                sp = fmaf(wc, p, sp);
                spu = fmaf(a, p, spu);
            }
            const float2 w4 = bc2((float)kD4[k]);
            d01 = fma2(w4, xy2(u[k]), d01);
            d23 = fma2(w4, zw2(u[k]), d23);
        }
        float2 f01 = fma2(bc2(al), d01, a01), f23 = fma2(bc2(al), d23, a23);
        if (l == 0)
            f01.y += sp;
        else
            f23.x += sp;
        f23.y += spu;
        const float2 mi6 = bc2(-tc.i6[l]);
        r01 = fma2(f01, mi6, r01);
        r23 = fma2(f23, mi6, r23);
        // --- viscous, same direction: D^{(l),2}(K_ll, Z) of Eq. (9)
        const float c1 = l == 0 ? mu43 : mu, c2 = l == 0 ? mu : mu43;
        float2 d2 = bc2(0.0f), e = bc2(0.0f);
        float d2T = 0.0f;
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            const float2 qm = xy2(q[m]);
            d2 = fma2(bc2((float)kD2[m]), qm, d2);
            d2T = fmaf((float)kD2[m], q[m].z, d2T);
            float2 b = bc2(0.0f);
#pragma unroll
            for (int nn = 0; nn < 5; ++nn)
                if (kB[m][nn] != 0.0) b = fma2(bc2((float)kB[m][nn]), xy2(q[nn]), b);
            e = fma2(qm, b, e);
        }
        const float i3h2 = tc.i3h2[l];
        v12 = fma2(make_float2(c1 * i3h2, c2 * i3h2), d2, v12);
        v3 = fmaf(ka * i3h2, d2T, v3);
        v3 = fmaf(tc.f4h2[l], fmaf(c1, e.x, c2 * e.y), v3);
        // --- viscous, mixed: D_c^{(l)}(K_lm D_c^{(m)} Z), m != l
        float2 sg = bc2(0.0f), cg = bc2(0.0f);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            if (k == 2) continue;
            const float2 wc = bc2((float)kDC[k]);
            // (d v, d u): y gradients at the x-neighbours, x gradients at the y-neighbours
            const float2 gp = xy2(l == 0 ? sGY[xl[k] - 2 * LX] : sGX[T::gx(la, lb) + (k - 2) * T::GXW]);
            sg = fma2(wc, gp, sg);
            cg = fma2(wc, mul2(xy2(q[k]), gp), cg);   // (u d v, v d u)
        }
        const float i6 = tc.i6[l];
        if (l == 0) {   // K_12 d_y Z: (g1, g2) = (-mu23 S_v, mu S_u), g3 = mu (v d u) - mu23 (u d v)
            v12 = fma2(make_float2(-mu23 * i6, mu * i6), sg, v12);
            v3 = fmaf(i6, fmaf(mu, cg.y, -mu23 * cg.x), v3);
        } else {        // K_21 d_x Z: (g1, g2) = (mu S_v, -mu23 S_u), g3 = mu (u d v) - mu23 (v d u)
            v12 = fma2(make_float2(mu * i6, -mu23 * i6), sg, v12);
            v3 = fmaf(i6, fmaf(mu, cg.x, -mu23 * cg.y), v3);
        }
    }
    res[0] = r01.x;
    res[1] = r01.y + v12.x;
    res[2] = r23.x + v12.y;
    res[3] = r23.y + v3;
}

// Total flux F^c_l - F^v_l at a node with node gradients (gx, gy) of (u, v, T).
template <class R>
__device__ __forceinline__ void node_flux(int l, R rho, R mx, R my, R E, R u, R v, R T, R gxu, R gxv, R gxT,
                                          R gyu, R gyv, R gyT, R mu, R ka, R F[4])
{
    const R p = rho * T;
    const R div = gxu + gyv;
    const R txy = mu * (gyu + gxv);
    if (l == 0) {
        const R txx = mu * (R(2) * gxu - R(2) / R(3) * div);
        F[0] = mx;
        F[1] = mx * u + p - txx;
        F[2] = my * u - txy;
        F[3] = (E + p) * u - (u * txx + v * txy + ka * gxT);
    } else {
        const R tyy = mu * (R(2) * gyv - R(2) / R(3) * div);
        F[0] = my;
        F[1] = mx * v - txy;
        F[2] = my * v + p - tyy;
        F[3] = (E + p) * v - (u * txy + v * tyy + ka * gyT);
    }
}

// Low-order total LLF flux between lattice nodes A and B along l on the half
// lattice (point low-order update, Sec. 3.4 reading): Eq. (19) with S from
// central differences on the lattice. FP64.
template <class R, int TX, int TY>
__device__ __noinline__ void lattice_llf(const V4<R> *sm, int l, int laA, int lbA, int laB, int lbB, double dx,
                                         double dy, double gamma, double mu, double ka, double F[4])
{
    using T = Tile2<TX, TY>;
    constexpr int LX = T::LX;
    const V4<R> *sU = sm + T::oU, *sQ = sm + T::oQ;
    double Fs[2][4], Us[2][4], rs[2], bs[2];
    const double gm1 = gamma - 1.0;
    for (int s = 0; s < 2; ++s) {
        const int la = s == 0 ? laA : laB, lb = s == 0 ? lbA : lbB;
        const int n = T::node(la, lb);
        const V4<R> un = sU[n];
        double Uv[4] = {(double)un.x, (double)un.y, (double)un.z, (double)un.w};
        const V4<R> qe = sQ[T::node(la + 1, lb)], qw = sQ[T::node(la - 1, lb)], qn = sQ[n + LX], qs = sQ[n - LX];
        // S: central differences on the lattice (spacing h/2, so 2 * (h/2) = h)
        double Sx[3] = {((double)qe.x - (double)qw.x) / dx, ((double)qe.y - (double)qw.y) / dx,
                        ((double)qe.z - (double)qw.z) / dx};
        double Sy[3] = {((double)qn.x - (double)qs.x) / dy, ((double)qn.y - (double)qs.y) / dy,
                        ((double)qn.z - (double)qs.z) / dy};
        double rho = Uv[0], u = Uv[1] / rho, v = Uv[2] / rho;
        double p = gm1 * (Uv[3] - (Uv[1] * Uv[1] + Uv[2] * Uv[2]) / (2.0 * rho));
        double Fl[4];
        node_flux<double>(l, rho, Uv[1], Uv[2], Uv[3], u, v, p / rho, Sx[0], Sx[1], Sx[2], Sy[0], Sy[1], Sy[2], mu, ka,
                          Fl);
        for (int c = 0; c < 4; ++c) Fs[s][c] = Fl[c], Us[s][c] = Uv[c];
        double c_ = sqrt(gamma * p / rho);
        rs[s] = fabs(l == 0 ? u : v) + c_;
        double div = Sx[0] + Sy[1];
        double t1, t2;
        if (l == 0) {
            t1 = mu * (2.0 * Sx[0] - 2.0 / 3.0 * div);
            t2 = mu * (Sy[0] + Sx[1]);
        } else {
            t1 = mu * (Sy[0] + Sx[1]);
            t2 = mu * (2.0 * Sy[1] - 2.0 / 3.0 * div);
        }
        double q = -ka * (l == 0 ? Sx[2] : Sy[2]);
        double re = p / gm1;   // rho e
        bs[s] = (sqrt(rho * rho * q * q + 2.0 * rho * re * (t1 * t1 + t2 * t2)) + rho * fabs(q)) / (2.0 * rho * re);
    }
    double lam = fmax(rs[0], rs[1]) + fmax(bs[0], bs[1]);
    for (int c = 0; c < 4; ++c) F[c] = 0.5 * (Fs[0][c] + Fs[1][c]) - 0.5 * lam * (Us[1][c] - Us[0][c]);
}

// ---------------------------------------------------------------------------
// The fused stage kernel
// ---------------------------------------------------------------------------
// One tile (bx, by) of one problem; the single-problem kernel runs one tile per
// CTA, the batched persistent kernel loops over (problem, tile) work items.
// Per-tile constants: copied (cp.async, one 4-byte word per thread) from the
// record k_tile_consts wrote for this stage, or, without one, formed by thread 0.
template <class R>
__device__ __forceinline__ void load_tile_consts(TileConst<R> &tc, const StageArgs &A, int tid)
{
    static_assert(sizeof(TileConst<R>) % 4 == 0, "word copy");
    constexpr int NW = sizeof(TileConst<R>) / 4;
    if (A.tconst) {
        if (tid < NW) cp_async_elem(reinterpret_cast<unsigned *>(&tc) + tid, reinterpret_cast<const unsigned *>(A.tconst) + tid);
    } else if (tid == 0) {
        tile_const_init<R>(tc, A, A.ctl->dt);
    }
}

// The per-tile constants of one stage, once per launch (one thread): the FP64
// products and conversions stay out of every tile's critical path.
template <class R>
__global__ void k_tile_consts(StageArgs A, TileConst<R> *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) tile_const_init<R>(*out, A, A.ctl->dt);
}

// The constants of all five stages of a step in one launch (thread s: stage s),
// written stride_bytes apart.
struct StageCoef5 {
    StageCoef k[5];
};
template <class R>
__global__ void k_tile_consts5(StageArgs A, StageCoef5 ks, char *out, int stride_bytes)
{
    const int s = threadIdx.x;
    if (blockIdx.x != 0 || s >= 5) return;
    StageArgs B = A;
    B.k = ks.k[s];
    tile_const_init<R>(*reinterpret_cast<TileConst<R> *>(out + (size_t)s * stride_bytes), B, A.ctl->dt);
    // the step's last stage merges the next CFL maxima from zero
    if (s == 0) A.ctl->cfl_mx[0] = A.ctl->cfl_mx[1] = 0ull;
}

// (u, v, T, c) of a lattice node, one reciprocal of rho: u = m_x/rho,
// v = m_y/rho, p = (gamma-1)(E - m.u/2), T = p/rho, c = sqrt(gamma T).
template <class R>
__device__ __forceinline__ V4<R> node_prims(const V4<R> &U, R gm1, R gam)
{
    const R r = frcp(U.x), u = U.y * r, v = U.z * r;
    const R p = gm1 * (U.w - R(0.5) * (U.y * u + U.z * v));
    const R Tn = p * r;
    return V4<R>{u, v, Tn, fsqrt(gam * Tn)};
}

// (u, v, p, T) of a cell average, one reciprocal of rho.
template <class R>
__device__ __forceinline__ V4<R> cell_prims(const V4<R> &U, R gm1)
{
    const R r = frcp(U.x), u = U.y * r, v = U.z * r;
    const R p = gm1 * (U.w - R(0.5) * (U.y * u + U.z * v));
    return V4<R>{u, v, p, p * r};
}

// High-order total flux of face item f (x-faces first, then y-faces) of the
// tile: Simpson's rule over the vertex, edge and vertex point fluxes of the face
// (Eq. (12)), each with its node gradients; written to the face's flux slot.
template <class R, int TX, int TY>
__device__ __forceinline__ void face_high_order(V4<R> *sm, int f, int ntx, int nty, R mu, R ka)
{
    using T = Tile2<TX, TY>;
    int l, fl, el;   // direction, face index along l (local), index along the face (local)
    if (f < T::NFX) {
        l = 0;
        fl = f % (TX + 1);
        el = f / (TX + 1);
        if (fl > ntx || el >= nty) return;
    } else {
        l = 1;
        const int u_ = f - T::NFX;
        el = u_ % TX;
        fl = u_ / TX;
        if (el >= ntx || fl > nty) return;
    }
    const V4<R> *sU = sm + T::oU, *sQ = sm + T::oQ, *sGX = sm + T::oGX, *sGY = sm + T::oGY;
    R FH[4] = {0, 0, 0, 0};
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const int la = l == 0 ? 2 + 2 * fl : 2 + 2 * el + s;
        const int lb = l == 0 ? 2 + 2 * el + s : 2 + 2 * fl;
        const int n = T::node(la, lb);
        const V4<R> U = sU[n], Qn = sQ[n], gx = sGX[T::gx(la, lb)], gy = sGY[T::gy(la, lb)];
        R Fn[4];
        node_flux<R>(l, U.x, U.y, U.z, U.w, Qn.x, Qn.y, Qn.z, gx.y, gx.x, gx.z, gy.y, gy.x, gy.z, mu, ka, Fn);
        const R ws = s == 1 ? R(4) / R(6) : R(1) / R(6);
#pragma unroll
        for (int c = 0; c < 4; ++c) FH[c] += ws * Fn[c];
    }
    V4<R> *slot = l == 0 ? sm + T::oFX + el * (TX + 1) + fl : sm + T::oFY + fl * TX + el;
    *slot = V4<R>{FH[0], FH[1], FH[2], FH[3]};
}

// Point nodes of the tile lattice (all nodes but the cell centres), numbered
// compactly row pair by row pair in the order of the de-interleaved records: an
// even lattice row holds (LX + 1) / 2 vertices and then (LX - 1) / 2 y-edges,
// the odd row after it (LX + 1) / 2 x-edges.
template <int LX, int LY>
__host__ __device__ constexpr int point_count()
{
    return ((LY + 1) / 2) * LX + (LY / 2) * ((LX + 1) / 2);
}
template <int LX>
__device__ __forceinline__ void point_node(int t, int &la, int &lb)
{
    constexpr int HE = (LX + 1) / 2, PAIR = LX + HE;
    const int pr = t / PAIR, r = t - pr * PAIR;
    if (r < LX) {
        lb = 2 * pr;
        la = r < HE ? 2 * r : 2 * (r - HE) + 1;
    } else {
        lb = 2 * pr + 1;
        la = 2 * (r - LX);
    }
}

// FP64 island of the point update (Sec. 3.4) for a point whose FP32 screen did
// not clear it: the exact test of the high-order value U^n + dt r, and where that
// leaves G_eps the low-order LLF point update on the half lattice and the Theta
// blend; returns the blended residual. Out of line: few points take it, and
// inlined, its FP64 conversions were scheduled ahead of the screen for every point.
template <class S>
struct PointFix {
    S r[4];
    int blended, bad;
};
template <class R, class S, int TX, int TY>
__device__ __noinline__ PointFix<S> point_island(const V4<R> *sm, int la, int lb, V4<R> un, V4<R> rr4, double dt,
                                                 double eps, double gamma, double mu, double kappa, double dx,
                                                 double dy)
{
    PointFix<S> f{};
    const R Un[4] = {un.x, un.y, un.z, un.w}, r[4] = {rr4.x, rr4.y, rr4.z, rr4.w};
    double Ud[4], UH[4];
    for (int c = 0; c < 4; ++c) Ud[c] = (double)Un[c], UH[c] = Ud[c] + dt * (double)r[c];
    const double gm1d = gamma - 1.0;
    const double pH = gm1d * (UH[3] - (UH[1] * UH[1] + UH[2] * UH[2]) / (2.0 * UH[0]));
    if (UH[0] >= eps && pH >= eps) return f;
    double UL[4] = {Ud[0], Ud[1], Ud[2], Ud[3]};
    for (int l = 0; l < 2; ++l) {
        const int ea = l == 0 ? 1 : 0, eb = l == 0 ? 0 : 1;
        double Fr[4], Fl[4];
        lattice_llf<R, TX, TY>(sm, l, la, lb, la + ea, lb + eb, dx, dy, gamma, mu, kappa, Fr);
        lattice_llf<R, TX, TY>(sm, l, la - ea, lb - eb, la, lb, dx, dy, gamma, mu, kappa, Fl);
        const double rl = dt / (0.5 * (l == 0 ? dx : dy));
        for (int c = 0; c < 4; ++c) UL[c] -= rl * (Fr[c] - Fl[c]);
    }
    if (!admissible2(UL, gm1d)) f.bad = 1;
    const double thr = theta_fn(UL[0], UH[0], fmin(eps, UL[0]));
    double Ur[4];
    for (int c = 0; c < 4; ++c) Ur[c] = (1.0 - thr) * UL[c] + thr * UH[c];
    const double pL = gm1d * (UL[3] - (UL[1] * UL[1] + UL[2] * UL[2]) / (2.0 * UL[0]));
    const double pr = gm1d * (Ur[3] - (Ur[1] * Ur[1] + Ur[2] * Ur[2]) / (2.0 * Ur[0]));
    const double th = thr * theta_fn(pL, pr, fmin(eps, pL));
    for (int c = 0; c < 4; ++c) f.r[c] = (S)(((1.0 - th) * UL[c] + th * UH[c] - Ud[c]) / dt);
    f.blended = 1;
    return f;
}

// FP64 island of a cell centre whose FP32 screen did not clear it (Sec. 2.2,
// Remark 3.1): the Simpson inversion from the cell average ab, the edge points
// e0..e3 and the vertices v0..v3 in FP64, scaled toward the average when it is
// below epsilon. Out of line, like the point island.
template <class R>
__device__ __noinline__ V4<R> centre_island(V4<R> ab, V4<R> e0, V4<R> e1, V4<R> e2, V4<R> e3, V4<R> v0, V4<R> v1,
                                            V4<R> v2, V4<R> v3, double g1, double eps)
{
    double Ub[4], Ud[4];
    for (int c = 0; c < 4; ++c) {
        const double edges = (double)comp(e0, c) + (double)comp(e1, c) + (double)comp(e2, c) + (double)comp(e3, c);
        const double verts = (double)comp(v0, c) + (double)comp(v1, c) + (double)comp(v2, c) + (double)comp(v3, c);
        Ub[c] = (double)comp(ab, c);
        Ud[c] = (36.0 * Ub[c] - 4.0 * edges - verts) / 16.0;
    }
    const double pc = g1 * (Ud[3] - (Ud[1] * Ud[1] + Ud[2] * Ud[2]) / (2.0 * Ud[0]));
    if (!(Ud[0] >= eps) || !(pc >= eps)) {
        const double thr = theta_fn(Ub[0], Ud[0], fmin(eps, Ub[0]));
        double Ur[4];
        for (int c = 0; c < 4; ++c) Ur[c] = (1.0 - thr) * Ub[c] + thr * Ud[c];
        const double pL = g1 * (Ub[3] - (Ub[1] * Ub[1] + Ub[2] * Ub[2]) / (2.0 * Ub[0]));
        const double pH = g1 * (Ur[3] - (Ur[1] * Ur[1] + Ur[2] * Ur[2]) / (2.0 * Ur[0]));
        const double th = thr * theta_fn(pL, pH, fmin(eps, pL));
        for (int c = 0; c < 4; ++c) Ud[c] = (1.0 - th) * Ub[c] + th * Ud[c];
    }
    return V4<R>{(R)Ud[0], (R)Ud[1], (R)Ud[2], (R)Ud[3]};
}

// FP64 island of a face whose FP32 screen did not clear it (mixed path, Sec. 3.3):
// face_pp_fp64 on the face's low-order cell fluxes fL / fR, averages uL / uR and
// high-order flux fh; returns the limited flux, theta^rho theta^p and whether a
// low-order state left G.
template <class R>
struct FaceFix {
    R F[4];
    R tpp;
    int bad;
};
template <class R>
__device__ __noinline__ FaceFix<R> face_island(V4<R> fL, V4<R> fR, V4<R> uL, V4<R> uR, V4<R> fh, R lam, R ts,
                                               double kk, double g1, double eps)
{
    const double FLc[4] = {fL.x, fL.y, fL.z, fL.w}, FRc[4] = {fR.x, fR.y, fR.z, fR.w};
    const double UbL[4] = {uL.x, uL.y, uL.z, uL.w}, UbR[4] = {uR.x, uR.y, uR.z, uR.w};
    const double FH[4] = {fh.x, fh.y, fh.z, fh.w};
    double Fd[4], tpp = 1.0;
    bool bad = false;
    face_pp_fp64(FLc, FRc, UbL, UbR, (double)lam, (double)ts, FH, kk, g1, eps, Fd, &tpp, &bad);
    FaceFix<R> f;
    for (int c = 0; c < 4; ++c) f.F[c] = (R)Fd[c];
    f.tpp = (R)tpp;
    f.bad = bad ? 1 : 0;
    return f;
}

// The four TMA copies of tile (bx, by) into the staging area, one per DoF site:
// columns [i0-2, i0+TX+1], rows [j0-2, j0+TY+1], the site's 4 component planes.
template <class R, int TX, int TY>
__device__ __forceinline__ void tile_issue(const StageArgs &A, int bx, int by, R *stg, const void *tmap,
                                           uint64_t *bar)
{
    constexpr int BOX = 4 * (TX + 4) * (TY + 4);
    mbar_expect_tx(bar, (unsigned)(4 * BOX * sizeof(R)) + (unsigned)A.extra_tx);
    for (int site = 0; site < 4; ++site) tma_load_3d(stg + site * BOX, tmap, bx * TX, by * TY, 4 * site, bar);
}

// One tile of the stage. TMA path (persistent CTAs): `it` counts the tiles this
// CTA has done; the first call sets up the barrier, the per-launch constants and
// the copies of its own tile; every call copies the NEXT tile (nbx, nby; none if
// nbx < 0) into the staging area as soon as that area is free (after the point
// phase), so the copies land while the face and cell phases run. Returns false
// when the tile's copies did not land in time (reported in Ctl.err): the CTA
// stops. Several problems (the batched kernel): `ntmap` is the tensor map of the
// next tile's problem (null: the same map), and with `multi` every tile loads
// its problem's constants and starts its own restart flag. `rmap0` / `rmap2`
// / `rmapin` are the row maps (box: the tile's cell rows) of u^n, of the
// auxiliary state and of the stage input: the cell update's inputs from them
// (in FP32 also the compensation words of the input's cell averages) are
// copied by TMA once the point phase is done, so they land while the low-order
// and face phases run.
template <class R, class S, int TX, int TY, int NTH>
__device__ __forceinline__ bool stage_tile(const StageArgs &A, int bx, int by, V4<R> *sm, const void *tmap,
                                           int it, int nbx, int nby, const void *ntmap, bool multi,
                                           const void *rmap0, const void *rmap2, const void *rmapin)
{
    using T = Tile2<TX, TY>;
    using Q4 = V4<R>;
    constexpr int LX = T::LX, CX = T::CX, QX = T::QX;
    __shared__ int s_bad, s_stop;
    __shared__ TileConst<R> tc;
    __shared__ __align__(8) uint64_t s_bar, s_bar6;
    const Layout &L = A.L;
    const int i0 = bx * TX, j0 = by * TY;
    const int tid = threadIdx.x;
    constexpr int nth = NTH;
    const int ntx = min(TX, L.n1 - i0), nty = min(TY, L.n2 - j0);
    const double eps = A.eps;
    constexpr int NP = point_count<LX, T::LY>();
    Q4 *sU = sm + T::oU, *sQ = sm + T::oQ, *sGX = sm + T::oGX, *sGY = sm + T::oGY;
    Q4 *sA = sm + T::oA, *sCQ = sm + T::oCQ, *sFX = sm + T::oFX, *sFY = sm + T::oFY;
    const Q4 benign = {R(1), R(0), R(0), R(2.5)};

    // ---- P0: load point values and cell averages (two-node / two-cell halo)
    static_assert(sizeof(R) == sizeof(S), "tile and storage precision are the same");
    // the tile's four 3D tensor copies land in a staging area in the
    // gradient space (unused outside P3/P4); one pass turns the planes into
    // the 4-component node and cell records
    constexpr int BX = TX + 4, BY = TY + 4, BOX = 4 * BX * BY;
    static_assert(BX == CX && BY == T::CY, "the box is the cell frame");
    static_assert(4 * BOX * sizeof(R) + 128 <= (size_t)(T::NGX + T::NGY) * sizeof(Q4), "staging fits");
    R *stg = reinterpret_cast<R *>((reinterpret_cast<uintptr_t>(sm + T::oGX) + 127) & ~(uintptr_t)127);
    // gas constants of the transposition pass: from the per-launch constants
    // once they are in place (no FP64 instruction per tile); several
    // problems: from this tile's problem
    const bool fresh = it == 0 || multi;   // this tile loads its constants
    const R gm1_in = fresh ? (R)(A.gamma - 1.0) : tc.gm1, gam_in = fresh ? (R)A.gamma : tc.gam;
    if (it == 0) {
        if (tid == 0) {
            mbar_init(&s_bar, 1);
            mbar_init(&s_bar6, 1);
            s_stop = 0;
            s_bad = 0;
        }
        __syncthreads();
        if (tid == 0) tile_issue<R, TX, TY>(A, bx, by, stg, tmap, &s_bar);
    }
    // the point combination's inputs of this tile (the point sites of u^n and
    // of the auxiliary state, the tile's rows) are fetched into L2 now, so that
    // the point phase reads them at L2 latency
    if (tid == 0 && rmap0) {
        for (int site = 1; site < 4; ++site) {
            if (A.k.a0 != 0.0) tma_prefetch_l2_3d(rmap0, i0, j0 + 2, 4 * site);
            if (A.k.a2 != 0.0 || A.k.acc) tma_prefetch_l2_3d(rmap2, i0, j0 + 2, 4 * site);
        }
    }
    // while the copies are in flight: the constants (published by the
    // cp.async wait and the barrier after the transposition)
    if (fresh) load_tile_consts<R>(tc, A, tid);
    if (multi && tid == 0) s_bad = 0;
    // a copy that has not landed after 2 s is reported, not waited for forever
    if (!mbar_wait(&s_bar, (unsigned)(it & 1), 2000000000ull)) {
        atomicOr(&A.ctl->err, 1);
        s_stop = 1;
    }
    for (int t = tid; t < NP; t += nth) {
        int la, lb;
        point_node<LX>(t, la, lb);
        const int a = 2 * i0 - 2 + la, b = 2 * j0 - 2 + lb;
        const bool ea = (a & 1) == 0, eb = (b & 1) == 0;
        const int site = ea ? (eb ? 3 : 1) : 2;
        const int i = ea ? (a >> 1) : ((a - 1) >> 1);
        const int j = eb ? (b >> 1) : ((b - 1) >> 1);
        const R *g = stg + site * BOX + (j - j0 + 2) * BX + (i - i0 + 2);
        const Q4 U = (i <= L.n1 + 2 && j <= L.n2 + 2) ? Q4{g[0], g[BX * BY], g[2 * BX * BY], g[3 * BX * BY]}
                                                      : benign;
        sU[T::node(la, lb)] = U;
        // the point's primitives right away (the centres get theirs in P1)
        sQ[T::node(la, lb)] = node_prims(U, gm1_in, gam_in);
    }
    for (int t = tid; t < T::NCA; t += nth) {
        const int i = i0 - 2 + t % CX, j = j0 - 2 + t / CX;
        const R *g = stg + t;
        sA[t] = (i <= L.n1 + 2 && j <= L.n2 + 2) ? Q4{g[0], g[BX * BY], g[2 * BX * BY], g[3 * BX * BY]} : benign;
    }
    if (fresh) cp_async_wait_all();
    __syncthreads();
    if (s_stop) return false;
    const double dt = A.ctl->dt;
    const R gam = tc.gam, gm1 = tc.gm1, mu = tc.mu, ka = tc.ka;

    // ---- P1: cell centres (Simpson inversion, Sec. 2.2) + centre scaling limiter
    // (Remark 3.1), and the primitive quantities (u, v, T, c) of the centres (the
    // point nodes got theirs in P0)
    for (int t = tid; t < T::NCQ; t += nth) {
        const int qi = t % QX, qj = t / QX;
        // centre (2 qi + 1, 2 qj + 1); its x-neighbours 2 qi, 2 qi + 2 are the
        // consecutive records w, w + 1 of the row's even half
        const int n = T::node(2 * qi + 1, 2 * qj + 1);
        const int w = (2 * qj + 1) * LX + qi;
        const Q4 ab = sA[(qj + 1) * CX + (qi + 1)];
        const Q4 e0 = sU[w], e1 = sU[w + 1], e2 = sU[n - LX], e3 = sU[n + LX];
        const Q4 v0 = sU[w - LX], v1 = sU[w + 1 - LX], v2 = sU[w + LX], v3 = sU[w + 1 + LX];
        R Uc[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const R edges = comp(e0, c) + comp(e1, c) + comp(e2, c) + comp(e3, c);
            const R verts = comp(v0, c) + comp(v1, c) + comp(v2, c) + comp(v3, c);
            Uc[c] = (R(36) * comp(ab, c) - R(4) * edges - verts) / R(16);
        }
        if (A.limiter != LIM_NONE) {
            R mag[4];
#pragma unroll
            for (int c = 0; c < 4; ++c)
                mag[c] = R(4) * (fabs(comp(ab, c)) + fabs(comp(e0, c)) + fabs(comp(e1, c)) + fabs(comp(e2, c)) +
                                 fabs(comp(e3, c)));
            if (!surely_above(Uc, mag, gm1, tc.eps)) {
                const V4<R> cf = centre_island<R>(ab, e0, e1, e2, e3, v0, v1, v2, v3, A.gamma - 1.0, eps);
                Uc[0] = cf.x, Uc[1] = cf.y, Uc[2] = cf.z, Uc[3] = cf.w;
            }
        }
        const Q4 U = Q4{Uc[0], Uc[1], Uc[2], Uc[3]};
        sU[n] = U;
        sQ[n] = node_prims(U, gm1, gam);
    }
    __syncthreads();

    // ---- P3: D_c gradients (Eq. (8)) of Z = (u, v, T) along x (lattice columns
    // [2, LX-3]) and along y (rows [2, LY-3]), stored compactly as (v, u, T, 0)
    {
        const R i6x = tc.i6[0], i6y = tc.i6[1];
        for (int t = tid; t < T::NGX; t += nth) {
            const int lb = t / T::GXW, la = T::gxcol_inv(t - lb * T::GXW), row = lb * LX;
            const int n = T::node(la, lb);
            const Q4 a = sQ[n - 1], b = sQ[row + T::col(la - 1)], c = sQ[row + T::col(la + 1)], d = sQ[n + 1];
            sGX[t] = Q4{(a.y - R(8) * b.y + R(8) * c.y - d.y) * i6x, (a.x - R(8) * b.x + R(8) * c.x - d.x) * i6x,
                        (a.z - R(8) * b.z + R(8) * c.z - d.z) * i6x, R(0)};
        }
        for (int t = tid; t < T::NGY; t += nth) {
            const int n = 2 * LX + t;
            const Q4 a = sQ[n - 2 * LX], b = sQ[n - LX], c = sQ[n + LX], d = sQ[n + 2 * LX];
            sGY[t] = Q4{(a.y - R(8) * b.y + R(8) * c.y - d.y) * i6y, (a.x - R(8) * b.x + R(8) * c.x - d.x) * i6y,
                        (a.z - R(8) * b.z + R(8) * c.z - d.z) * i6y, R(0)};
        }
    }
    __syncthreads();

    // ---- P4: point residual, point scaling limiter (Sec. 3.4), RK combination, store
    {
        const bool perx = L.bc[0] == BC_PERIODIC, pery = L.bc[2] == BC_PERIODIC;
        const bool lastx = i0 + ntx == L.n1, lasty = j0 + nty == L.n2;
        const int ncell = ntx * nty, nreg = 3 * ncell;
        const int ecol = (lastx && !perx) ? 2 * nty : 0;
        const int erow = (lasty && !pery) ? 2 * ntx : 0;
        const int ecor = (lastx && !perx && lasty && !pery) ? 1 : 0;
        const int tot = nreg + ecol + erow + ecor;
        for (int t = tid; t < tot + T::NFX + T::NFY; t += nth) {
            if (t >= tot) {
                // high-order total face flux: Simpson over vertex, edge, vertex
                face_high_order<R, TX, TY>(sm, t - tot, ntx, nty, mu, ka);
                continue;
            }
            // own points, ordered so that neighbouring threads read neighbouring
            // lattice nodes: the even lattice rows (vertex, y-edge, vertex, ...)
            // as runs of 2 ntx consecutive nodes, then the x-edges of the odd rows
            int la, lb;
            if (t < nreg) {
                if (t < 2 * ncell) {
                    // an even row: its ntx vertices, then its ntx y-edges (a
                    // full-width tile divides by the constant TX)
                    const int rw = ntx == TX ? t / (2 * TX) : t / (2 * ntx), k = t - rw * (2 * ntx);
                    la = k < ntx ? 2 + 2 * k : 3 + 2 * (k - ntx);
                    lb = 2 + 2 * rw;
                } else {
                    const int cc = t - 2 * ncell, jl = ntx == TX ? cc / TX : cc / ntx;
                    la = 2 + 2 * (cc - jl * ntx);
                    lb = 3 + 2 * jl;
                }
            } else if (t < nreg + ecol) {
                la = 2 + 2 * ntx;
                lb = 2 + (t - nreg);
            } else if (t < nreg + ecol + erow) {
                lb = 2 + 2 * nty;
                la = 2 + (t - nreg - ecol);
            } else {
                la = 2 + 2 * ntx;
                lb = 2 + 2 * nty;
            }
            const int n = T::node(la, lb);
            // global position of the point; the combination inputs (u^n, the
            // auxiliary state) are loaded first so that their latency hides
            // behind the residual
            const int a = 2 * i0 - 2 + la, b = 2 * j0 - 2 + lb;
            const bool ea = (a & 1) == 0, eb = (b & 1) == 0;
            const int site = ea ? (eb ? 3 : 1) : 2;
            const long long po0 = plane_of(L, site, 0) + cell_off(L, ea ? (a >> 1) : ((a - 1) >> 1),
                                                                   eb ? (b >> 1) : ((b - 1) >> 1));
            S g0[4] = {S(0), S(0), S(0), S(0)}, g2[4] = {S(0), S(0), S(0), S(0)};
            if (tc.ua0) {
#pragma unroll
                for (int c = 0; c < 4; ++c) g0[c] = ((const S *)A.u0)[po0 + c * L.plane];
            }
            if (tc.ua2 || A.k.acc) {
#pragma unroll
                for (int c = 0; c < 4; ++c) g2[c] = ((const S *)A.aux)[po0 + c * L.plane];
            }
            R r[4];
            if constexpr (sizeof(R) == 4)
                point_residual_f32<TX, TY>(sm, la, lb, tc, r);
            else
                point_residual<R, TX, TY>(sm, la, lb, tc, r);
            if (A.source)
                r[3] += (R)tg_point_source(A.mu, A.kappa, A.gamma, L.lo[0], L.lo[1], L.dx, L.dy, a, b,
                                           A.ctl->t + A.k.ct * dt);
            // the RK combination of point values runs in the storage precision S
            const Q4 Un4 = sU[n];
            const R Un[4] = {Un4.x, Un4.y, Un4.z, Un4.w};
            S res[4] = {(S)r[0], (S)r[1], (S)r[2], (S)r[3]};
            S U[4] = {(S)Un[0], (S)Un[1], (S)Un[2], (S)Un[3]};
            if (A.limiter != LIM_NONE) {
                R UHr[4], mag[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    UHr[c] = Un[c] + tc.dt * r[c];
                    mag[c] = fabs(Un[c]) + fabs(tc.dt * r[c]);
                }
                if (!surely_above(UHr, mag, gm1, tc.eps)) {
                    const PointFix<S> f = point_island<R, S, TX, TY>(sm, la, lb, Un4, Q4{r[0], r[1], r[2], r[3]}, dt,
                                                                      eps, A.gamma, A.mu, A.kappa, L.dx, L.dy);
                    if (f.bad) s_bad = 1;
                    if (f.blended) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) res[c] = f.r[c];
                    }
                }
            }
            // store
            S o[4];
            const S ws = tc.w;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                S v = A.k.residual ? S(0) : tc.a1 * U[c];
                if (tc.ua0) v += tc.a0 * g0[c];
                if (tc.ua2) v += tc.a2 * g2[c];
                o[c] = v + ws * res[c];
                if (A.k.acc) ((S *)A.aux)[po0 + c * L.plane] = tc.b2 * g2[c] + tc.b1 * U[c] + tc.bldt * res[c];
            }
            if (A.k.wall_fix) {
                // wall point values: zero (normal) momentum, internal energy kept;
                // a moving wall sets the tangential momentum to rho U_w (sides in
                // order, so a corner takes the velocity of its y-side)
                for (int side = 0; side < 4; ++side) {
                    const int kind = L.bc[side];
                    if (kind != BC_WALL && kind != BC_SYMMETRY && kind != BC_MOVING) continue;
                    const int l = side >> 1;
                    const int pos = l == 0 ? a : b, lim = (side & 1) ? 2 * (l == 0 ? L.n1 : L.n2) : 0;
                    if (pos != lim) continue;
                    S ke0 = o[1] * o[1] + o[2] * o[2];
                    if (kind != BC_SYMMETRY || l == 0) o[1] = S(0);
                    if (kind != BC_SYMMETRY || l == 1) o[2] = S(0);
                    if (kind == BC_MOVING) o[2 - l] = (S)((double)o[0] * L.wall_speed[side]);
                    S ke1 = o[1] * o[1] + o[2] * o[2];
                    o[3] -= (ke0 - ke1) / (S(2) * o[0]);
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) ((S *)A.out)[po0 + c * L.plane] = o[c];
        }
    }

    // the lattice state, primitives and gradients are dead from here on: the
    // low-order cell records overwrite them, and the next tile's copies go to the
    // staging area (ordered after this tile's generic accesses to it)
    __syncthreads();
    // the cell update's inputs from u^n (stages 2-4) and from the auxiliary
    // state (stages 4-5): the tile's cell rows of the cell-average planes (and,
    // in FP32, of their compensation planes), by TMA into the dead lattice space
    // past the low-order cell records
    R *p6 = reinterpret_cast<R *>((reinterpret_cast<uintptr_t>(sm + T::oCQ + 4 * T::NCQ) + 127) & ~(uintptr_t)127);
    constexpr int P6W = TX + 4, P6BOX = 4 * P6W * TY, P6N = sizeof(S) == 4 ? 2 : 1;   // planes per input: hi (+ lo)
    static_assert((4 * T::NCQ + 8) * sizeof(Q4) + 2 * P6N * P6BOX * sizeof(R) <= 2 * (size_t)T::NL * sizeof(Q4),
                  "cell-update inputs fit in the lattice space");
    const bool in0 = tc.ua0, in2 = tc.ua2 || A.k.acc;
    // FP32: the compensation words of the input's cell averages, in the gradient
    // space past the staging area of the next tile's copies
    constexpr bool kLo = sizeof(S) == 4;
    const bool inlo = kLo && !A.k.residual;
    R *const plo = reinterpret_cast<R *>((reinterpret_cast<uintptr_t>(stg + 4 * BOX) + 127) & ~(uintptr_t)127);
    static_assert(!kLo || 256 + (4 * BOX + P6BOX) * sizeof(R) <= (size_t)(T::NGX + T::NGY) * sizeof(Q4),
                  "the input's compensation rows fit past the staging area");
    if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        if (nbx >= 0) tile_issue<R, TX, TY>(A, nbx, nby, stg, ntmap ? ntmap : tmap, &s_bar);
        const int nin = (in0 ? 1 : 0) + (in2 ? 1 : 0);
        mbar_expect_tx(&s_bar6, (unsigned)((nin * P6N + (inlo ? 1 : 0)) * P6BOX * sizeof(R)));
        for (int q = 0; q < P6N; ++q) {   // plane 16 + c holds the compensation word of component c
            if (in0) tma_load_3d(p6 + q * P6BOX, rmap0, i0, j0 + 2, 16 * q, &s_bar6);
            if (in2) tma_load_3d(p6 + (P6N + q) * P6BOX, rmap2, i0, j0 + 2, 16 * q, &s_bar6);
        }
        if (inlo) tma_load_3d(plo, rmapin, i0, j0 + 2, 16, &s_bar6);
    }

    // ---- P5a: low-order cell quantities (Sec. 3.1, 3.2) on cells [i0-1, i0+TX] x [j0-1, j0+TY]
    // FP64: the primitives (u, v, p, T) of every cell of the frame first, once
    // each, past the cell-update inputs (each cell's quantities need those of its
    // four neighbours, and a reciprocal costs many FP64 instructions; in FP32 it
    // is one approximate instruction and recomputing is cheaper than the records)
    Q4 *sW = reinterpret_cast<Q4 *>(p6 + 2 * P6N * P6BOX);
    if constexpr (sizeof(R) == 8) {
        static_assert((4 * T::NCQ + 8) * sizeof(Q4) + 2 * P6N * P6BOX * sizeof(R) + T::NCA * sizeof(Q4) <=
                          2 * (size_t)T::NL * sizeof(Q4),
                      "cell primitives fit in the lattice space");
        for (int t = tid; t < T::NCA; t += nth) sW[t] = cell_prims(sA[t], gm1);
        __syncthreads();
    }
    for (int t = tid; t < T::NCQ; t += nth) {
        const int ca = (t / QX + 1) * CX + (t % QX + 1);
        const Q4 U = sA[ca];
        Q4 W, We, Ww, Wn, Ws;
        if constexpr (sizeof(R) == 8) {
            W = sW[ca], We = sW[ca + 1], Ww = sW[ca - 1], Wn = sW[ca + CX], Ws = sW[ca - CX];
        } else {
            W = cell_prims(U, gm1), We = cell_prims(sA[ca + 1], gm1), Ww = cell_prims(sA[ca - 1], gm1);
            Wn = cell_prims(sA[ca + CX], gm1), Ws = cell_prims(sA[ca - CX], gm1);
        }
        const R i2x = tc.i2[0], i2y = tc.i2[1];
        const R Sxu = (We.x - Ww.x) * i2x, Sxv = (We.y - Ww.y) * i2x, SxT = (We.w - Ww.w) * i2x;
        const R Syu = (Wn.x - Ws.x) * i2y, Syv = (Wn.y - Ws.y) * i2y, SyT = (Wn.w - Ws.w) * i2y;
        const R rho = U.x, u = W.x, v = W.y, p = W.z, Tc = W.w;
        R Fx[4], Fy[4];
        node_flux<R>(0, rho, U.y, U.z, U.w, u, v, Tc, Sxu, Sxv, SxT, Syu, Syv, SyT, mu, ka, Fx);
        node_flux<R>(1, rho, U.y, U.z, U.w, u, v, Tc, Sxu, Sxv, SxT, Syu, Syv, SyT, mu, ka, Fy);
        const R cs = fsqrt(gam * Tc);
        // Lemma 3.2 bound b_l with tau_l = (tau_1l, tau_2l), q_l = -kappa dT/dx_l
        const R div = Sxu + Syv;
        const R txx = mu * (R(2) * Sxu - R(2) / R(3) * div), tyy = mu * (R(2) * Syv - R(2) / R(3) * div);
        const R txy = mu * (Syu + Sxv);
        const R re = p / gm1;
        const R qx = -ka * SxT, qy = -ka * SyT;
        const R ib = frcp(R(2) * rho * re);
        const R bx = (fsqrt(rho * rho * qx * qx + R(2) * rho * re * (txx * txx + txy * txy)) + rho * fabs(qx)) * ib;
        const R by = (fsqrt(rho * rho * qy * qy + R(2) * rho * re * (txy * txy + tyy * tyy)) + rho * fabs(qy)) * ib;
        // Sec. 3.2 sensors: the larger of the two pressure ratios (FP64: one
        // division, the ratios compared by cross-multiplication)
        const R ax = fabs(We.z - R(2) * p + Ww.z), bxs = fabs(We.z + R(2) * p + Ww.z);
        const R ay = fabs(Wn.z - R(2) * p + Ws.z), bys = fabs(Wn.z + R(2) * p + Ws.z);
        R pxy;
        if constexpr (sizeof(R) == 8)
            pxy = ax * bys >= ay * bxs ? ax / bxs : ay / bys;
        else
            pxy = dmax(ax * frcp(bxs), ay * frcp(bys));
        const R curl = Sxv - Syu;
        const R ph2 = -div * frsqrt(div * div + curl * curl + R(1e-13));
        sCQ[CQ_FX * T::NCQ + t] = Q4{Fx[0], Fx[1], Fx[2], Fx[3]};
        sCQ[CQ_FY * T::NCQ + t] = Q4{Fy[0], Fy[1], Fy[2], Fy[3]};
        sCQ[CQ_RB * T::NCQ + t] = Q4{fabs(u) + cs, fabs(v) + cs, bx, by};
        sCQ[CQ_PH * T::NCQ + t] = Q4{pxy, dmax(ph2, R(0)), R(0), R(0)};
    }
    __syncthreads();

    // ---- P5b: face fluxes: high order (Simpson), low order (Eq. (19)), theta_s
    // (Eq. (22)), theta^rho theta^p (Sec. 3.3)
    {
        const long long nfx = (long long)(L.n1 + 1) * L.n2;
        for (int t = tid; t < T::NFX + T::NFY; t += nth) {
            int l, fl, el;   // direction, face index along l (local), index along the face (local)
            if (t < T::NFX) {
                l = 0;
                fl = t % (TX + 1);
                el = t / (TX + 1);
                if (fl > ntx || el >= nty) continue;
            } else {
                l = 1;
                const int u_ = t - T::NFX;
                el = u_ % TX;
                fl = u_ / TX;
                if (el >= ntx || fl > nty) continue;
            }
            // high-order total flux of P4; the limited flux replaces it in place
            Q4 *fslot = l == 0 ? sFX + el * (TX + 1) + fl : sFY + fl * TX + el;
            const Q4 fh4 = *fslot;
            const R FH[4] = {fh4.x, fh4.y, fh4.z, fh4.w};
            R Fout[4];
            R tsr = R(1), tppr = R(1);
            if (A.limiter == LIM_NONE) {
                for (int c = 0; c < 4; ++c) Fout[c] = FH[c];
            } else {
                // cells L (before the face) and R (after), in the NCQ and NCA frames
                int qL, qR, aL, aR;
                if (l == 0) {
                    qL = (el + 1) * QX + fl;
                    qR = qL + 1;
                    aL = (el + 2) * CX + fl + 1;
                    aR = aL + 1;
                } else {
                    qL = fl * QX + el + 1;
                    qR = qL + QX;
                    aL = (fl + 1) * CX + el + 2;
                    aR = aL + CX;
                }
                const int fo = l == 0 ? CQ_FX : CQ_FY;
                const Q4 fL4 = sCQ[fo * T::NCQ + qL], fR4 = sCQ[fo * T::NCQ + qR];
                const Q4 rbL = sCQ[CQ_RB * T::NCQ + qL], rbR = sCQ[CQ_RB * T::NCQ + qR];
                const Q4 uL4 = sA[aL], uR4 = sA[aR];
                const R FLc[4] = {fL4.x, fL4.y, fL4.z, fL4.w}, FRc[4] = {fR4.x, fR4.y, fR4.z, fR4.w};
                const R UbL[4] = {uL4.x, uL4.y, uL4.z, uL4.w}, UbR[4] = {uR4.x, uR4.y, uR4.z, uR4.w};
                const R lam = l == 0 ? dmax(rbL.x, rbR.x) + dmax(rbL.z, rbR.z) : dmax(rbL.y, rbR.y) + dmax(rbL.w, rbR.w);
                if (A.limiter == LIM_S_PP) {
                    const Q4 phL = sCQ[CQ_PH * T::NCQ + qL], phR = sCQ[CQ_PH * T::NCQ + qR];
                    tsr = fexp(-tc.cs * dmax(phL.x, phR.x) * dmax(phL.y, phR.y));
                }
                bool done = false;
                if constexpr (sizeof(R) == 4) {
                    // FP32 screen: when all four intermediate states of Eq. (20) and
                    // Sec. 3.3 are surely above epsilon, theta^rho = theta^p = 1 and no
                    // low-order state leaves G, so the FP64 island is skipped.
                    const R kk = l == 0 ? tc.kkx : tc.kky;
                    R FL[4], FLs[4], mag[4], ULp[4], UHp[4], ULm[4], UHm[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        FL[c] = R(0.5) * (FLc[c] + FRc[c]) - R(0.5) * lam * (UbR[c] - UbL[c]);
                        FLs[c] = FL[c] + tsr * (FH[c] - FL[c]);
                        mag[c] = fabs(UbL[c]) + fabs(UbR[c]) +
                                 kk * (fabs(FLc[c]) + fabs(FRc[c]) + lam * (fabs(UbL[c]) + fabs(UbR[c])) + fabs(FH[c]));
                        ULp[c] = UbL[c] - kk * (FL[c] - FLc[c]);
                        UHp[c] = UbL[c] - kk * (FLs[c] - FLc[c]);
                        ULm[c] = UbR[c] - kk * (FRc[c] - FL[c]);
                        UHm[c] = UbR[c] - kk * (FRc[c] - FLs[c]);
                    }
                    if (surely_above(ULp, mag, gm1, tc.eps) && surely_above(UHp, mag, gm1, tc.eps) &&
                        surely_above(ULm, mag, gm1, tc.eps) && surely_above(UHm, mag, gm1, tc.eps)) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) Fout[c] = FLs[c];
                        done = true;
                    }
                }
                if constexpr (sizeof(R) == 4) {
                    if (!done) {
                        const FaceFix<R> f = face_island<R>(fL4, fR4, uL4, uR4, fh4, lam, tsr,
                                                            4.0 * dt / (l == 0 ? L.dx : L.dy), A.gamma - 1.0, eps);
                        if (f.bad) s_bad = 1;
#pragma unroll
                        for (int c = 0; c < 4; ++c) Fout[c] = f.F[c];
                        tppr = f.tpp;
                        done = true;
                    }
                }
                if (!done) {
                    // FP64 island: intermediate states (factor 2 d mu_l, d = 2), theta^rho, theta^p
                    double FLcd[4], FRcd[4], UbLd[4], UbRd[4], FHd[4], Fd[4], tppd = 1.0;
                    for (int c = 0; c < 4; ++c) {
                        FLcd[c] = FLc[c], FRcd[c] = FRc[c], UbLd[c] = UbL[c], UbRd[c] = UbR[c], FHd[c] = FH[c];
                    }
                    bool bad = false;
                    face_pp_fp64(FLcd, FRcd, UbLd, UbRd, (double)lam, (double)tsr, FHd,
                                 4.0 * dt / (l == 0 ? L.dx : L.dy), A.gamma - 1.0, eps, Fd, &tppd, &bad);
                    if (bad) s_bad = 1;
                    for (int c = 0; c < 4; ++c) Fout[c] = (R)Fd[c];
                    tppr = (R)tppd;
                }
            }
            *fslot = Q4{Fout[0], Fout[1], Fout[2], Fout[3]};
            if (A.theta) {
                const int gf = l == 0 ? i0 + fl : j0 + fl;   // global face index along l
                const int ge = l == 0 ? j0 + el : i0 + el;
                const bool own = l == 0 ? (fl < ntx || gf == L.n1) : (fl < nty || gf == L.n2);
                if (own) {
                    const long long id = l == 0 ? (long long)ge * (L.n1 + 1) + gf : nfx + (long long)gf * L.n1 + ge;
                    const long long nft = nfx + (long long)L.n1 * (L.n2 + 1);
                    A.theta[id] = (double)tsr;
                    A.theta[nft + id] = (double)tppr;
                }
            }
        }
    }
    __syncthreads();

    // ---- P6: cell residual (flux differences, Eq. (23)), RK combination, store
    // (its u^n and auxiliary inputs landed in p6: [input][plane][row][col], the
    // columns from i0 - 2)
    if (!mbar_wait(&s_bar6, (unsigned)(it & 1), 2000000000ull)) {
        atomicOr(&A.ctl->err, 1);
        return false;
    }
    const R *p6u0 = p6, *p6aux = p6 + P6N * P6BOX;
    S cfl1 = S(0), cfl2 = S(0);   // CFL maxima of the output cell averages (k.cfl_out)
    if constexpr (sizeof(S) == 8) {
        const double w = A.k.residual ? 1.0 : A.k.cl * dt;
        const double idx = L.idx[0], idy = L.idx[1];
        for (int t = tid; t < ntx * nty; t += nth) {
            const int jl = ntx == TX ? t / TX : t / ntx, il = t - jl * ntx;
            const Q4 fxr = sFX[jl * (TX + 1) + il + 1], fxl = sFX[jl * (TX + 1) + il];
            const Q4 fyt = sFY[(jl + 1) * TX + il], fyb = sFY[jl * TX + il];
            const Q4 ui = sA[(jl + 2) * CX + (il + 2)];
            const long long po0 = plane_of(L, 0, 0) + cell_off(L, i0 + il, j0 + jl);
            const int q6 = jl * P6W + il + 2;
            double g0[4] = {0, 0, 0, 0}, g2[4] = {0, 0, 0, 0};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (in0) g0[c] = p6u0[c * P6W * TY + q6];
                if (in2) g2[c] = p6aux[c * P6W * TY + q6];
            }
            const double src = A.source ? tg_cell_source(A.mu, A.kappa, A.gamma, L.lo[0], L.lo[1], L.dx, L.dy,
                                                         i0 + il, j0 + jl, A.ctl->t + A.k.ct * dt)
                                        : 0.0;
            S o4[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                double res =
                    -((double)comp(fxr, c) - (double)comp(fxl, c)) * idx - ((double)comp(fyt, c) - (double)comp(fyb, c)) * idy;
                if (c == 3 && A.source) res += src;
                const long long po = po0 + c * L.plane;
                const double Uin = comp(ui, c);
                double v = A.k.residual ? 0.0 : A.k.a1 * Uin;
                if (tc.ua0) v += A.k.a0 * g0[c];
                if (tc.ua2) v += A.k.a2 * g2[c];
                if (A.k.acc) {
                    const double ac = A.k.b2 * g2[c] + A.k.b1 * Uin + A.k.bl * dt * res;
                    ((S *)A.aux)[po] = (S)ac;
                }
                o4[c] = (S)(v + w * res);
                ((S *)A.out)[po] = o4[c];
            }
            if (A.k.cfl_out) cfl_terms(A.cfl, o4[0], o4[1], o4[2], o4[3], cfl1, cfl2);
        }
    } else {
        // mixed precision: cell averages are stored as hi + lo (float-float); the
        // flux differences are formed exactly and the combination is compensated,
        // so the update is conservative to far below FP32 roundoff
        const float fidx = tc.idx, fidy = tc.idy;
        const ff a0 = tc.fa0, a1 = tc.fa1, a2 = tc.fa2, wx = tc.fwx, wy = tc.fwy;
        const ff b1 = tc.fb1, b2 = tc.fb2, bx = tc.fbx, by = tc.fby;
        float *out = (float *)A.out;
        float *aux = (float *)A.aux;
        for (int t = tid; t < ntx * nty; t += nth) {
            const int jl = ntx == TX ? t / TX : t / ntx, il = t - jl * ntx;
            const long long off = cell_off(L, i0 + il, j0 + jl);
            float o4[4] = {1.f, 0.f, 0.f, 1.f};
            // the compensation words of the input (landed in plo), u^n and the
            // auxiliary state (landed in p6)
            const int q6 = jl * P6W + il + 2;
            float ulo[4], g0h[4], g0l[4], g2h[4], g2l[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                ulo[c] = inlo ? plo[c * P6W * TY + q6] : 0.f;
                g0h[c] = in0 ? p6u0[c * P6W * TY + q6] : 0.f;
                g0l[c] = in0 ? p6u0[P6BOX + c * P6W * TY + q6] : 0.f;
                g2h[c] = in2 ? p6aux[c * P6W * TY + q6] : 0.f;
                g2l[c] = in2 ? p6aux[P6BOX + c * P6W * TY + q6] : 0.f;
            }
            const Q4 fxr = sFX[jl * (TX + 1) + il + 1], fxl = sFX[jl * (TX + 1) + il];
            const Q4 fyt = sFY[(jl + 1) * TX + il], fyb = sFY[jl * TX + il];
            const Q4 ui = sA[(jl + 2) * CX + (il + 2)];
            // manufactured energy source (FP64, only when enabled): its weighted
            // contributions enter the compensated sums as float-float values
            float src_f = 0.f;
            ff src_inc = {0.f, 0.f}, src_acc = {0.f, 0.f};
            if (A.source) {
                const double src = tg_cell_source(A.mu, A.kappa, A.gamma, L.lo[0], L.lo[1], L.dx, L.dy, i0 + il,
                                                  j0 + jl, A.ctl->t + A.k.ct * dt);
                src_f = (float)src;
                src_inc = ff_from(A.k.cl * dt * src);
                src_acc = ff_from(A.k.bl * dt * src);
            }
            if (!A.source && !A.k.residual) {
                // components in pairs (rho, m_x), (m_y, E) through two-lane FP32
                // instructions: the same float-float operations lane by lane
#pragma unroll
                for (int hp = 0; hp < 2; ++hp) {
                    const int c = 2 * hp;
                    const float2 fr = hp ? zw2(fxr) : xy2(fxr), fl = hp ? zw2(fxl) : xy2(fxl);
                    const float2 ft = hp ? zw2(fyt) : xy2(fyt), fb = hp ? zw2(fyb) : xy2(fyb);
                    const ff2 dxf = ff2_two_sum(fl, neg2(fr)), dyf = ff2_two_sum(fb, neg2(ft));   // exact
                    const ff2 inc = ff2_add(ff2_mul(wx, dxf), ff2_mul(wy, dyf));
                    const ff2 uv = {hp ? zw2(ui) : xy2(ui), make_float2(ulo[c], ulo[c + 1])};
                    const ff2 g0 = {make_float2(g0h[c], g0h[c + 1]), make_float2(g0l[c], g0l[c + 1])};
                    const ff2 g2 = {make_float2(g2h[c], g2h[c + 1]), make_float2(g2l[c], g2l[c + 1])};
                    ff2 v = ff2_mul(a1, uv);
                    if (tc.ua0) v = ff2_add(v, ff2_mul(a0, g0));
                    if (tc.ua2) v = ff2_add(v, ff2_mul(a2, g2));
                    if (A.k.acc) {
                        ff2 ac = ff2_add(ff2_mul(b2, g2), ff2_mul(b1, uv));
                        ac = ff2_add(ac, ff2_add(ff2_mul(bx, dxf), ff2_mul(by, dyf)));
                        aux[plane_of(L, 0, c) + off] = ac.h.x;
                        aux[comp_plane(L, c) + off] = ac.l.x;
                        aux[plane_of(L, 0, c + 1) + off] = ac.h.y;
                        aux[comp_plane(L, c + 1) + off] = ac.l.y;
                    }
                    v = ff2_add(v, inc);
                    out[plane_of(L, 0, c) + off] = v.h.x;
                    out[comp_plane(L, c) + off] = v.l.x;
                    out[plane_of(L, 0, c + 1) + off] = v.h.y;
                    out[comp_plane(L, c + 1) + off] = v.l.y;
                    o4[c] = v.h.x;
                    o4[c + 1] = v.h.y;
                }
                if (A.k.cfl_out) cfl_terms(A.cfl, o4[0], o4[1], o4[2], o4[3], cfl1, cfl2);
                continue;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float fr = comp(fxr, c), fl = comp(fxl, c), ft = comp(fyt, c), fb = comp(fyb, c);
                const long long po = plane_of(L, 0, c) + off, pl = comp_plane(L, c) + off;
                const bool has_src = c == 3 && A.source;
                if (A.k.residual) {
                    out[po] = -(fr - fl) * fidx - (ft - fb) * fidy + (has_src ? src_f : 0.f);
                    out[pl] = 0.f;
                    continue;
                }
                const ff dxf = ff_two_sum(fl, -fr), dyf = ff_two_sum(fb, -ft);   // exact
                ff inc = ff_add(ff_mul(wx, dxf), ff_mul(wy, dyf));
                if (has_src) inc = ff_add(inc, src_inc);
                const ff uv = {(float)comp(ui, c), ulo[c]};
                ff v = ff_mul(a1, uv);
                if (tc.ua0) v = ff_add(v, ff_mul(a0, ff{g0h[c], g0l[c]}));
                if (tc.ua2) v = ff_add(v, ff_mul(a2, ff{g2h[c], g2l[c]}));
                if (A.k.acc) {
                    ff ac = ff_add(ff_mul(b2, ff{g2h[c], g2l[c]}), ff_mul(b1, uv));
                    ac = ff_add(ac, ff_add(ff_mul(bx, dxf), ff_mul(by, dyf)));
                    if (has_src) ac = ff_add(ac, src_acc);
                    aux[po] = ac.h;
                    aux[pl] = ac.l;
                }
                v = ff_add(v, inc);
                out[po] = v.h;
                out[pl] = v.l;
                o4[c] = v.h;
            }
            if (A.k.cfl_out) cfl_terms(A.cfl, o4[0], o4[1], o4[2], o4[3], cfl1, cfl2);
        }
    }
    if (A.k.cfl_out) {
        // merge the tile's maxima: warp, then one atomic per warp (non-negative
        // doubles order like their bit patterns)
        double m1 = cfl1, m2 = cfl2;
        for (int o = 16; o > 0; o >>= 1) {
            m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
            m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
        }
        if ((tid & 31) == 0) {
            atomicMax(&A.ctl->cfl_mx[0], (unsigned long long)__double_as_longlong(m1));
            atomicMax(&A.ctl->cfl_mx[1], (unsigned long long)__double_as_longlong(m2));
        }
    }
    if (tid == 0 && s_bad) atomicOr(&A.ctl->notpp, 1);
    return true;
}

// Resident CTAs per SM that the register budget must allow: as many as the
// tile's shared memory admits (228 KB per SM, 1 KB reserved per CTA, static
// shared variables), but never fewer registers per thread than the kernel needs
// without heavy spilling (128 in FP32, 200 in FP64). FP32 16x8: four CTAs of
// 128 threads or two of 256; FP32 32x8: two; FP64 16x8: two of 128, one of 256.
template <class R, int TX, int TY, int NTH>
constexpr int stage_min_ctas()
{
    constexpr int by_smem = 233472 / (int)(Tile2<TX, TY>::template bytes<R>() + 1024 + 512);
    constexpr int by_regs = 65536 / (NTH * (sizeof(R) == 8 ? 200 : 128));
    constexpr int m = by_smem < by_regs ? by_smem : by_regs;
    return m < 1 ? 1 : m;
}

// Persistent CTAs (as many as fit on the GPU at once) walk the tiles in steps
// of the grid size, x fastest; tiles are loaded by TMA through the tensor map of
// the stage input (a 3D map: x = element of a row, y = row, z = plane), each
// tile's copies issued while the previous tile finishes.
template <class R, class S, int TX, int TY, int NTH>
__global__ void __launch_bounds__(NTH, stage_min_ctas<R, TX, TY, NTH>())
    k_stage2d(StageArgs A, const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap rmap0,
              const __grid_constant__ CUtensorMap rmap2, const __grid_constant__ CUtensorMap rmapin)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int tiles_x = (A.L.n1 + TX - 1) / TX, ntiles = tiles_x * ((A.L.n2 + TY - 1) / TY);
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int tn = t + gridDim.x;
        const bool more = tn < ntiles;
        if (!stage_tile<R, S, TX, TY, NTH>(A, t % tiles_x, t / tiles_x, reinterpret_cast<V4<R> *>(smem_raw),
                                           &tmap, it, more ? tn % tiles_x : -1, more ? tn / tiles_x : -1, nullptr,
                                           false, &rmap0, &rmap2, &rmapin))
            break;
        // the next tile's records overwrite this tile's
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// CFL time step of Eq. (13): per-block maxima, then one finalising block.
// ---------------------------------------------------------------------------
// Cell (i, j) of linear cell index t (x fastest); 32-bit division when the grid
// allows it (64-bit division is a long instruction sequence).
__device__ __forceinline__ void cell_ij(const Layout &L, long long t, bool small, int &i, int &j)
{
    if (small) {
        const int tt = (int)t;
        j = tt / L.n1;
        i = tt - j * L.n1;
    } else {
        j = (int)(t / L.n1);
        i = (int)(t - (long long)j * L.n1);
    }
}

// Per-block maxima of the two terms of Eq. (13) over the cell averages. Each
// thread takes DT_UNROLL cells a block width apart (coalesced) and issues all of
// their loads before any arithmetic, so that enough loads are in flight to
// stream the four cell-average planes at HBM speed.
constexpr int DT_UNROLL = 4;
template <class S>
__global__ void k_dt_partial2d(Layout L, const S *buf, CflConst k, double *partial)
{
    const long long nc = (long long)L.n1 * L.n2;
    const bool small = nc < (1ll << 31);   // 32-bit index arithmetic suffices
    const long long stride = (long long)gridDim.x * blockDim.x * DT_UNROLL;
    S f1 = 0, f2 = 0;
    for (long long t0 = (long long)blockIdx.x * blockDim.x * DT_UNROLL + threadIdx.x; t0 < nc; t0 += stride) {
        S rho[DT_UNROLL], mx[DT_UNROLL], my[DT_UNROLL], E[DT_UNROLL];
#pragma unroll
        for (int u = 0; u < DT_UNROLL; ++u) {
            const long long t = t0 + (long long)u * blockDim.x;
            rho[u] = S(1), mx[u] = S(0), my[u] = S(0), E[u] = S(0);
            if (t < nc) {
                int i, j;
                cell_ij(L, t, small, i, j);
                const long long off = cell_off(L, i, j);
                rho[u] = buf[plane_of(L, 0, 0) + off], mx[u] = buf[plane_of(L, 0, 1) + off];
                my[u] = buf[plane_of(L, 0, 2) + off], E[u] = buf[plane_of(L, 0, 3) + off];
            }
        }
#pragma unroll
        for (int u = 0; u < DT_UNROLL; ++u)
            if (t0 + (long long)u * blockDim.x < nc) cfl_terms(k, rho[u], mx[u], my[u], E[u], f1, f2);
    }
    double m1 = f1, m2 = f2;
    for (int o = 16; o > 0; o >>= 1) {
        m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    }
    __shared__ double s1[32], s2[32];
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) s1[wid] = m1, s2[wid] = m2;
    __syncthreads();
    if (wid == 0) {
        int nw = (blockDim.x + 31) >> 5;
        m1 = lane < nw ? s1[lane] : 0.0;
        m2 = lane < nw ? s2[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
            m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
        }
        if (lane == 0) partial[2 * blockIdx.x] = m1, partial[2 * blockIdx.x + 1] = m2;
    }
}

static __global__ void k_dt_final(const double *partial, int nparts, Ctl *ctl, int clip)
{
    double m1 = 0.0, m2 = 0.0;
    for (int t = threadIdx.x; t < nparts; t += blockDim.x) {
        m1 = fmax(m1, partial[2 * t]);
        m2 = fmax(m2, partial[2 * t + 1]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    }
    __shared__ double s1[32], s2[32];
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) s1[wid] = m1, s2[wid] = m2;
    __syncthreads();
    if (threadIdx.x == 0) {
        int nw = (blockDim.x + 31) >> 5;
        for (int k = 1; k < nw; ++k) m1 = fmax(m1, s1[k]), m2 = fmax(m2, s2[k]);
        double dt = 1.0 / (m1 + m2);
        ctl->dt_cfl = dt;
        if (clip && ctl->t_end > ctl->t && ctl->t + dt > ctl->t_end) dt = ctl->t_end - ctl->t;
        ctl->dt = dt;
        ctl->notpp = 0;
    }
}

// ---------------------------------------------------------------------------
// Validation of a freshly set state: admissible DoFs and periodic duplicates.
// flag bit 0: inadmissible DoF, bit 1: periodic duplicate mismatch.
// ---------------------------------------------------------------------------
template <class S>
__global__ void k_validate2d(Layout L, const S *buf, double gamma, int *flag)
{
    const int n1 = L.n1, n2 = L.n2;
    const long long per_site[4] = {(long long)n1 * n2, (long long)(n1 + 1) * n2, (long long)n1 * (n2 + 1),
                                   (long long)(n1 + 1) * (n2 + 1)};
    const long long total = per_site[0] + per_site[1] + per_site[2] + per_site[3];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        long long r = t;
        int site = 0;
        while (r >= per_site[site]) r -= per_site[site++];
        int w = (site == 1 || site == 3) ? n1 + 1 : n1;
        int i = (int)(r % w), j = (int)(r / w);
        long long off = cell_off(L, i, j);
        double U[4];
        for (int c = 0; c < 4; ++c) U[c] = (double)buf[plane_of(L, site, c) + off];
        if (!admissible_input2(U)) atomicOr(flag, 1);
        bool ptx = site == 1 || site == 3, pty = site == 2 || site == 3;
        int si = i, sj = j;
        if (ptx && i == n1 && L.bc[0] == BC_PERIODIC) si = 0;
        if (pty && j == n2 && L.bc[2] == BC_PERIODIC) sj = 0;
        if (si != i || sj != j) {
            long long o2 = cell_off(L, si, sj);
            for (int c = 0; c < 4; ++c)
                if (buf[plane_of(L, site, c) + off] != buf[plane_of(L, site, c) + o2]) atomicOr(flag, 2);
        }
    }
}

}  // namespace afns
