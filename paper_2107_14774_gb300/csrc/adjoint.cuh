// adjoint.cuh -- reverse-mode (vector-Jacobian) form of the per-node collision
// of collide.cuh and the kernels of the discrete adjoint of the fused
// collide-and-stream update.
//
// Forward map of one step (pull convention): f^{n+1}_a(x) = g^n_a(x - e_a) with
// g^n(x) = C(f^n(x); F(x), omega_nu, omega_xi) the collision of Sec. 3.2 / App. D,
// or g^n_opp(a)(x) across a wall.  For an objective J(f^T, F) the adjoint is
//   lambda_g^n_a(x) = lambda^{n+1}_a(x + e_a)      (transposed streaming;
//                   = lambda^{n+1}_opp(a)(x)         across a wall)
//   lambda^n(x)     = (dC/df)^T lambda_g^n(x)
//   dJ/dF(x)       += (dC/dF)^T lambda_g^n(x),   dJ/domega += sum_x (dC/domega)^T lambda_g^n(x).
// The VJP below recomputes the forward intermediates of one node and walks them
// back in reverse order; every line is the transpose of one line of
// raw_moments / relax_node / back_transform.
#pragma once

#include "kernels.cuh"

namespace lbc {

template <class T>
struct RelaxBar {
    RawMoments<T> m;   // d/d raw moments
    T Fx, Fy, Fz;      // d/d body force
    T wn, wb;          // d/d omega_nu, omega_xi
};

// Reverse of relax_node<T, CORR> (CORR != FULL).  ob: adjoints of the PostState.
template <class T, int CORR>
__device__ __forceinline__ RelaxBar<T> relax_node_vjp(const RawMoments<T> &m, const Phys<T> &P, T Fx, T Fy, T Fz,
                                                      const PostState<T> &ob)
{
    static_assert(CORR != LB_CORR_FULL, "the adjoint covers the local correction modes");
    // ---- forward recomputation ----
    const T dr = m.dr;
    const T rho = T(1) + dr;
    const T irho = div_(T(1), rho);
    const T qx = m.jx + T(0.5) * Fx, qy = m.jy + T(0.5) * Fy, qz = m.jz + T(0.5) * Fz;
    const T ux = qx * irho, uy = qy * irho, uz = qz * irho;
    const T n200 = m.pxx - P.cs2ax[0] * dr - rho * ux * ux + ux * Fx;
    const T n020 = m.pyy - P.cs2ax[1] * dr - rho * uy * uy + uy * Fy;
    const T n002 = m.pzz - P.cs2ax[2] * dr - rho * uz * uz + uz * Fz;
    const T k110 = m.pxy - rho * ux * uy + T(0.5) * (ux * Fy + uy * Fx);
    const T k101 = m.pxz - rho * ux * uz + T(0.5) * (ux * Fz + uz * Fx);
    const T k011 = m.pyz - rho * uy * uz + T(0.5) * (uy * Fz + uz * Fy);
    const T N2s = n200 + n020 + n002;
    const T k2d1 = n200 - n020;
    const T k2d2 = n200 - n002;
    const T al = (CORR == LB_CORR_LOWMACH) ? T(0) : T(1);
    const T ux2 = al * ux * ux, uy2 = al * uy * uy, uz2 = al * uz * uz;
    const T c2n = P.two_cs2_wn, c2b = P.two_cs2_wb;
    const T hx = T(0.5) * P.an[0] + T(1.5) * ux2;
    const T hy = T(0.5) * P.an[1] + T(1.5) * uy2;
    const T hz = T(0.5) * P.an[2] + T(1.5) * uz2;
    const T Csx = (hx - c2n) * rho, Cbx = (hx - c2b) * rho;
    const T Csy = (c2n - hy) * rho, Cby = (hy - c2b) * rho;
    const T Csz = (c2n - hz) * rho, Cbz = (hz - c2b) * rho;
    const T Rb = N2s, Rs1 = k2d1, Rs2 = k2d2;
    const T num = -Csz * Cby * Rs1 - Csy * (Cbz * Rs2 - Csz * Rb);
    const T den = -Csx * Csz * Cby - Csy * (Csx * Cbz - Csz * Cbx);
    const T X = div_(num, den);
    const T yn = Rs1 - Csx * X, zn = Rs2 - Csx * X;
    const T Y = div_(yn, Csy), Z = div_(zn, Csz);
    const T qxx = -rho * (T(3) * ux2 + P.an[0]);
    const T qyy = -rho * (T(3) * uy2 + P.an[1]);
    const T qzz = -rho * (T(3) * uz2 + P.an[2]);
    T E2s = T(0), E2d1 = T(0), E2d2 = T(0);
    if (CORR != LB_CORR_NONE) {
        E2s = P.tb * (qxx * X + qyy * Y + qzz * Z);
        E2d1 = P.tn * (qxx * X - qyy * Y);
        E2d2 = P.tn * (qxx * X - qzz * Z);
    }
    const T wn = P.wn, wb = P.wb;
    const T om = T(1) - wn;

    // ---- reverse sweep ----
    RelaxBar<T> b;
    T Fx_b = T(0.5) * ob.hFx, Fy_b = T(0.5) * ob.hFy, Fz_b = T(0.5) * ob.hFz;
    const T third = T(1) / T(3);
    const T t2s_b = (ob.d200 + ob.d020 + ob.d002) * third;
    const T t2d1_b = (ob.d200 - T(2) * ob.d020 + ob.d002) * third;
    const T t2d2_b = (ob.d200 + ob.d020 - T(2) * ob.d002) * third;
    T k110_b = om * ob.t110, k101_b = om * ob.t101, k011_b = om * ob.t011;
    T wn_b = -(ob.t110 * k110 + ob.t101 * k101 + ob.t011 * k011);
    T wb_b = T(0);
    // t2d2 = k2d2 + wn (E2d2 - k2d2), etc.
    T k2d2_b = (T(1) - wn) * t2d2_b;
    const T E2d2_b = wn * t2d2_b;
    wn_b += (E2d2 - k2d2) * t2d2_b;
    T k2d1_b = (T(1) - wn) * t2d1_b;
    const T E2d1_b = wn * t2d1_b;
    wn_b += (E2d1 - k2d1) * t2d1_b;
    T N2s_b = (T(1) - wb) * t2s_b;
    const T E2s_b = wb * t2s_b;
    wb_b += (E2s - N2s) * t2s_b;
    T rho_b = T(0), ux_b = ob.ux, uy_b = ob.uy, uz_b = ob.uz;
    if (CORR != LB_CORR_NONE) {
        // E2d2 = tn (qxx X - qzz Z); E2d1 = tn (qxx X - qyy Y); E2s = tb (qxx X + qyy Y + qzz Z)
        const T tn_b = (qxx * X - qzz * Z) * E2d2_b + (qxx * X - qyy * Y) * E2d1_b;
        const T tb_b = (qxx * X + qyy * Y + qzz * Z) * E2s_b;
        const T sX = P.tn * (E2d2_b + E2d1_b) + P.tb * E2s_b;   // coefficient of qxx X
        T qxx_b = sX * X, X_b = sX * qxx;
        T qyy_b = (P.tb * E2s_b - P.tn * E2d1_b) * Y;
        T Y_b = (P.tb * E2s_b - P.tn * E2d1_b) * qyy;
        T qzz_b = (P.tb * E2s_b - P.tn * E2d2_b) * Z;
        T Z_b = (P.tb * E2s_b - P.tn * E2d2_b) * qzz;
        // tn = 1/wn - 1/2, tb = 1/wb - 1/2
        wn_b += -div_(tn_b, wn * wn);
        wb_b += -div_(tb_b, wb * wb);
        // q.. = -rho (3 u.2 + an)
        T ux2_b = -T(3) * rho * qxx_b, uy2_b = -T(3) * rho * qyy_b, uz2_b = -T(3) * rho * qzz_b;
        rho_b += -(T(3) * ux2 + P.an[0]) * qxx_b - (T(3) * uy2 + P.an[1]) * qyy_b - (T(3) * uz2 + P.an[2]) * qzz_b;
        // Z = zn / Csz, Y = yn / Csy, zn = Rs2 - Csx X, yn = Rs1 - Csx X
        const T zn_b = div_(Z_b, Csz), yn_b = div_(Y_b, Csy);
        T Csz_b = -Z * zn_b, Csy_b = -Y * yn_b;
        T Rs2_b = zn_b, Rs1_b = yn_b;
        T Csx_b = -X * (zn_b + yn_b);
        X_b += -Csx * (zn_b + yn_b);
        // X = num / den
        const T num_b = div_(X_b, den), den_b = -X * num_b;
        T Cby_b = T(0), Cbz_b = T(0), Cbx_b = T(0), Rb_b = T(0);
        // den = -Csx Csz Cby - Csy (Csx Cbz - Csz Cbx)
        Csx_b += (-Csz * Cby - Csy * Cbz) * den_b;
        Csz_b += (-Csx * Cby + Csy * Cbx) * den_b;
        Cby_b += -Csx * Csz * den_b;
        Csy_b += -(Csx * Cbz - Csz * Cbx) * den_b;
        Cbz_b += -Csy * Csx * den_b;
        Cbx_b += Csy * Csz * den_b;
        // num = -Csz Cby Rs1 - Csy (Cbz Rs2 - Csz Rb)
        Csz_b += (-Cby * Rs1 + Csy * Rb) * num_b;
        Cby_b += -Csz * Rs1 * num_b;
        Rs1_b += -Csz * Cby * num_b;
        Csy_b += -(Cbz * Rs2 - Csz * Rb) * num_b;
        Cbz_b += -Csy * Rs2 * num_b;
        Rs2_b += -Csy * Cbz * num_b;
        Rb_b += Csy * Csz * num_b;
        // C.. = (h. - c2.) rho etc.
        T hx_b = rho * (Csx_b + Cbx_b);
        T hy_b = rho * (Cby_b - Csy_b);
        T hz_b = rho * (Cbz_b - Csz_b);
        const T c2n_b = rho * (-Csx_b + Csy_b + Csz_b);
        const T c2b_b = -rho * (Cbx_b + Cby_b + Cbz_b);
        rho_b += (hx - c2n) * Csx_b + (hx - c2b) * Cbx_b + (c2n - hy) * Csy_b + (hy - c2b) * Cby_b +
                 (c2n - hz) * Csz_b + (hz - c2b) * Cbz_b;
        // c2n = 2 cs2 / wn
        wn_b += -div_(c2n_b * c2n, wn);
        wb_b += -div_(c2b_b * c2b, wb);
        ux2_b += T(1.5) * hx_b;
        uy2_b += T(1.5) * hy_b;
        uz2_b += T(1.5) * hz_b;
        ux_b += T(2) * al * ux * ux2_b;
        uy_b += T(2) * al * uy * uy2_b;
        uz_b += T(2) * al * uz * uz2_b;
        N2s_b += Rb_b;
        k2d1_b += Rs1_b;
        k2d2_b += Rs2_b;
    }
    const T n200_b = N2s_b + k2d1_b + k2d2_b;
    const T n020_b = N2s_b - k2d1_b;
    const T n002_b = N2s_b - k2d2_b;
    // k011 = pyz - rho uy uz + (uy Fz + uz Fy)/2, etc.
    b.m.pyz = k011_b;
    rho_b -= uy * uz * k011_b;
    uy_b += (-rho * uz + T(0.5) * Fz) * k011_b;
    uz_b += (-rho * uy + T(0.5) * Fy) * k011_b;
    Fz_b += T(0.5) * uy * k011_b;
    Fy_b += T(0.5) * uz * k011_b;
    b.m.pxz = k101_b;
    rho_b -= ux * uz * k101_b;
    ux_b += (-rho * uz + T(0.5) * Fz) * k101_b;
    uz_b += (-rho * ux + T(0.5) * Fx) * k101_b;
    Fz_b += T(0.5) * ux * k101_b;
    Fx_b += T(0.5) * uz * k101_b;
    b.m.pxy = k110_b;
    rho_b -= ux * uy * k110_b;
    ux_b += (-rho * uy + T(0.5) * Fy) * k110_b;
    uy_b += (-rho * ux + T(0.5) * Fx) * k110_b;
    Fy_b += T(0.5) * ux * k110_b;
    Fx_b += T(0.5) * uy * k110_b;
    // n200 = pxx - cs2x dr - rho ux^2 + ux Fx, etc. (cs2 of each axis' rest weights)
    b.m.pxx = n200_b;
    b.m.pyy = n020_b;
    b.m.pzz = n002_b;
    T dr_b = ob.dr - (P.cs2ax[0] * n200_b + P.cs2ax[1] * n020_b + P.cs2ax[2] * n002_b);
    rho_b -= ux * ux * n200_b + uy * uy * n020_b + uz * uz * n002_b;
    ux_b += (-T(2) * rho * ux + Fx) * n200_b;
    uy_b += (-T(2) * rho * uy + Fy) * n020_b;
    uz_b += (-T(2) * rho * uz + Fz) * n002_b;
    Fx_b += ux * n200_b;
    Fy_b += uy * n020_b;
    Fz_b += uz * n002_b;
    // u = q irho, q = j + F/2, irho = 1 / rho
    const T qx_b = irho * ux_b, qy_b = irho * uy_b, qz_b = irho * uz_b;
    const T irho_b = qx * ux_b + qy * uy_b + qz * uz_b;
    b.m.jx = qx_b;
    b.m.jy = qy_b;
    b.m.jz = qz_b;
    Fx_b += T(0.5) * qx_b;
    Fy_b += T(0.5) * qy_b;
    Fz_b += T(0.5) * qz_b;
    rho_b -= irho * irho * irho_b;
    dr_b += rho_b;
    b.m.dr = dr_b;
    b.Fx = Fx_b;
    b.Fy = Fy_b;
    b.Fz = Fz_b;
    b.wn = wn_b;
    b.wb = wb_b;
    return b;
}

// Adjoints of the per-axis columns, folded into d/du of that axis.
template <class T>
__device__ __forceinline__ T axis_cols_vjp(T u, T ic, const T (&g0_b)[3], const T (&g1_b)[3], const T (&dphi_b)[3])
{
    const T a = u * ic;
    T a_b = T(0.5) * (g0_b[2] - g0_b[0]) + ic * (g1_b[0] - T(2) * g1_b[1] + g1_b[2]) +
            T(0.5) * (dphi_b[2] - dphi_b[0]);
    const T b_b = T(0.5) * (g0_b[0] + g0_b[2] + dphi_b[0] + dphi_b[2]) - g0_b[1] - dphi_b[1];
    a_b += T(2) * a * b_b;
    return ic * a_b;
}

// Reverse of back_transform: L = adjoint of h~ (in), returns the PostState adjoint.
template <class T>
__device__ __forceinline__ PostState<T> back_transform_vjp(const T (&L)[Q], const PostState<T> &o, const Phys<T> &P)
{
    const AxisCols<T> X = axis_cols(o.ux, P.ic[0], P.ic2[0], P.w0[0], P.wpm[0]);
    const AxisCols<T> Y = axis_cols(o.uy, P.ic[1], P.ic2[1], P.w0[1], P.wpm[1]);
    const AxisCols<T> Z = axis_cols(o.uz, P.ic[2], P.ic2[2], P.w0[2], P.wpm[2]);
    T A00[3], A10[3], A01[3], A11[3], A20[3], A02[3];
#pragma unroll
    for (int z = 0; z < 3; ++z) {
        A00[z] = o.hFz * Z.g1[z] + o.d002 * Z.g2[z];
        A10[z] = o.hFx * Z.g0[z] + o.t101 * Z.g1[z];
        A01[z] = o.hFy * Z.g0[z] + o.t011 * Z.g1[z];
        A11[z] = o.t110 * Z.g0[z];
        A20[z] = o.d200 * Z.g0[z];
        A02[z] = o.d020 * Z.g0[z];
    }
    T ax[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) ax[x] = o.dr * X.phi[x] + X.dphi[x];

    T ax_b[3] = {T(0), T(0), T(0)}, g0x_b[3] = {T(0), T(0), T(0)}, g1x_b[3] = {T(0), T(0), T(0)};
    T g0y_b[3] = {T(0), T(0), T(0)}, g1y_b[3] = {T(0), T(0), T(0)}, dphiy_b[3] = {T(0), T(0), T(0)};
    T g0z_b[3] = {T(0), T(0), T(0)}, g1z_b[3] = {T(0), T(0), T(0)}, dphiz_b[3] = {T(0), T(0), T(0)};
    T A00_b[3] = {T(0), T(0), T(0)}, A10_b[3] = {T(0), T(0), T(0)}, A01_b[3] = {T(0), T(0), T(0)};
    T A11_b[3] = {T(0), T(0), T(0)}, A20_b[3] = {T(0), T(0), T(0)}, A02_b[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int y = 0; y < 3; ++y)
#pragma unroll
        for (int z = 0; z < 3; ++z) {
            const T B0 = A00[z] * Y.g0[y] + A01[z] * Y.g1[y] + A02[z] * Y.g2[y];
            const T B1 = A10[z] * Y.g0[y] + A11[z] * Y.g1[y];
            const T B2 = A20[z] * Y.g0[y];
            const T Pyz = Y.phi[y] * Z.phi[z];
            T B0_b = T(0), B1_b = T(0), B2_b = T(0), Pyz_b = T(0), Dyz_b = T(0);
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                const T l = L[dir_of(x - 1, y - 1, z - 1)];
                B0_b += l * X.g0[x];
                B1_b += l * X.g1[x];
                B2_b += l * X.g2[x];
                Pyz_b += l * ax[x];
                Dyz_b += l * X.w[x];
                ax_b[x] += l * Pyz;
                g0x_b[x] += l * B0;
                g1x_b[x] += l * B1;
            }
            // Dyz = dphi_y phi_z + w_y dphi_z ; Pyz = phi_y phi_z (phi = w + dphi)
            dphiy_b[y] += Dyz_b * Z.phi[z] + Pyz_b * Z.phi[z];
            dphiz_b[z] += Dyz_b * (Y.dphi[y] + Y.w[y]) + Pyz_b * Y.phi[y];
            // B2 = A20 g0y ; B1 = A10 g0y + A11 g1y ; B0 = A00 g0y + A01 g1y + A02 g2y
            A20_b[z] += B2_b * Y.g0[y];
            A10_b[z] += B1_b * Y.g0[y];
            A11_b[z] += B1_b * Y.g1[y];
            A00_b[z] += B0_b * Y.g0[y];
            A01_b[z] += B0_b * Y.g1[y];
            A02_b[z] += B0_b * Y.g2[y];
            g0y_b[y] += B2_b * A20[z] + B1_b * A10[z] + B0_b * A00[z];
            g1y_b[y] += B1_b * A11[z] + B0_b * A01[z];
        }
    PostState<T> ob;
    // ax = dr phi_x + dphi_x
    T dr_b = T(0), dphix_b[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        dr_b += ax_b[x] * X.phi[x];
        dphix_b[x] = ax_b[x] * (o.dr + T(1));   // through phi_x = w + dphi_x and dphi_x itself
    }
    ob.dr = dr_b;
    T d020_b = T(0), d200_b = T(0), t110_b = T(0), hFy_b = T(0), t011_b = T(0), hFx_b = T(0), t101_b = T(0);
    T hFz_b = T(0), d002_b = T(0);
#pragma unroll
    for (int z = 0; z < 3; ++z) {
        d020_b += A02_b[z] * Z.g0[z];
        d200_b += A20_b[z] * Z.g0[z];
        t110_b += A11_b[z] * Z.g0[z];
        hFy_b += A01_b[z] * Z.g0[z];
        t011_b += A01_b[z] * Z.g1[z];
        hFx_b += A10_b[z] * Z.g0[z];
        t101_b += A10_b[z] * Z.g1[z];
        hFz_b += A00_b[z] * Z.g1[z];
        d002_b += A00_b[z] * Z.g2[z];
        g0z_b[z] += A02_b[z] * o.d020 + A20_b[z] * o.d200 + A11_b[z] * o.t110 + A01_b[z] * o.hFy + A10_b[z] * o.hFx;
        g1z_b[z] += A01_b[z] * o.t011 + A10_b[z] * o.t101 + A00_b[z] * o.hFz;
    }
    ob.d020 = d020_b;
    ob.d200 = d200_b;
    ob.d002 = d002_b;
    ob.t110 = t110_b;
    ob.t101 = t101_b;
    ob.t011 = t011_b;
    ob.hFx = hFx_b;
    ob.hFy = hFy_b;
    ob.hFz = hFz_b;
    ob.ux = axis_cols_vjp(o.ux, P.ic[0], g0x_b, g1x_b, dphix_b);
    ob.uy = axis_cols_vjp(o.uy, P.ic[1], g0y_b, g1y_b, dphiy_b);
    ob.uz = axis_cols_vjp(o.uz, P.ic[2], g0z_b, g1z_b, dphiz_b);
    return ob;
}

// Reverse of raw_moments: adjoint of h from adjoints of the ten moments.
template <class T>
__device__ __forceinline__ void raw_moments_vjp(const RawMoments<T> &mb, const Phys<T> &P, T (&hb)[Q])
{
    const T r = P.c[1], s = P.c[2];
    const T jy = r * mb.jy, jz = s * mb.jz, pyy = r * r * mb.pyy, pzz = s * s * mb.pzz;
    const T pxy = r * mb.pxy, pxz = s * mb.pxz, pyz = r * s * mb.pyz;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int x = ex(a), y = ey(a), z = ez(a);
        T v = mb.dr;
        if (x) v += T(x) * mb.jx + mb.pxx;
        if (y) v += T(y) * jy + pyy;
        if (z) v += T(z) * jz + pzz;
        if (x * y) v += T(x * y) * pxy;
        if (x * z) v += T(x * z) * pxz;
        if (y * z) v += T(y * z) * pyz;
        hb[a] = v;
    }
}

// Per-node VJP of the whole collision: given h (pre-collision deviations) and
// L = dJ/d h~, returns dJ/dh in L (in place) and the force / rate adjoints.
template <class T, int CORR>
__device__ __forceinline__ RelaxBar<T> collide_vjp(const T (&h)[Q], T (&L)[Q], const Phys<T> &P, T Fx, T Fy, T Fz)
{
    const RawMoments<T> m = raw_moments(h, P);
    const PostState<T> o = relax_node<T, CORR>(m, P, Fx, Fy, Fz, T(0), T(0), T(0));
    const PostState<T> ob = back_transform_vjp(L, o, P);
    const RelaxBar<T> rb = relax_node_vjp<T, CORR>(m, P, Fx, Fy, Fz, ob);
    raw_moments_vjp(rb.m, P, L);
    return rb;
}

}  // namespace lbc

namespace lbc {

constexpr int kAdjThreads = 128;

// Block sum of two doubles into out[blockIndex * 2 + c] (added, so that one
// array accumulates over many launches of the same grid in a fixed order).
__device__ __forceinline__ void block_sum2_accumulate(double a, double b, double *out)
{
    __shared__ double sh[2][kAdjThreads];
    const int t = threadIdx.x + threadIdx.y * blockDim.x;
    sh[0][t] = a;
    sh[1][t] = b;
    __syncthreads();
    for (int s = kAdjThreads / 2; s > 0; s >>= 1) {
        if (t < s) {
            sh[0][t] += sh[0][t + s];
            sh[1][t] += sh[1][t + s];
        }
        __syncthreads();
    }
    if (t == 0) {
        const long long bid = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
        out[2 * bid] += sh[0][0];
        out[2 * bid + 1] += sh[1][0];
    }
}

// Seed of the adjoint for the mean kinetic energy J = (1/N) sum_x |j|^2 / (2 rho),
// j = sum f e + F/2 (Eq. 12), at the final state: lambda_a = (u . e_a - |u|^2/2)/N,
// dJ/dF = u / (2N) (direct dependence through the F/2 shift), and per-block J.
template <int ST>
__global__ void __launch_bounds__(kAdjThreads)
k_adjoint_seed(const typename Codec<ST>::S *__restrict__ src, Geom g, Phys<typename Codec<ST>::T> P,
               DirConst<typename Codec<ST>::T> D, typename Codec<ST>::T F0, typename Codec<ST>::T F1,
               typename Codec<ST>::T F2, const typename Codec<ST>::T *__restrict__ ff,
               typename Codec<ST>::T *__restrict__ lam, typename Codec<ST>::T *__restrict__ dJdF,
               double *__restrict__ jpart)
{
    using T = typename Codec<ST>::T;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    double Jx = 0.0;
    if (i < g.nx && j < g.ny) {
        const long long N = g.N;
        const Pull q = make_pull(g, i, j, k);
        T h[Q];
        pull_node<ST>(h, src, q, N, D, P, T(0));
        const RawMoments<T> m = raw_moments(h, P);
        T Fx = F0, Fy = F1, Fz = F2;
        if (ff) {
            Fx += ff[q.base];
            Fy += ff[N + q.base];
            Fz += ff[2 * N + q.base];
        }
        const T rho = T(1) + m.dr;
        const T jx = m.jx + T(0.5) * Fx, jy = m.jy + T(0.5) * Fy, jz = m.jz + T(0.5) * Fz;
        const T ux = jx / rho, uy = jy / rho, uz = jz / rho;
        const T iN = T(1) / T(N);
        const T u2 = ux * ux + uy * uy + uz * uz;
        Jx = 0.5 * (double)rho * (double)u2 / (double)N;
        const T vx = ux, vy = P.c[1] * uy, vz = P.c[2] * uz;   // u . e_a = ex ux + r ey uy + s ez uz
        if (lam) {
#pragma unroll
            for (int a = 0; a < Q; ++a)
                lam[(long long)a * N + q.base] = (T(ex(a)) * vx + T(ey(a)) * vy + T(ez(a)) * vz - T(0.5) * u2) * iN;
        }
        if (dJdF) {
            dJdF[q.base] = T(0.5) * ux * iN;
            dJdF[N + q.base] = T(0.5) * uy * iN;
            dJdF[2 * N + q.base] = T(0.5) * uz * iN;
        }
    }
    block_sum2_accumulate(Jx, 0.0, jpart);
}

// One step of the discrete adjoint (see the top of this file).  src = stored state
// S^n (pull layout, so that pulling gives f^n); lam_in = lambda^{n+1} and lam_out =
// lambda^n in natural layout [27][N].
// Resident CTAs per SM requested from the compiler.  Left free, the adjoint step with LOCAL
// corrections takes 188 registers (two CTAs of 128 threads per SM).  At four CTAs (128
// registers, 44 B spilled) the whole lb_adjoint_ke call on 128x64x64 with a per-node force
// field, T = 500, K = 50, took 56.8 ms on GB300 against 72.0 ms left free (three CTAs
// 60.2 ms, five CTAs 62.8 ms with 624 B spilled).
#ifndef LBC_ADJ_MINBLOCKS
#define LBC_ADJ_MINBLOCKS 4
#endif
template <int ST, int CORR>
__global__ void __launch_bounds__(kAdjThreads, LBC_ADJ_MINBLOCKS)
k_adjoint(const typename Codec<ST>::S *__restrict__ src, const typename Codec<ST>::T *__restrict__ lam_in,
          typename Codec<ST>::T *__restrict__ lam_out, Geom g, Phys<typename Codec<ST>::T> P,
          DirConst<typename Codec<ST>::T> D, typename Codec<ST>::T F0, typename Codec<ST>::T F1,
          typename Codec<ST>::T F2, const typename Codec<ST>::T *__restrict__ ff,
          typename Codec<ST>::T *__restrict__ dJdF, double *__restrict__ wpart)
{
    using T = typename Codec<ST>::T;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    double wn_b = 0.0, wb_b = 0.0;
    if (i < g.nx && j < g.ny) {
        const long long N = g.N;
        const Pull q = make_pull(g, i, j, k);
        T h[Q];
        pull_node<ST>(h, src, q, N, D, P, T(0));
        // transposed streaming: lambda_g_a(x) = lambda_a(x + e_a), or lambda_opp(a)(x) across a wall
        T L[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const int cx = 1 - ex(a), cy = 1 - ey(a), cz = 1 - ez(a);   // index of the source x + e_a
            const bool out = q.xo[cx] | q.yo[cy] | q.zo[cz];
            const long long off = out ? (long long)opp(a) * N + q.base
                                      : (long long)a * N + q.zoff[cz] + q.yoff[cy] + q.xs[cx];
            L[a] = __ldg(lam_in + off);
        }
        T Fx = F0, Fy = F1, Fz = F2;
        if (ff) {
            Fx += __ldg(ff + q.base);
            Fy += __ldg(ff + N + q.base);
            Fz += __ldg(ff + 2 * N + q.base);
        }
        const RelaxBar<T> rb = collide_vjp<T, CORR>(h, L, P, Fx, Fy, Fz);
#pragma unroll
        for (int a = 0; a < Q; ++a) lam_out[(long long)a * N + q.base] = L[a];
        dJdF[q.base] += rb.Fx;
        dJdF[N + q.base] += rb.Fy;
        dJdF[2 * N + q.base] += rb.Fz;
        wn_b = (double)rb.wn;
        wb_b = (double)rb.wb;
    }
    block_sum2_accumulate(wn_b, wb_b, wpart);
}

// The adjoint step marching along z (4-byte storage): each thread keeps its (x, y) node
// and steps through kAdjPlanes planes.  The 27 pulled state words and the 27 transposed
// lambda words of a plane are copied into the thread's own column of a two-slot shared
// memory stage by 4-byte cp.async, those of the next plane being issued before the
// current plane is waited for, so that the loads travel while the per-node VJP (about
// 2,400 instructions) runs; the force field and the dJ/dF to be updated are loaded into
// registers ahead of their use.  The same arithmetic as k_adjoint, node by node; only
// the FP64 partial sums of dJ/domega are summed in another order.
// Measured on GB300 (lb_adjoint_ke, 128x64x64 with a force field, T = 500, FP32): three
// CTAs per SM (170 registers, no spill) take the K = 1 call to 41.4 ms against 44.1 ms for
// k_adjoint; at four CTAs (128 registers, ~90 B spilled) it took 46.7-48.3 ms.  Two or four
// planes per thread measure alike; eight leave too few CTAs on this lattice.
#ifndef LBC_ADJ_PLANES
#define LBC_ADJ_PLANES 4
#endif
#ifndef LBC_ADJ_MARCH_MINBLOCKS
#define LBC_ADJ_MARCH_MINBLOCKS 3
#endif
constexpr int kAdjPlanes = LBC_ADJ_PLANES;
constexpr size_t kAdjStageBytes = (size_t)2 * 2 * Q * kAdjThreads * 4;

template <int ST, int CORR>
__global__ void __launch_bounds__(kAdjThreads, LBC_ADJ_MARCH_MINBLOCKS)
k_adjoint_march(const typename Codec<ST>::S *__restrict__ src, const typename Codec<ST>::T *__restrict__ lam_in,
                typename Codec<ST>::T *__restrict__ lam_out, Geom g, Phys<typename Codec<ST>::T> P,
                DirConst<typename Codec<ST>::T> D, typename Codec<ST>::T F0, typename Codec<ST>::T F1,
                typename Codec<ST>::T F2, const typename Codec<ST>::T *__restrict__ ff,
                typename Codec<ST>::T *__restrict__ dJdF, double *__restrict__ wpart)
{
    using C = Codec<ST>;
    using T = typename C::T;
    static_assert(sizeof(typename C::S) == 4 && sizeof(T) == 4, "the staged adjoint copies 4-byte words");
    extern __shared__ __align__(16) unsigned adj_stage[];   // [slot][word][thread], words 0..26 state, 27..53 lambda
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = (int)blockIdx.z * kAdjPlanes;
    const int kend = min(k0 + kAdjPlanes, g.nz);
    const long long N = g.N;
    double wn_b = 0.0, wb_b = 0.0;
    auto slot = [&](int s, int w) -> unsigned * { return adj_stage + ((size_t)s * 2 * Q + w) * kAdjThreads + tid; };
    auto issue = [&](int k, int s) {
        const Pull q = make_pull(g, i, j, k);
        const unsigned *sw = reinterpret_cast<const unsigned *>(src);
        const unsigned *lw = reinterpret_cast<const unsigned *>(lam_in);
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const int cx = ex(a) + 1, cy = ey(a) + 1, cz = ez(a) + 1;
            const bool out = q.xo[cx] | q.yo[cy] | q.zo[cz];
            const long long soff = out ? (long long)opp(a) * N + q.base
                                       : (long long)a * N + q.zoff[cz] + q.yoff[cy] + q.xs[cx];
            cp_async4(slot(s, a), sw + soff);
            const int mx = 1 - ex(a), my = 1 - ey(a), mz = 1 - ez(a);   // the source x + e_a
            const bool mout = q.xo[mx] | q.yo[my] | q.zo[mz];
            const long long loff = mout ? (long long)opp(a) * N + q.base
                                        : (long long)a * N + q.zoff[mz] + q.yoff[my] + q.xs[mx];
            cp_async4(slot(s, Q + a), lw + loff);
        }
        cp_async_commit();
    };
    if (i < g.nx && j < g.ny) {
        issue(k0, 0);
        for (int k = k0; k < kend; ++k) {
            const int s = (k - k0) & 1;
            const long long base = (long long)k * g.nx * g.ny + (long long)j * g.nx + i;
            T Fx = F0, Fy = F1, Fz = F2;
            if (ff) {
                Fx += __ldg(ff + base);
                Fy += __ldg(ff + N + base);
                Fz += __ldg(ff + 2 * N + base);
            }
            const T d0 = dJdF[base], d1 = dJdF[N + base], d2 = dJdF[2 * N + base];
            if (k + 1 < kend) {
                issue(k + 1, s ^ 1);
                asm volatile("cp.async.wait_group 1;\n" ::: "memory");
            } else {
                cp_async_wait_all();
            }
            T h[Q], L[Q];
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                h[a] = C::load(__uint_as_float(*slot(s, a)), D.w[a], D.iscale[a]);
                L[a] = __uint_as_float(*slot(s, Q + a));
            }
            const RelaxBar<T> rb = collide_vjp<T, CORR>(h, L, P, Fx, Fy, Fz);
#pragma unroll
            for (int a = 0; a < Q; ++a) lam_out[(long long)a * N + base] = L[a];
            dJdF[base] = d0 + rb.Fx;
            dJdF[N + base] = d1 + rb.Fy;
            dJdF[2 * N + base] = d2 + rb.Fz;
            wn_b += (double)rb.wn;
            wb_b += (double)rb.wb;
        }
    }
    // block sum in fixed order, in the stage memory (no copies are in flight any more)
    __syncthreads();
    double *sh = reinterpret_cast<double *>(adj_stage);
    sh[tid] = wn_b;
    sh[kAdjThreads + tid] = wb_b;
    __syncthreads();
    for (int s = kAdjThreads / 2; s > 0; s >>= 1) {
        if (tid < s) {
            sh[tid] += sh[tid + s];
            sh[kAdjThreads + tid] += sh[kAdjThreads + tid + s];
        }
        __syncthreads();
    }
    if (tid == 0) {
        const long long bid = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
        wpart[2 * bid] += sh[0];
        wpart[2 * bid + 1] += sh[kAdjThreads];
    }
}

// Per-node VJP of the collision alone for n independent nodes (test entry point):
// f [27][n] populations, F [3][n], L [27][n] = dJ/df~  ->  fb [27][n] = dJ/df,
// Fb [3][n], wpart per block (dJ/domega_nu, dJ/domega_xi).
template <int ST, int CORR>
__global__ void __launch_bounds__(kAdjThreads)
k_collide_vjp(const typename Codec<ST>::T *__restrict__ f, const typename Codec<ST>::T *__restrict__ F,
              const typename Codec<ST>::T *__restrict__ Lin, typename Codec<ST>::T *__restrict__ fb,
              typename Codec<ST>::T *__restrict__ Fb, long long n, Phys<typename Codec<ST>::T> P,
              DirConst<typename Codec<ST>::T> D, double *__restrict__ wpart)
{
    using T = typename Codec<ST>::T;
    const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double wn_b = 0.0, wb_b = 0.0;
    if (x < n) {
        T h[Q], L[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            h[a] = f[a * n + x] - D.w[a];
            L[a] = Lin[a * n + x];
        }
        const RelaxBar<T> rb = collide_vjp<T, CORR>(h, L, P, F[x], F[n + x], F[2 * n + x]);
#pragma unroll
        for (int a = 0; a < Q; ++a) fb[a * n + x] = L[a];
        Fb[x] = rb.Fx;
        Fb[n + x] = rb.Fy;
        Fb[2 * n + x] = rb.Fz;
        wn_b = (double)rb.wn;
        wb_b = (double)rb.wb;
    }
    block_sum2_accumulate(wn_b, wb_b, wpart);
}

}  // namespace lbc
