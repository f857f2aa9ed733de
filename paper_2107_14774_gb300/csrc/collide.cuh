// collide.cuh -- per-node collision of the cuboid D3Q27 central-moment scheme
// (Sec. 3.2; Apps. A-G), written for registers and for the deviation form.
//
// The node state enters and leaves as deviations h_a = f_a - w_a from the rest
// weights (rho0 = 1).  The transforms P, S, F(u) and their inverses are applied
// in their separable one-dimensional form: the monomial basis {1, e, e^2} per
// axis and the three velocities {-c, 0, c} per axis make P, S and F(u) tensor
// products of 3x3 factors, so the 27x27 products of Apps. A-C and E-G reduce to
// 3-point transforms along one axis at a time.  Because every relaxation rate
// other than omega_nu and omega_xi is 1 (App. D), the post-collision central
// moments equal their Maxwellian equilibria (Eq. 9) except
//   k~_100 = F_x / 2 (and y, z),  k~_110 = (1 - omega_nu) k_110 (and 101, 011),
//   the three diagonal second-order moments (relaxed via B, B^-1 with the
//   corrected equilibria of Eq. 63 / App. D);
// so only the ten raw moments of order <= 2 are needed on the way in, and on the
// way out f~ = f^eq(rho, u) + M(u)^-1 (k~ - k^eq), where the second term has only
// nine non-zero central-moment inputs.
//
// The code is generic in the lane type V: float or double for one node per
// thread, or F2 (two nodes per thread in the packed FP32x2 instructions of
// sm_100+) for the linear transforms around the per-node scalar collision.
#pragma once

#include "lattice.cuh"

namespace lbc {

// Two FP32 lanes evaluated with the packed FFMA2/FADD2/FMUL2 instructions.
struct F2 {
    float2 v;
    __device__ __forceinline__ F2() {}
    __device__ __forceinline__ F2(float c) : v(make_float2(c, c)) {}
    __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ explicit F2(float2 x) : v(x) {}
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(__fmul2_rn(a.v, make_float2(-1.f, -1.f))); }
__device__ __forceinline__ F2 &operator+=(F2 &a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2 &operator-=(F2 &a, F2 b) { return a = a - b; }

__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ F2 fma_(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }

// The kernels' CORR template word carries the lb_corr mode in its low bits and,
// in kRawModel, the choice of the raw-moment scheme (3DCRM) instead of the
// central-moment one.
constexpr int kRawModel = 16;
__host__ __device__ constexpr int corr_mode(int c) { return c & 15; }
__host__ __device__ constexpr bool raw_model(int c) { return (c & kRawModel) != 0; }

template <class V> struct Scalar { using type = V; };
template <> struct Scalar<F2> { using type = float; };

// Per-axis columns of the inverse central-moment transform M(u)^-1 for one axis
// with speed c and velocity u (velocity index v = -1, 0, +1 -> [0], [1], [2]):
// the 1-D populations whose central moments about u are (1,0,0), (0,1,0),
// (0,0,1).  Raw moments (1, u, u^2), (0, 1, 2u), (0, 0, 1) mapped to the three
// velocities by g(0) = M0 - M2/c^2, g(+-c) = (M2/c^2 +- M1/c)/2.
template <class V>
struct AxisCols {
    V g0[3], g1[3], g2[3];  // columns for central moments of order 0, 1, 2
    V phi[3], dphi[3];      // equilibrium factor phi = g0 + cs2 g2 and phi - w
    V w[3];                 // 1-D rest weights
};

template <class V, class T>
__device__ __forceinline__ AxisCols<V> axis_cols(V u, T ic, T ic2, T w0, T wpm)
{
    AxisCols<V> A;
    const V a = u * V(ic);       // u / c
    const V b = a * a;           // u^2 / c^2
    const V hb = V(T(0.5)) * b, ha = V(T(0.5)) * a;
    A.g0[0] = hb - ha;
    A.g0[1] = V(T(1)) - b;
    A.g0[2] = hb + ha;
    const V hic = V(T(0.5) * ic);
    const V aic = a * V(ic);     // u / c^2
    A.g1[0] = aic - hic;
    A.g1[1] = V(T(-2)) * aic;
    A.g1[2] = aic + hic;
    A.g2[0] = V(T(0.5) * ic2);
    A.g2[1] = V(-ic2);
    A.g2[2] = V(T(0.5) * ic2);
    A.dphi[0] = A.g0[0];
    A.dphi[1] = -b;
    A.dphi[2] = A.g0[2];
    A.w[0] = V(wpm);
    A.w[1] = V(w0);
    A.w[2] = V(wpm);
    A.phi[0] = V(wpm) + A.dphi[0];
    A.phi[1] = V(w0) + A.dphi[1];
    A.phi[2] = V(wpm) + A.dphi[2];
    return A;
}

// Hydrodynamic output of a collision.
template <class T>
struct NodeMacro {
    T rho, ux, uy, uz;
};

// Pre-collision moments of order <= 2 of one node, from the deviations h.
// Cubic raw moments are summed along x-lines, then y, then z (App. A in
// separable form); the cuboid scaling S (Eq. 59, App. B) follows.
template <class V>
struct RawMoments {
    V dr;                      // sum h   (rho - 1)
    V jx, jy, jz;              // sum h e (cuboid e)
    V pxx, pyy, pzz, pxy, pxz, pyz;  // sum h e_i e_j
};

template <class V, class T>
__device__ __forceinline__ RawMoments<V> raw_moments(const V (&h)[Q], const Phys<T> &P)
{
    // x-lines: for each (ey, ez) the sums over ex of h, h ex, h ex^2
    V X0[3][3], X1[3][3], X2[3][3];
#pragma unroll
    for (int jy = 0; jy < 3; ++jy)
#pragma unroll
        for (int jz = 0; jz < 3; ++jz) {
            const V hm = h[dir_of(-1, jy - 1, jz - 1)];
            const V h0 = h[dir_of(0, jy - 1, jz - 1)];
            const V hp = h[dir_of(1, jy - 1, jz - 1)];
            const V t = hp + hm;
            X0[jy][jz] = t + h0;
            X1[jy][jz] = hp - hm;
            X2[jy][jz] = t;
        }
    // y stage (only the combinations of total order <= 2 are kept)
    V Y00[3], Y01[3], Y02[3], Y10[3], Y11[3], Y20[3];
#pragma unroll
    for (int jz = 0; jz < 3; ++jz) {
        const V s = X0[2][jz] + X0[0][jz];
        Y00[jz] = s + X0[1][jz];
        Y01[jz] = X0[2][jz] - X0[0][jz];
        Y02[jz] = s;
        Y10[jz] = X1[0][jz] + X1[1][jz] + X1[2][jz];
        Y11[jz] = X1[2][jz] - X1[0][jz];
        Y20[jz] = X2[0][jz] + X2[1][jz] + X2[2][jz];
    }
    RawMoments<V> m;
    const V s00 = Y00[2] + Y00[0];
    m.dr = s00 + Y00[1];
    const V m001 = Y00[2] - Y00[0];
    const V m002 = s00;
    const V m010 = Y01[0] + Y01[1] + Y01[2];
    const V m011 = Y01[2] - Y01[0];
    const V m020 = Y02[0] + Y02[1] + Y02[2];
    const V m100 = Y10[0] + Y10[1] + Y10[2];
    const V m101 = Y10[2] - Y10[0];
    const V m110 = Y11[0] + Y11[1] + Y11[2];
    const V m200 = Y20[0] + Y20[1] + Y20[2];
    // S: scale by r^n s^p (Eq. 59)
    const T r = P.c[1], s = P.c[2];
    m.jx = m100;
    m.jy = V(r) * m010;
    m.jz = V(s) * m001;
    m.pxx = m200;
    m.pyy = V(r * r) * m020;
    m.pzz = V(s * s) * m002;
    m.pxy = V(r) * m110;
    m.pxz = V(s) * m101;
    m.pyz = V(r * s) * m011;
    return m;
}

// Post-collision central moments of one node that differ from the Maxwellian
// equilibrium (deviations), plus the hydrodynamic state.
template <class V>
struct PostState {
    V dr, ux, uy, uz;           // rho - 1, velocity (with F/2, Eq. 12)
    V hFx, hFy, hFz;            // k~_100 = F/2 (omega_1 = 1)
    V t110, t101, t011;         // (1 - omega_nu) k_1..
    V d200, d020, d002;         // k~_200 - cs2 rho, ...
};

// Division used by the per-node collision: IEEE for double; for float the fast
// approximate division (within 2 ulp for the divisors met here: the density and the
// O(cs2) coefficients of the strain-rate system, far from the range limits).  It
// took the FP32 two-node kernel from 30.8 to 31.7 GLUPS and FP16 storage from 37.3
// to 38.6 GLUPS on GB300, with every FP32 parity bound unchanged; LBC_IEEE_DIV
// restores a correctly rounded reciprocal times the numerator.
__device__ __forceinline__ double div_(double a, double b) { return a / b; }
#ifdef LBC_IEEE_DIV
__device__ __forceinline__ float div_(float a, float b) { return a * __frcp_rn(b); }
#else
__device__ __forceinline__ float div_(float a, float b) { return __fdividef(a, b); }
#endif
__device__ __forceinline__ F2 div_(F2 a, F2 b) { return F2(div_(a.v.x, b.v.x), div_(a.v.y, b.v.y)); }

// Relaxation of one node (App. D) from its raw moments (V = float/double for one
// node, F2 for two nodes in packed lanes).  F: body force at the node; gr:
// density gradient (used by LB_CORR_FULL only).
template <class V, int CORR>
__device__ __forceinline__ PostState<V> relax_node(const RawMoments<V> &m, const Phys<typename Scalar<V>::type> &P,
                                                   V Fx, V Fy, V Fz, V grx, V gry, V grz)
{
    using T = typename Scalar<V>::type;
    constexpr int CM = corr_mode(CORR);
    const V half = V(T(0.5));
    const V dr = m.dr;
    const V rho = V(T(1)) + dr;
    // rho u = sum f e + F/2 (Eq. 12), with u = q - q dr / rho (q = sum f e + F/2): the
    // rounding of 1 + dr (2^-24 relative in FP32, of one sign while the density
    // changes slowly) then only touches the small correction term
    const V ndr = dr * div_(V(T(-1)), rho);
    const V qx = fma_(half, Fx, m.jx), qy = fma_(half, Fy, m.jy), qz = fma_(half, Fz, m.jz);
    const V ux = fma_(qx, ndr, qx);
    const V uy = fma_(qy, ndr, qy);
    const V uz = fma_(qz, ndr, qz);

    // second-order central moments (App. C), diagonal ones as deviations from cs2 rho:
    // k_200 - cs2 rho = sum h ex^2 - cs2 (rho - 1) - rho ux^2 + ux Fx, etc., with the
    // second moment of the rest weights of each axis as cs2
    const V rux = rho * ux, ruy = rho * uy, ruz = rho * uz;
    const V n200 = fma_(ux, Fx - rux, m.pxx - V(P.cs2ax[0]) * dr);
    const V n020 = fma_(uy, Fy - ruy, m.pyy - V(P.cs2ax[1]) * dr);
    const V n002 = fma_(uz, Fz - ruz, m.pzz - V(P.cs2ax[2]) * dr);
    const V k110 = m.pxy - rux * uy + half * (ux * Fy + uy * Fx);
    const V k101 = m.pxz - rux * uz + half * (ux * Fz + uz * Fx);
    const V k011 = m.pyz - ruy * uz + half * (uy * Fz + uz * Fy);

    // B: combined diagonal moments (App. D); N2s = k_2s - 3 cs2 rho
    const V N2s = n200 + n020 + n002;
    const V k2d1 = n200 - n020;
    const V k2d2 = n200 - n002;

    // corrected equilibria of the combined moments (App. D, Eq. 63), as deviations
    V E2s = V(T(0)), E2d1 = V(T(0)), E2d2 = V(T(0));
    if (CM != LB_CORR_NONE) {
        const V al = V((CM == LB_CORR_LOWMACH) ? T(0) : T(1));
        const V ux2 = al * ux * ux, uy2 = al * uy * uy, uz2 = al * uz * uz;
        const V an0 = V(P.an[0]), an1 = V(P.an[1]), an2 = V(P.an[2]);
        // density-gradient terms (FULL only): A, B, C and e-terms
        V ebr = V(T(0)), esr1 = V(T(0)), esr2 = V(T(0));
        if (CM == LB_CORR_FULL) {
            const V A = half * an0 * ux, B = half * an1 * uy, C = half * an2 * uz;
            esr1 = -A * grx + B * gry;
            esr2 = -A * grx + C * grz;
            ebr = -A * grx - B * gry - C * grz;
        }
        const V Rb = N2s + ebr, Rs1 = k2d1 + esr1, Rs2 = k2d2 + esr2;
        const V onep5 = V(T(1.5));
        const V hx = fma_(onep5, ux2, half * an0);
        const V hy = fma_(onep5, uy2, half * an1);
        const V hz = fma_(onep5, uz2, half * an2);
        const V c2n = V(P.two_cs2_wn), c2b = V(P.two_cs2_wb);
        const V Csx = (hx - c2n) * rho;
        const V Cbx = (hx - c2b) * rho;
        const V Csy = (c2n - hy) * rho;
        const V Cby = (hy - c2b) * rho;
        const V Csz = (c2n - hz) * rho;
        const V Cbz = (hz - c2b) * rho;
        // Eq. 49 / App. D: Cramer's rule on the 3x3 system
        const V num = -Csz * Cby * Rs1 - Csy * (Cbz * Rs2 - Csz * Rb);
        const V den = -Csx * Csz * Cby - Csy * (Csx * Cbz - Csz * Cbx);
        const V dxux = div_(num, den);
        const V dyuy = div_(Rs1 - Csx * dxux, Csy);
        const V dzuz = div_(Rs2 - Csx * dxux, Csz);
        // theta coefficients (Eq. 38-40 in the shear/bulk notation of App. D)
        const V three = V(T(3));
        const V qx = -rho * fma_(three, ux2, an0);
        const V qy = -rho * fma_(three, uy2, an1);
        const V qz = -rho * fma_(three, uz2, an2);
        const V tb = V(P.tb), tn = V(P.tn);
        E2s = tb * (qx * dxux + qy * dyuy + qz * dzuz);
        E2d1 = tn * (qx * dxux - qy * dyuy);
        E2d2 = tn * (qx * dxux - qz * dzuz);
        if (CM == LB_CORR_FULL) {
            // lambda coefficients: s-terms -, +, + ; b-terms -, -, -
            const V lx = an0 * ux, ly = an1 * uy, lz = an2 * uz;
            E2s -= tb * (lx * grx + ly * gry + lz * grz);
            E2d1 += tn * (-lx * grx + ly * gry);
            E2d2 += tn * (-lx * grx + lz * grz);
        }
    }
    // relaxation (App. D)
    const V wn = V(P.wn), wb = V(P.wb);
    const V t2s = fma_(wb, E2s - N2s, N2s);
    const V t2d1 = fma_(wn, E2d1 - k2d1, k2d1);
    const V t2d2 = fma_(wn, E2d2 - k2d2, k2d2);
    const V onemw = V(T(1) - P.wn);
    PostState<V> o;
    o.dr = dr;
    o.ux = ux;
    o.uy = uy;
    o.uz = uz;
    o.t110 = onemw * k110;
    o.t101 = onemw * k101;
    o.t011 = onemw * k011;
    // B^-1 (end of App. D), deviations of k~_200, k~_020, k~_002 from cs2 rho
    const V third = V(T(1) / T(3));
    const V two = V(T(2));
    o.d200 = (t2s + t2d1 + t2d2) * third;
    o.d020 = (t2s - two * t2d1 + t2d2) * third;
    o.d002 = (t2s + t2d1 - two * t2d2) * third;
    o.hFx = half * Fx;
    o.hFy = half * Fy;
    o.hFz = half * Fz;
    if constexpr (raw_model(CORR)) {
        // Raw-moment scheme (Sec. 3.1 raw formulation; Sec. 7): relaxing the raw second-
        // order moments with the raw sources of Eq. 11 leaves them above the central
        // scheme's post-collision values by half the raw source moments; the
        // deviations below are taken from the raw equilibria of Eq. 10, and every
        // raw moment above second order is its equilibrium.
        o.d200 = fma_(ux, Fx, o.d200);
        o.d020 = fma_(uy, Fy, o.d020);
        o.d002 = fma_(uz, Fz, o.d002);
        o.t110 = fma_(half, fma_(Fx, uy, Fy * ux), o.t110);
        o.t101 = fma_(half, fma_(Fx, uz, Fz * ux), o.t101);
        o.t011 = fma_(half, fma_(Fy, uz, Fz * uy), o.t011);
    }
    return o;
}

// Back to populations: h~ = f^eq(rho, u) - w + M(u)^-1 (k~ - k^eq) (Apps. E-G).
// Each post-collision deviation is handed to out(a, value) as soon as it is
// formed (a store, or a write into a register array).  RAW: the deviations are
// raw moments, mapped by P^-1 S^-1 alone (the columns of M(0)^-1).
template <bool RAW = false, class V, class T, class Out>
__device__ __forceinline__ void back_transform_to(Out &&out, const PostState<V> &o, const Phys<T> &P)
{
    const AxisCols<V> X = axis_cols(o.ux, P.ic[0], P.ic2[0], P.w0[0], P.wpm[0]);
    const AxisCols<V> Y = axis_cols(o.uy, P.ic[1], P.ic2[1], P.w0[1], P.wpm[1]);
    const AxisCols<V> Z = axis_cols(o.uz, P.ic[2], P.ic2[2], P.w0[2], P.wpm[2]);
    const V zero = V(T(0));
    const AxisCols<V> GX = RAW ? axis_cols(zero, P.ic[0], P.ic2[0], P.w0[0], P.wpm[0]) : X;
    const AxisCols<V> GY = RAW ? axis_cols(zero, P.ic[1], P.ic2[1], P.w0[1], P.wpm[1]) : Y;
    const AxisCols<V> GZ = RAW ? axis_cols(zero, P.ic[2], P.ic2[2], P.w0[2], P.wpm[2]) : Z;

    // rho phi_x phi_y phi_z - w_x w_y w_z = (dr phi_x + dphi_x) P_yz + w_x D_yz with
    // P_yz = phi_y phi_z and D_yz = phi_y phi_z - w_y w_z = dphi_y phi_z + w_y dphi_z
    V ax[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) ax[x] = fma_(o.dr, X.phi[x], X.dphi[x]);
    // z outermost keeps only one z-slice of the intermediate arrays alive
#pragma unroll
    for (int z = 0; z < 3; ++z) {
        // z stage of M^-1 on the sparse non-equilibrium central moments
        const V A00 = fma_(o.hFz, GZ.g1[z], o.d002 * GZ.g2[z]);
        const V A10 = fma_(o.hFx, GZ.g0[z], o.t101 * GZ.g1[z]);
        const V A01 = fma_(o.hFy, GZ.g0[z], o.t011 * GZ.g1[z]);
        const V A11 = o.t110 * GZ.g0[z];
        const V A20 = o.d200 * GZ.g0[z];
        const V A02 = o.d020 * GZ.g0[z];
#pragma unroll
        for (int y = 0; y < 3; ++y) {
            const V B0 = fma_(A00, GY.g0[y], fma_(A01, GY.g1[y], A02 * GY.g2[y]));
            const V B1 = fma_(A10, GY.g0[y], A11 * GY.g1[y]);
            const V B2 = A20 * GY.g0[y];
            const V Pyz = Y.phi[y] * Z.phi[z];
            const V Dyz = fma_(Y.dphi[y], Z.phi[z], Y.w[y] * Z.dphi[z]);
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                const V heq = fma_(ax[x], Pyz, X.w[x] * Dyz);
                out(dir_of(x - 1, y - 1, z - 1), fma_(B0, GX.g0[x], fma_(B1, GX.g1[x], fma_(B2, GX.g2[x], heq))));
            }
        }
    }
}

template <bool RAW = false, class V, class T>
__device__ __forceinline__ void back_transform(V (&h)[Q], const PostState<V> &o, const Phys<T> &P)
{
    back_transform_to<RAW>([&](int a, V v) { h[a] = v; }, o, P);
}

// One collision, in place on the deviations h of one node (Sec. 3.2 steps, App. D).
template <class T, int CORR>
__device__ __forceinline__ NodeMacro<T> collide(T (&h)[Q], const Phys<T> &P, T Fx, T Fy, T Fz,
                                                T grx = T(0), T gry = T(0), T grz = T(0))
{
    const RawMoments<T> m = raw_moments(h, P);
    const PostState<T> o = relax_node<T, CORR>(m, P, Fx, Fy, Fz, grx, gry, grz);
    back_transform<raw_model(CORR)>(h, o, P);
    NodeMacro<T> out;
    out.rho = T(1) + o.dr;
    out.ux = o.ux;
    out.uy = o.uy;
    out.uz = o.uz;
    return out;
}

// Two collisions (two nodes in the lanes of F2), in place.  The linear transforms
// run in packed FP32x2 instructions; the per-node relaxation runs per lane.
template <int CORR, class Out>
__device__ __forceinline__ void collide_pair(const F2 (&h)[Q], Out &&out, const Phys<float> &P, F2 F0, F2 F1, F2 F2_,
                                             F2 grx = F2(0.f), F2 gry = F2(0.f), F2 grz = F2(0.f))
{
    const RawMoments<F2> m = raw_moments(h, P);
    const PostState<F2> o = relax_node<F2, CORR>(m, P, F0, F1, F2_, grx, gry, grz);
    back_transform_to<raw_model(CORR)>(out, o, P);
}

// Equilibrium deviations h^eq_a = f^eq_a(rho, u) - w_a (init and moving walls).
template <class T>
__device__ __forceinline__ void equilibrium_dev(T (&h)[Q], const Phys<T> &P, T rho, T ux, T uy, T uz)
{
    const AxisCols<T> X = axis_cols(ux, P.ic[0], P.ic2[0], P.w0[0], P.wpm[0]);
    const AxisCols<T> Y = axis_cols(uy, P.ic[1], P.ic2[1], P.w0[1], P.wpm[1]);
    const AxisCols<T> Z = axis_cols(uz, P.ic[2], P.ic2[2], P.w0[2], P.wpm[2]);
    const T dr = rho - T(1);
#pragma unroll
    for (int y = 0; y < 3; ++y)
#pragma unroll
        for (int z = 0; z < 3; ++z) {
            const T Pyz = Y.phi[y] * Z.phi[z];
            const T Dyz = Y.dphi[y] * Z.phi[z] + Y.w[y] * Z.dphi[z];
#pragma unroll
            for (int x = 0; x < 3; ++x)
                h[dir_of(x - 1, y - 1, z - 1)] = (dr * X.phi[x] + X.dphi[x]) * Pyz + X.w[x] * Dyz;
        }
}

}  // namespace lbc
