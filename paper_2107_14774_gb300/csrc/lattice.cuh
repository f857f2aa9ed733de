// lattice.cuh -- D3Q27 stencil of the cuboid lattice, per-axis constants and
// population storage codecs (device side of liblbcuboid).
//
// The integer stencil and its ordering are those of the paper (Eq. 1a-1c: the
// cuboid velocities are (ex, r*ey, s*ez) with the integer components below).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "lbcuboid.h"

namespace lbc {

constexpr int Q = 27;

// Integer components of direction a (paper ordering, Eq. 1a-1c).
__host__ __device__ constexpr int ex(int a)
{
    constexpr int t[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
    return t[a];
}
__host__ __device__ constexpr int ey(int a)
{
    constexpr int t[Q] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1, 1, 1, -1, -1};
    return t[a];
}
__host__ __device__ constexpr int ez(int a)
{
    constexpr int t[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1};
    return t[a];
}
// Direction with the opposite velocity.
__host__ __device__ constexpr int opp(int a)
{
    int r = 0;
    for (int b = 0; b < Q; ++b)
        if (ex(b) == -ex(a) && ey(b) == -ey(a) && ez(b) == -ez(a)) r = b;
    return r;
}
// Direction with integer velocity (x, y, z), each in {-1, 0, 1}.
__host__ __device__ constexpr int dir_of(int x, int y, int z)
{
    int r = 0;
    for (int b = 0; b < Q; ++b)
        if (ex(b) == x && ey(b) == y && ez(b) == z) r = b;
    return r;
}

// Physical constants of one context, in the compute type T.  Per axis
// (0 = x with speed 1, 1 = y with speed r, 2 = z with speed s):
//   ic  = 1/c, ic2 = 1/c^2,
//   w0  = 1 - cs2/c^2 and wpm = cs2/(2 c^2): the rest weights of the 1-D
//         three-velocity distribution with moments (1, 0, cs2), rounded so
//         that w0 + 2 wpm = 1 holds exactly in T;
//   cs2ax = 2 wpm c^2: the second moment those rounded weights carry;
//   an  = 3 cs2 - c^2 (anisotropy factor of Eq. 38-40).
template <class T>
struct Phys {
    T c[3], ic[3], ic2[3], w0[3], wpm[3], an[3], cs2ax[3];
    T cs2;
    T wn, wb;          // omega_nu, omega_xi
    T tn, tb;          // 1/omega - 1/2
    T two_cs2_wn, two_cs2_wb;
};

template <class T>
inline Phys<T> make_phys(double r, double s, double cs2, double wn, double wb)
{
    Phys<T> p;
    const double c[3] = {1.0, r, s};
    for (int i = 0; i < 3; ++i) {
        p.c[i] = (T)c[i];
        p.ic[i] = (T)(1.0 / c[i]);
        p.ic2[i] = (T)(1.0 / (c[i] * c[i]));
        // The equilibrium factor of each axis is phi = w + dphi with sum(dphi) = 0, so
        // every collision multiplies the mass deviation and the momentum by the sums
        // w0 + 2 wpm of the other axes.  Rounded independently to FP32 these sums miss
        // 1 by up to 3e-8 (2/3 + 2 (1/6) rounds to 1 + 2^-25), which compounds into a
        // steady growth of the velocity amplitude of 6e-8 per step; so the larger of
        // the two weights is rounded and the other is formed from it exactly (the
        // subtraction from 1 is exact by Sterbenz's lemma, halving/doubling are exact).
        const double q = cs2 / (c[i] * c[i]);
        T w0, wpm;
        if (q <= 0.5) {
            w0 = (T)(1.0 - q);
            wpm = (T(1) - w0) * T(0.5);
        } else {
            wpm = (T)(0.5 * q);
            w0 = T(1) - T(2) * wpm;
        }
        p.w0[i] = w0;
        p.wpm[i] = wpm;
        p.cs2ax[i] = (T)(2.0 * (double)wpm * c[i] * c[i]);
        p.an[i] = (T)(3.0 * cs2 - c[i] * c[i]);
    }
    p.cs2 = (T)cs2;
    p.wn = (T)wn;
    p.wb = (T)wb;
    p.tn = (T)(1.0 / wn - 0.5);
    p.tb = (T)(1.0 / wb - 0.5);
    p.two_cs2_wn = (T)(2.0 * cs2 / wn);
    p.two_cs2_wb = (T)(2.0 * cs2 / wb);
    return p;
}

// ---------------------------------------------------------------------------
// Storage codecs.  Every kernel works on the deviation h_a = f_a - w_a (rho0 = 1)
// in the compute type; the codec converts between h and the stored value.

template <int ST> struct Codec;

template <> struct Codec<LB_F64> {
    using S = double;
    using T = double;
    static constexpr bool shifted = false;
    static __device__ __forceinline__ T load(S v, T w, float) { return v - w; }
    static __device__ __forceinline__ S store(T h, T w, float) { return w + h; }
};
template <> struct Codec<LB_F32> {
    using S = float;
    using T = float;
    static constexpr bool shifted = false;
    static __device__ __forceinline__ T load(S v, T w, float) { return v - w; }
    static __device__ __forceinline__ S store(T h, T w, float) { return w + h; }
};
template <> struct Codec<LB_F32_SHIFTED> {
    using S = float;
    using T = float;
    static constexpr bool shifted = true;
    static __device__ __forceinline__ T load(S v, T, float) { return v; }
    static __device__ __forceinline__ S store(T h, T, float) { return h; }
};
// binary16 with a per-direction power-of-two scale (multiplication by an exact
// power of two is exact, so only the final round to nearest even loses bits).
template <> struct Codec<LB_F16_SHIFTED> {
    using S = __half;
    using T = float;
    static constexpr bool shifted = true;
    static __device__ __forceinline__ T load(S v, T, float inv_scale) { return __half2float(v) * inv_scale; }
    static __device__ __forceinline__ S store(T h, T, float scale) { return __float2half_rn(h * scale); }
};
template <> struct Codec<LB_BF16_SHIFTED> {
    using S = __nv_bfloat16;
    using T = float;
    static constexpr bool shifted = true;
    static __device__ __forceinline__ T load(S v, T, float) { return __bfloat162float(v); }
    static __device__ __forceinline__ S store(T h, T, float) { return __float2bfloat16_rn(h); }
};

// Per-direction constants passed by value to the kernels.
template <class T>
struct DirConst {
    T w[Q];            // rest weights w_a = f^eq_a(1, 0)
    float scale[Q];    // storage scale (FP16 only; 1 otherwise)
    float iscale[Q];
};

// Grid geometry: extents, wall flags and the stride of each axis.  A step launch
// updates the z-planes kz0, kz0 + kzs, ... below kz1 (all planes: 0, 1, nz); zofs
// is the global z index of plane 0, which differs from 0 only in a sub-domain (a
// z-slab with ghost planes) and enters only the stochastic-rounding draws, so that a
// decomposed run draws the same bits as the whole lattice.
struct Geom {
    int nx, ny, nz;
    int wall[3];       // 1 = half-way bounce-back walls normal to that axis
    long long N;       // nx * ny * nz
    int kz0, kz1, kzs; // planes updated by a step launch
    int zofs;          // global z of plane 0
};

}  // namespace lbc
