// kernels.cuh -- CUDA kernels of liblbcuboid (templates; instantiated per storage
// type in step_*.cu).
//
// State layout ("pull" convention).  The context stores S[27][N]: after a step,
// S_a(x) holds the post-collision population f~_a(x, t) of node x itself.  The
// pre-collision population of the next step is then obtained by streaming
// (Sec. 3.2: f_a(x, t+1) = f~_a(x - e_a, t)) when it is read:
//     f_a(x) = S_a(x - e_a)              if x - e_a is inside (periodic axes wrap)
//     f_a(x) = S_opp(a)(x) + lid term    if x - e_a lies beyond a wall
// (half-way bounce-back, Sec. 4).  Every stored value is read by exactly one
// (node, direction) pair, so one fused kernel reads 27 and writes 27 values per
// node and nothing else.
#pragma once

#include "collide.cuh"

namespace lbc {

// ---------------------------------------------------------------------------
// Stochastic rounding of the 16-bit storage forms (optional, lb_config.rounding).
// Random bits: the lowbias32 integer hash (C. Wellons) of a per-node key, then one
// xorshift32 step (G. Marsaglia, 2003) per stored value.  The conversion is the
// hardware stochastic-rounding cvt.rs of sm_100+ (unbiased: E[round(x)] = x).
__device__ __forceinline__ unsigned hash32(unsigned x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
__device__ __forceinline__ unsigned xorshift32(unsigned &s)
{
    s ^= s << 13;
    s ^= s >> 17;
    s ^= s << 5;
    return s;
}
// Packed pair: `lo` goes to the lower 16 bits, `hi` to the upper ones.
__device__ __forceinline__ unsigned cvt_rs_bf16x2(float lo, float hi, unsigned rbits)
{
    unsigned d;
    asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
    return d;
}
__device__ __forceinline__ unsigned cvt_rs_f16x2(float lo, float hi, unsigned rbits)
{
    unsigned d;
    asm("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
    return d;
}

constexpr int kBlockX = 32;   // threads along x per block
constexpr int kBlockThreads = 128;

// Source coordinates x - e of one node along each axis: index 0 for e = -1,
// 1 for e = 0, 2 for e = +1.  out[] marks sources beyond a wall.
struct Pull {
    long long base;     // index of the node itself
    int xs[3];          // x - e_x
    long long yoff[3];  // (y - e_y) * nx
    long long zoff[3];  // (z - e_z) * nx * ny
    bool xo[3], yo[3], zo[3];
};

__device__ __forceinline__ void axis_sources(int c, int n, int wall, int (&src)[3], bool (&out)[3])
{
    // e = -1 -> c + 1, e = 0 -> c, e = +1 -> c - 1
    int p = c + 1, m = c - 1;
    out[0] = false;
    out[1] = false;
    out[2] = false;
    if (p >= n) {
        if (wall) out[0] = true;
        p -= n;
    }
    if (m < 0) {
        if (wall) out[2] = true;
        m += n;
    }
    src[0] = p;
    src[1] = c;
    src[2] = m;
}

__device__ __forceinline__ Pull make_pull(const Geom &g, int i, int j, int k)
{
    Pull q;
    int ys[3], zs[3];
    axis_sources(i, g.nx, g.wall[0], q.xs, q.xo);
    axis_sources(j, g.ny, g.wall[1], ys, q.yo);
    axis_sources(k, g.nz, g.wall[2], zs, q.zo);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        q.yoff[t] = (long long)ys[t] * g.nx;
        q.zoff[t] = (long long)zs[t] * g.nx * g.ny;
    }
    q.base = q.zoff[1] + q.yoff[1] + i;
    return q;
}

// Storage offset read for direction a at this node.
template <int A>
__device__ __forceinline__ long long pull_offset(const Pull &q, long long N)
{
    constexpr int cx = ex(A) + 1, cy = ey(A) + 1, cz = ez(A) + 1;
    const bool out = q.xo[cx] | q.yo[cy] | q.zo[cz];
    const long long in_off = (long long)A * N + q.zoff[cz] + q.yoff[cy] + q.xs[cx];
    const long long bb_off = (long long)opp(A) * N + q.base;
    return out ? bb_off : in_off;
}

// Does direction a reach this node across the lid (the wall at j = ny - 1/2)?
template <int A>
__device__ __forceinline__ bool from_lid(const Pull &q)
{
    return ey(A) == -1 && q.yo[0];
}

template <int ST, int A>
struct LoadDir {
    using C = Codec<ST>;
    using T = typename C::T;
    static __device__ __forceinline__ void run(T (&h)[Q], const typename C::S *__restrict__ src,
                                               const Pull &q, long long N, const DirConst<T> &D)
    {
        h[A] = C::load(__ldg(src + pull_offset<A>(q, N)), D.w[A], D.iscale[A]);
        LoadDir<ST, A + 1>::run(h, src, q, N, D);
    }
};
template <int ST>
struct LoadDir<ST, Q> {
    using C = Codec<ST>;
    using T = typename C::T;
    static __device__ __forceinline__ void run(T (&)[Q], const typename C::S *__restrict__, const Pull &,
                                               long long, const DirConst<T> &) {}
};

// Pre-collision deviations h_a = f_a(x, t) - w_a of one node, streamed in.
// With a moving lid the incoming links across it get the momentum-augmented
// term -[f^eq_opp(a) - f^eq_a](rho_w, U) of Sec. 4, with
// the wall density taken as the fluid node's density sum_a S_a(x) (mass is
// conserved by the collision, so this is rho(x, t-1)).
template <int ST>
__device__ __forceinline__ void pull_node(typename Codec<ST>::T (&h)[Q], const typename Codec<ST>::S *__restrict__ src,
                                          const Pull &q, long long N, const DirConst<typename Codec<ST>::T> &D,
                                          const Phys<typename Codec<ST>::T> &P, typename Codec<ST>::T lid_u)
{
    using C = Codec<ST>;
    using T = typename C::T;
    LoadDir<ST, 0>::run(h, src, q, N, D);
    if (lid_u != T(0) && q.yo[0]) {
        T rho_w = T(1);
#pragma unroll
        for (int a = 0; a < Q; ++a) rho_w += C::load(__ldg(src + (long long)a * N + q.base), D.w[a], D.iscale[a]);
        // f^eq(rho_w, (U,0,0)): only the x factor depends on U; the correction
        // f^eq_a - f^eq_opp(a) = rho_w phi_y phi_z (phi_x(ex) - phi_x(-ex)) = rho_w phi_y phi_z ex U
        const AxisCols<T> Y = axis_cols(T(0), P.ic[1], P.ic2[1], P.w0[1], P.wpm[1]);
        const AxisCols<T> Z = axis_cols(T(0), P.ic[2], P.ic2[2], P.w0[2], P.wpm[2]);
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            if (ey(a) == -1 && ex(a) != 0) {
                // incoming a, outgoing b = opp(a): f_a = f~_b - [f^eq_b - f^eq_a]
                //                                      = f~_b + rho_w phi_y phi_z ex(a) U
                h[a] += rho_w * Y.phi[ey(a) + 1] * Z.phi[ez(a) + 1] * T(ex(a)) * lid_u;
            }
        }
    }
}

template <int ST, int CORR>
__global__ void __launch_bounds__(kBlockThreads)
k_step(const typename Codec<ST>::S *__restrict__ src, typename Codec<ST>::S *__restrict__ dst, Geom g,
       Phys<typename Codec<ST>::T> P, DirConst<typename Codec<ST>::T> D, typename Codec<ST>::T F0,
       typename Codec<ST>::T F1, typename Codec<ST>::T F2, const typename Codec<ST>::T *__restrict__ ff,
       const typename Codec<ST>::T *__restrict__ rho_field, typename Codec<ST>::T lid_u, unsigned sr_key)
{
    using C = Codec<ST>;
    using T = typename C::T;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = g.kz0 + (int)blockIdx.z * g.kzs;
    if (i >= g.nx || j >= g.ny) return;
    const long long N = g.N;
    const Pull q = make_pull(g, i, j, k);
    T h[Q];
    pull_node<ST>(h, src, q, N, D, P, lid_u);
    T Fx = F0, Fy = F1, Fz = F2;
    if (ff) {
        Fx += __ldg(ff + q.base);
        Fy += __ldg(ff + N + q.base);
        Fz += __ldg(ff + 2 * N + q.base);
    }
    T grx = T(0), gry = T(0), grz = T(0);
    if (CORR == LB_CORR_FULL) {
        // second-order central differences of the current density; one-sided
        // second-order differences next to a wall (spacings 1, r, s)
        const int n[3] = {g.nx, g.ny, g.nz};
        const int c[3] = {i, j, k};
        const long long stride[3] = {1, (long long)g.nx, (long long)g.nx * g.ny};
        T gr[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const T ih = P.ic[ax];
            const long long x = q.base, st = stride[ax];
            T d = T(0);
            if (n[ax] == 1) {
                d = T(0);
            } else if (!g.wall[ax]) {
                const long long xp = (c[ax] == n[ax] - 1) ? x - (long long)(n[ax] - 1) * st : x + st;
                const long long xm = (c[ax] == 0) ? x + (long long)(n[ax] - 1) * st : x - st;
                d = (__ldg(rho_field + xp) - __ldg(rho_field + xm)) * (T(0.5) * ih);
            } else if (n[ax] == 2) {
                d = (c[ax] == 0 ? __ldg(rho_field + x + st) - __ldg(rho_field + x)
                                : __ldg(rho_field + x) - __ldg(rho_field + x - st)) * ih;
            } else if (c[ax] == 0) {
                d = (T(-3) * __ldg(rho_field + x) + T(4) * __ldg(rho_field + x + st) - __ldg(rho_field + x + 2 * st))
                    * (T(0.5) * ih);
            } else if (c[ax] == n[ax] - 1) {
                d = (T(3) * __ldg(rho_field + x) - T(4) * __ldg(rho_field + x - st) + __ldg(rho_field + x - 2 * st))
                    * (T(0.5) * ih);
            } else {
                d = (__ldg(rho_field + x + st) - __ldg(rho_field + x - st)) * (T(0.5) * ih);
            }
            gr[ax] = d;
        }
        grx = gr[0];
        gry = gr[1];
        grz = gr[2];
    }
    collide<T, CORR>(h, P, Fx, Fy, Fz, grx, gry, grz);
    if (ST == LB_F16_SHIFTED || ST == LB_BF16_SHIFTED) {
        if (sr_key) {
            const unsigned gbase = (unsigned)q.base + (unsigned)g.zofs * (unsigned)g.nx * (unsigned)g.ny;
            unsigned rs = hash32(gbase * 0x9e3779b1u + sr_key) | 1u;
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                const unsigned r = xorshift32(rs);
                const float v = (float)h[a] * D.scale[a];
                const unsigned packed = (ST == LB_F16_SHIFTED) ? cvt_rs_f16x2(v, 0.f, r) : cvt_rs_bf16x2(v, 0.f, r);
                reinterpret_cast<unsigned short *>(dst)[(long long)a * N + q.base] = (unsigned short)(packed & 0xffffu);
            }
            return;
        }
    }
#pragma unroll
    for (int a = 0; a < Q; ++a) dst[(long long)a * N + q.base] = C::store(h[a], D.w[a], D.scale[a]);
}

// ---------------------------------------------------------------------------
// Two-node variant of k_step for the FP32-arithmetic storage forms.  Each thread
// updates the x-adjacent nodes (i0, i0+1), i0 even: populations with ex = 0 and
// every store move as one aligned 2-element vector; the two x-shifted source
// elements of ex = +-1 are single loads.  The linear parts of the collision run
// in packed FP32x2 instructions (collide_pair).  Offsets are 32-bit (the host
// only selects this kernel when 27 N < 2^32), the source row of each (ey, ez) is
// computed once, and periodic wrap in y and z is folded into those row offsets.
// Requirements (checked on the host): nx even, no walls normal to x, no moving
// lid, corrections other than FULL.

// Raw stored pair of two x-adjacent values (what the loads return) and its
// decoding into deviations h, per storage type.  Keeping the raw words lets a
// thread hold the next plane's loads in flight while it computes the current one.
template <int ST> struct PairIO;
template <> struct PairIO<LB_F32> {
    using S = float;
    using Raw = float2;
    static __device__ __forceinline__ Raw ld2(const S *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
    static __device__ __forceinline__ Raw ld11(const S *p0, const S *p1) { return make_float2(__ldg(p0), __ldg(p1)); }
    static __device__ __forceinline__ F2 dec(Raw r, float w, float) { return F2(r) - F2(w); }
    static __device__ __forceinline__ void st2(S *p, F2 h, float w, float)
    {
        *reinterpret_cast<float2 *>(p) = (h + F2(w)).v;
    }
    static __device__ __forceinline__ void st2sr(S *p, F2 h, float w, float s, unsigned) { st2(p, h, w, s); }
};
template <> struct PairIO<LB_F32_SHIFTED> {
    using S = float;
    using Raw = float2;
    static __device__ __forceinline__ Raw ld2(const S *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
    static __device__ __forceinline__ Raw ld11(const S *p0, const S *p1) { return make_float2(__ldg(p0), __ldg(p1)); }
    static __device__ __forceinline__ F2 dec(Raw r, float, float) { return F2(r); }
    static __device__ __forceinline__ void st2(S *p, F2 h, float, float) { *reinterpret_cast<float2 *>(p) = h.v; }
    static __device__ __forceinline__ void st2sr(S *p, F2 h, float w, float s, unsigned) { st2(p, h, w, s); }
};
// 16-bit forms: the raw word holds the element at the lower address in its low half.
__device__ __forceinline__ unsigned ld16x2(const void *p) { return __ldg(reinterpret_cast<const unsigned *>(p)); }
__device__ __forceinline__ unsigned ld16_16(const void *p0, const void *p1)
{
    const unsigned lo = __ldg(reinterpret_cast<const unsigned short *>(p0));
    const unsigned hi = __ldg(reinterpret_cast<const unsigned short *>(p1));
    return __byte_perm(lo, hi, 0x5410);
}
template <> struct PairIO<LB_F16_SHIFTED> {
    using S = __half;
    using Raw = unsigned;
    static __device__ __forceinline__ Raw ld2(const S *p) { return ld16x2(p); }
    static __device__ __forceinline__ Raw ld11(const S *p0, const S *p1) { return ld16_16(p0, p1); }
    static __device__ __forceinline__ F2 dec(Raw r, float, float iscale)
    {
        __half2 v;
        memcpy(&v, &r, sizeof(v));
        return F2(__half22float2(v)) * F2(iscale);
    }
    static __device__ __forceinline__ void st2(S *p, F2 h, float, float scale)
    {
        *reinterpret_cast<__half2 *>(p) = __float22half2_rn((h * F2(scale)).v);
    }
    static __device__ __forceinline__ void st2sr(S *p, F2 h, float, float scale, unsigned rbits)
    {
        const F2 v = h * F2(scale);
        *reinterpret_cast<unsigned *>(p) = cvt_rs_f16x2(v.v.x, v.v.y, rbits);
    }
};
template <> struct PairIO<LB_BF16_SHIFTED> {
    using S = __nv_bfloat16;
    using Raw = unsigned;
    static __device__ __forceinline__ Raw ld2(const S *p) { return ld16x2(p); }
    static __device__ __forceinline__ Raw ld11(const S *p0, const S *p1) { return ld16_16(p0, p1); }
    static __device__ __forceinline__ F2 dec(Raw r, float, float)
    {
        // a bfloat16 is the upper half of the float with the same bits
        return F2(__uint_as_float(r << 16), __uint_as_float(r & 0xffff0000u));
    }
    static __device__ __forceinline__ void st2(S *p, F2 h, float, float)
    {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __float22bfloat162_rn(h.v);
    }
    static __device__ __forceinline__ void st2sr(S *p, F2 h, float, float, unsigned rbits)
    {
        *reinterpret_cast<unsigned *>(p) = cvt_rs_bf16x2(h.v.x, h.v.y, rbits);
    }
};

// Base pointers of the 27 direction arrays of the source and destination
// buffers, passed by value so that every load and store address is one
// multiply-add of a 32-bit element index onto a kernel-parameter pointer.
template <class S>
struct DirPtrs {
    const S *src[Q];
    S *dst[Q];
};

// Issue the loads of the two nodes (i0, i0+1) of row j, plane k.  YZW: the lattice
// has walls normal to y or z (without them no link is tested for a bounce-back).
template <int ST, bool YZW>
__device__ __forceinline__ void pair_fetch(typename PairIO<ST>::Raw (&raw)[Q], const DirPtrs<typename Codec<ST>::S> &ptr,
                                           const Geom &g, int i0, unsigned xm, unsigned xp, const int (&ys)[3],
                                           const bool (&yo)[3], int k)
{
    using IO = PairIO<ST>;
    int zs[3];
    bool zo[3];
    axis_sources(k, g.nz, g.wall[2], zs, zo);
    const unsigned nx = (unsigned)g.nx, nxy = (unsigned)g.nx * (unsigned)g.ny;
    unsigned rowbase[3][3];
#pragma unroll
    for (int cy = 0; cy < 3; ++cy)
#pragma unroll
        for (int cz = 0; cz < 3; ++cz) rowbase[cy][cz] = (unsigned)zs[cz] * nxy + (unsigned)ys[cy] * nx;
    const unsigned self = rowbase[1][1] + (unsigned)i0;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int cx = ex(a) + 1, cy = ey(a) + 1, cz = ez(a) + 1;
        if (YZW && (yo[cy] | zo[cz])) {
            // half-way bounce-back across a y or z wall: f_a(x) = S_opp(a)(x) for both nodes
            raw[a] = IO::ld2(ptr.src[opp(a)] + self);
        } else {
            const unsigned rb = rowbase[cy][cz];
            const typename Codec<ST>::S *p = ptr.src[a];
            if (cx == 1)
                raw[a] = IO::ld2(p + (rb + (unsigned)i0));
            else if (cx == 2)   // ex = +1: sources i0 - 1, i0
                raw[a] = IO::ld11(p + (rb + xm), p + (rb + (unsigned)i0));
            else                // ex = -1: sources i0 + 1, i0 + 2
                raw[a] = IO::ld11(p + (rb + (unsigned)i0 + 1u), p + (rb + xp));
        }
    }
}

// Density gradient along y or z of the two nodes at `self` (index of the first) from
// the density field: second-order central differences (periodic wrap), one-sided
// second-order differences next to a wall, first order if the axis has two nodes
// (c: the nodes' coordinate on the axis, n its extent, st its stride, ih = 1/spacing).
__device__ __forceinline__ F2 ld_rho2(const float *rf, unsigned i)
{
    return F2(__ldg(reinterpret_cast<const float2 *>(rf + i)));
}
__device__ __forceinline__ F2 grad_pair_axis(const float *__restrict__ rf, unsigned self, unsigned st, int c, int n,
                                             int wall, float ih)
{
    if (n == 1) return F2(0.f);
    if (!wall) {
        const unsigned p = (c == n - 1) ? self - (unsigned)(n - 1) * st : self + st;
        const unsigned m = (c == 0) ? self + (unsigned)(n - 1) * st : self - st;
        return (ld_rho2(rf, p) - ld_rho2(rf, m)) * F2(0.5f * ih);
    }
    if (n == 2)
        return (c == 0 ? ld_rho2(rf, self + st) - ld_rho2(rf, self) : ld_rho2(rf, self) - ld_rho2(rf, self - st)) *
               F2(ih);
    if (c == 0)
        return (F2(-3.f) * ld_rho2(rf, self) + F2(4.f) * ld_rho2(rf, self + st) - ld_rho2(rf, self + 2u * st)) *
               F2(0.5f * ih);
    if (c == n - 1)
        return (F2(3.f) * ld_rho2(rf, self) - F2(4.f) * ld_rho2(rf, self - st) + ld_rho2(rf, self - 2u * st)) *
               F2(0.5f * ih);
    return (ld_rho2(rf, self + st) - ld_rho2(rf, self - st)) * F2(0.5f * ih);
}

// Density pre-pass of LB_CORR_FULL for the two-node kernel: the pre-collision density
// of the nodes (i0, i0+1), pulled with the same loads as the step (sum of the 27
// deviations in direction order, as in k_density).
template <int ST, bool YZW>
__global__ void __launch_bounds__(kBlockThreads)
k_density_pair(DirPtrs<typename Codec<ST>::S> ptr, Geom g, DirConst<float> D, float *__restrict__ rho)
{
    using IO = PairIO<ST>;
    const int i0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = g.kz0 + (int)blockIdx.z * g.kzs;
    if (i0 >= g.nx || j >= g.ny) return;
    const unsigned nx = (unsigned)g.nx, nxy = (unsigned)g.nx * (unsigned)g.ny;
    int ys[3];
    bool yo[3];
    axis_sources(j, g.ny, g.wall[1], ys, yo);
    const unsigned xm = (i0 == 0) ? nx - 1u : (unsigned)i0 - 1u;
    const unsigned xp = (i0 + 2 == g.nx) ? 0u : (unsigned)i0 + 2u;
    typename IO::Raw raw[Q];
    pair_fetch<ST, YZW>(raw, ptr, g, i0, xm, xp, ys, yo, k);
    F2 s(0.f);
#pragma unroll
    for (int a = 0; a < Q; ++a) s += IO::dec(raw[a], D.w[a], D.iscale[a]);
    const unsigned self = (unsigned)k * nxy + (unsigned)j * nx + (unsigned)i0;
    *reinterpret_cast<float2 *>(rho + self) = (F2(1.f) + s).v;
}

// ZC consecutive planes per thread: the loads of plane k+1 are issued before the
// collision of plane k, so that every warp keeps memory requests in flight while
// it computes (software pipelining across z).
// Resident CTAs per SM requested from the compiler.  With walls normal to y or z five
// CTAs of 128 threads (at most 102 registers; the compiler takes 96 and spills a few
// words) hide the load latency better than four at 126 registers: measured on GB300,
// FP32 on 768-wide rows with y walls 25.2 -> 31.4 GLUPS, BF16 and FP16 on that channel
// 38.2 -> 41.5 and 34.8 -> 38.1.  Without y/z walls the kernel issues fewer instructions
// per load and runs best at four CTAs (up to 126 registers, no spill): FP32 30.3 -> 32.1
// GLUPS on the 512x256x256 decaying flow, BF16 45.8 -> 47.6, FP16 44.7 -> 45.1.
// Stochastic rounding keeps five: at four, BF16 + SR ran 43.2 against 43.6 GLUPS and
// FP16 + SR 40.1 against 41.5 on the decaying flow.
#ifndef LBC_PAIR_MINBLOCKS
#define LBC_PAIR_MINBLOCKS 5
#endif
#ifndef LBC_PAIR_SR_MINBLOCKS
#define LBC_PAIR_SR_MINBLOCKS 5
#endif
#ifndef LBC_PAIR_PERIODIC_MINBLOCKS
#define LBC_PAIR_PERIODIC_MINBLOCKS 4
#endif
template <int ST, bool SR, bool YZW>
constexpr int pair_min_blocks()
{
    return SR ? LBC_PAIR_SR_MINBLOCKS : (!YZW ? LBC_PAIR_PERIODIC_MINBLOCKS : LBC_PAIR_MINBLOCKS);
}
template <int ST, int CORR, int ZC, bool SR, bool YZW>
__global__ void __launch_bounds__(kBlockThreads, pair_min_blocks<ST, SR, YZW>())
k_step_pair(DirPtrs<typename Codec<ST>::S> ptr, Geom g, Phys<float> P, DirConst<float> D, float F0, float F1,
            float F2s, const float *__restrict__ ff, const float *__restrict__ rf, unsigned sr_key)
{
    using IO = PairIO<ST>;
    const int i0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = g.kz0 + (int)blockIdx.z * ZC * g.kzs;
    if (i0 >= g.nx || j >= g.ny) return;
    const int kend = ZC == 1 ? k0 + 1 : min(k0 + ZC, g.kz1);   // the grid covers exactly the planes
    const unsigned nx = (unsigned)g.nx, nxy = (unsigned)g.nx * (unsigned)g.ny;
    int ys[3];
    bool yo[3];
    axis_sources(j, g.ny, g.wall[1], ys, yo);
    const unsigned xm = (i0 == 0) ? nx - 1u : (unsigned)i0 - 1u;       // source of ex = +1 for node i0
    const unsigned xp = (i0 + 2 == g.nx) ? 0u : (unsigned)i0 + 2u;     // source of ex = -1 for node i0+1
    typename IO::Raw raw[Q];
    pair_fetch<ST, YZW>(raw, ptr, g, i0, xm, xp, ys, yo, k0);
    for (int k = k0; k < kend; ++k) {
        F2 h[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) h[a] = IO::dec(raw[a], D.w[a], D.iscale[a]);
        if (k + 1 < kend) pair_fetch<ST, YZW>(raw, ptr, g, i0, xm, xp, ys, yo, k + 1);
        const unsigned self = (unsigned)k * nxy + (unsigned)j * nx + (unsigned)i0;
        F2 Fx(F0), Fy(F1), Fz(F2s);
        if (ff) {
            const unsigned N = (unsigned)g.N;
            Fx += F2(__ldg(reinterpret_cast<const float2 *>(ff + self)));
            Fy += F2(__ldg(reinterpret_cast<const float2 *>(ff + N + self)));
            Fz += F2(__ldg(reinterpret_cast<const float2 *>(ff + 2u * N + self)));
        }
        F2 grx(0.f), gry(0.f), grz(0.f);
        if constexpr (corr_mode(CORR) == LB_CORR_FULL) {
            // density gradient of both nodes from the density pre-pass (the same
            // stencils as the one-node kernel; x is periodic in this kernel)
            const unsigned row = self - (unsigned)i0;
            const F2 rc(__ldg(reinterpret_cast<const float2 *>(rf + self)));
            grx = F2(rc.v.y - __ldg(rf + row + xm), __ldg(rf + row + xp) - rc.v.x) * F2(0.5f * P.ic[0]);
            gry = grad_pair_axis(rf, self, nx, j, g.ny, g.wall[1], P.ic[1]);
            grz = grad_pair_axis(rf, self, nxy, k, g.nz, g.wall[2], P.ic[2]);
        }
        if constexpr (SR) {
            unsigned rs = hash32((self + (unsigned)g.zofs * nxy) * 0x9e3779b1u + sr_key) | 1u;
            collide_pair<CORR>(
                h, [&](int a, F2 v) { IO::st2sr(ptr.dst[a] + self, v, D.w[a], D.scale[a], xorshift32(rs)); }, P, Fx,
                Fy, Fz, grx, gry, grz);
        } else {
            collide_pair<CORR>(h, [&](int a, F2 v) { IO::st2(ptr.dst[a] + self, v, D.w[a], D.scale[a]); }, P, Fx, Fy,
                               Fz, grx, gry, grz);
        }
    }
}

// FULL corrections in one pass (lattices periodic in y and z, rows of a multiple of 64
// nodes).  A CTA owns a tile of 64 nodes x ROWS rows and marches kFullPlanes planes along
// z.  Before colliding plane k it computes the densities of plane k + 1 for the tile and
// its axis halo -- the rows above and below, and the node on either side of each row --
// into a ring of four density planes in shared memory; the gradient of plane k then
// comes from the ring (second-order central differences, as in the two-node kernel).
// Every density is the sum of a node pair's 27 pulled deviations in direction order,
// exactly as in k_density_pair, so the result equals the two-pass path bit for bit.  A
// thread's own pair is among the pairs whose density it computes, so the words it pulls
// for plane k + 1 are parked in its column of a two-plane stash in shared memory and
// collided from there one iteration later: the populations of a plane are read from
// HBM once; the halo pulls are served from L2.
#ifndef LBC_FULL_PLANES
#define LBC_FULL_PLANES 16
#endif
constexpr int kFullPlanes = LBC_FULL_PLANES;
constexpr int kFullW = 2 * kBlockX + 2;   // the tile's 64 nodes and one on either side
// Rows per CTA: 8 for 2-byte storage, 4 for 4-byte storage (the stash holds two planes
// of the CTA's raw words: 55 KB either way, so that three CTAs fit an SM).
template <int ST>
__host__ __device__ constexpr int full_rows() { return sizeof(typename Codec<ST>::S) == 2 ? 8 : 4; }
template <int ST>
__host__ __device__ constexpr size_t full_smem()
{
    return (size_t)4 * (full_rows<ST>() + 2) * kFullW * sizeof(float) +
           (size_t)2 * Q * full_rows<ST>() * kBlockX * sizeof(typename PairIO<ST>::Raw);
}

// Pulled words and density of the node pair (i0, i0 + 1) of row j, plane k of a lattice
// periodic in y and z.
template <int ST>
__device__ __forceinline__ F2 pair_pull_density(typename PairIO<ST>::Raw (&raw)[Q],
                                                const DirPtrs<typename Codec<ST>::S> &ptr, const Geom &g,
                                                const DirConst<float> &D, int i0, int j, int k)
{
    using IO = PairIO<ST>;
    int ys[3];
    bool yo[3];
    axis_sources(j, g.ny, 0, ys, yo);
    const unsigned nx = (unsigned)g.nx;
    const unsigned xm = (i0 == 0) ? nx - 1u : (unsigned)i0 - 1u;
    const unsigned xp = (i0 + 2 == g.nx) ? 0u : (unsigned)i0 + 2u;
    pair_fetch<ST, false>(raw, ptr, g, i0, xm, xp, ys, yo, k);
    F2 s(0.f);
#pragma unroll
    for (int a = 0; a < Q; ++a) s += IO::dec(raw[a], D.w[a], D.iscale[a]);
    return F2(1.f) + s;
}

// Resident CTAs per SM: three of 128 threads for 4-byte storage (168 registers), two of
// 256 threads for 2-byte storage (128 registers; three would spill).
template <int ST>
__host__ __device__ constexpr int full_min_blocks() { return sizeof(typename Codec<ST>::S) == 2 ? 2 : 3; }

template <int ST>
__global__ void __launch_bounds__(kBlockX * full_rows<ST>(), full_min_blocks<ST>())
k_step_full(DirPtrs<typename Codec<ST>::S> ptr, Geom g, Phys<float> P, DirConst<float> D, float F0, float F1,
            float F2s, const float *__restrict__ ff)
{
    using IO = PairIO<ST>;
    using Raw = typename IO::Raw;
    constexpr int ROWS = full_rows<ST>();
    constexpr int NT = kBlockX * ROWS;
    extern __shared__ __align__(16) char full_smem_raw[];
    // ring of density planes: row 0 = the row above the tile, rows 1..rows = the tile,
    // row rows + 1 = the row below; column 0 = the node left of the tile, 1..64 the
    // tile, 65 the node right of it
    auto R = reinterpret_cast<float (*)[ROWS + 2][kFullW]>(full_smem_raw);
    // stash[plane & 1][a][thread]: the raw words of each thread's own pair
    auto stash = reinterpret_cast<Raw (*)[Q][NT]>(full_smem_raw + (size_t)4 * (ROWS + 2) * kFullW * sizeof(float));
    const int lane = threadIdx.x, wy = threadIdx.y;
    const int t = wy * kBlockX + lane;
    const int i0t = (int)blockIdx.x * 2 * kBlockX;
    const int j0 = (int)blockIdx.y * ROWS;
    const int rows = min(ROWS, g.ny - j0);
    const int k0 = (int)blockIdx.z * kFullPlanes;
    const int kend = min(k0 + kFullPlanes, g.nz);
    const int nint = rows * kBlockX, ntask = nint + 2 * kBlockX + 2 * rows;

    // densities of plane kk (periodic in z) into ring slot (kk + 4) & 3; the thread's own
    // pair (task t < nint: row wy, pair lane) also goes to stash slot kk & 1
    auto densities = [&](int kk) {
        const int kw = kk < 0 ? kk + g.nz : (kk >= g.nz ? kk - g.nz : kk);
        float (*Rs)[kFullW] = R[(kk + 4) & 3];
        for (int task = t; task < ntask; task += NT) {
            Raw raw[Q];
            if (task < nint) {                       // the tile's own pairs
                const int r = task / kBlockX, p = task % kBlockX;
                const F2 rho = pair_pull_density<ST>(raw, ptr, g, D, i0t + 2 * p, j0 + r, kw);
                Rs[1 + r][1 + 2 * p] = rho.v.x;
                Rs[1 + r][2 + 2 * p] = rho.v.y;
                if (task == t) {
#pragma unroll
                    for (int a = 0; a < Q; ++a) stash[kk & 1][a][t] = raw[a];
                }
            } else if (task < nint + 2 * kBlockX) {  // the rows above and below
                const int h = (task - nint) / kBlockX, p = (task - nint) % kBlockX;
                int jj = h == 0 ? j0 - 1 : j0 + rows;
                jj = jj < 0 ? jj + g.ny : (jj >= g.ny ? jj - g.ny : jj);
                const F2 rho = pair_pull_density<ST>(raw, ptr, g, D, i0t + 2 * p, jj, kw);
                const int rr = h == 0 ? 0 : rows + 1;
                Rs[rr][1 + 2 * p] = rho.v.x;
                Rs[rr][2 + 2 * p] = rho.v.y;
            } else {                                 // the nodes left and right of each row
                const int q = task - nint - 2 * kBlockX, r = q / 2, side = q % 2;
                if (side == 0) {
                    const int il = i0t == 0 ? g.nx - 2 : i0t - 2;
                    Rs[1 + r][0] = pair_pull_density<ST>(raw, ptr, g, D, il, j0 + r, kw).v.y;
                } else {
                    const int ir = i0t + 2 * kBlockX == g.nx ? 0 : i0t + 2 * kBlockX;
                    Rs[1 + r][kFullW - 1] = pair_pull_density<ST>(raw, ptr, g, D, ir, j0 + r, kw).v.x;
                }
            }
        }
    };

    densities(k0 - 1);
    densities(k0);
    const int i0 = i0t + 2 * lane, j = j0 + wy;
    const bool on = wy < rows;
    const unsigned nx = (unsigned)g.nx, nxy = (unsigned)g.nx * (unsigned)g.ny;
    const int c = 1 + 2 * lane, r = 1 + wy;
    for (int k = k0; k < kend; ++k) {
        densities(k + 1);
        __syncthreads();   // plane k + 1 complete; planes k - 1 and k were completed before
        if (on) {
            F2 h[Q];
#pragma unroll
            for (int a = 0; a < Q; ++a) h[a] = IO::dec(stash[k & 1][a][t], D.w[a], D.iscale[a]);
            const unsigned self = (unsigned)k * nxy + (unsigned)j * nx + (unsigned)i0;
            F2 Fx(F0), Fy(F1), Fz(F2s);
            if (ff) {
                const unsigned N = (unsigned)g.N;
                Fx += F2(__ldg(reinterpret_cast<const float2 *>(ff + self)));
                Fy += F2(__ldg(reinterpret_cast<const float2 *>(ff + N + self)));
                Fz += F2(__ldg(reinterpret_cast<const float2 *>(ff + 2u * N + self)));
            }
            const float (*Rc)[kFullW] = R[(k + 4) & 3];
            const float (*Rm)[kFullW] = R[(k + 3) & 3];
            const float (*Rp)[kFullW] = R[(k + 5) & 3];
            const F2 grx = (F2(Rc[r][c + 1], Rc[r][c + 2]) - F2(Rc[r][c - 1], Rc[r][c])) * F2(0.5f * P.ic[0]);
            const F2 gry = g.ny == 1 ? F2(0.f)
                                     : (F2(Rc[r + 1][c], Rc[r + 1][c + 1]) - F2(Rc[r - 1][c], Rc[r - 1][c + 1])) *
                                           F2(0.5f * P.ic[1]);
            const F2 grz = g.nz == 1 ? F2(0.f)
                                     : (F2(Rp[r][c], Rp[r][c + 1]) - F2(Rm[r][c], Rm[r][c + 1])) * F2(0.5f * P.ic[2]);
            collide_pair<LB_CORR_FULL>(h, [&](int a, F2 v) { IO::st2(ptr.dst[a] + self, v, D.w[a], D.scale[a]); },
                                       P, Fx, Fy, Fz, grx, gry, grz);
        }
    }
}

// Two nodes per thread marching along z, with the sources of the next plane staged in
// shared memory (16-bit storage).  A warp owns one 64-node segment of row j (32 words,
// a word being the two 16-bit values of a node pair) and kMarchPlanes consecutive
// planes.  For each direction it copies the 32 words of the segment in the source row,
// plus the word left of the segment (e_x = +1) or right of it (e_x = -1), into shared
// memory with per-lane 4-byte cp.async, and cuts the x-shifted pairs out of two
// neighbouring words there.  The copies of plane k + 1 are issued as soon as plane k
// has been read out of the stage, so they are in flight while plane k is collided and
// stored, without holding registers.
#ifndef LBC_MARCH_PLANES
#define LBC_MARCH_PLANES 8
#endif
#ifndef LBC_MARCH_MINBLOCKS
#define LBC_MARCH_MINBLOCKS 5
#endif
constexpr int kMarchPlanes = LBC_MARCH_PLANES;
constexpr int kStageWords = kBlockX + 2;   // the segment's words and one on either side

__device__ __forceinline__ void cp_async4(unsigned *smem, const unsigned *gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Issue the copies of plane k into stage[a][0 .. kStageWords): the lane's own word
// (index wi of its row) at 1 + lane; lane 0 adds the word wl left of the segment, the
// last active lane the word wr right of it.  Across a y or z wall the source is the
// node's own word of the opposite direction (half-way bounce-back).
template <int ST, bool YZW>
__device__ __forceinline__ void march_issue(unsigned (*stage)[kStageWords], const DirPtrs<typename Codec<ST>::S> &ptr,
                                            const Geom &g, int lane, bool left, bool right, unsigned wi, unsigned wl,
                                            unsigned wr, const int (&ys)[3], const bool (&yo)[3], int k)
{
    int zs[3];
    bool zo[3];
    axis_sources(k, g.nz, g.wall[2], zs, zo);
    const unsigned hx = (unsigned)g.nx >> 1, hxy = hx * (unsigned)g.ny;   // words per row, per plane
    unsigned rowbase[3][3];
#pragma unroll
    for (int cy = 0; cy < 3; ++cy)
#pragma unroll
        for (int cz = 0; cz < 3; ++cz) rowbase[cy][cz] = (unsigned)zs[cz] * hxy + (unsigned)ys[cy] * hx;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int cx = ex(a) + 1, cy = ey(a) + 1, cz = ez(a) + 1;
        if (YZW && (yo[cy] | zo[cz])) {
            cp_async4(&stage[a][1 + lane], reinterpret_cast<const unsigned *>(ptr.src[opp(a)]) + rowbase[1][1] + wi);
        } else {
            const unsigned *p = reinterpret_cast<const unsigned *>(ptr.src[a]) + rowbase[cy][cz];
            cp_async4(&stage[a][1 + lane], p + wi);
            if (cx == 2 && left) cp_async4(&stage[a][0], p + wl);
            if (cx == 0 && right) cp_async4(&stage[a][2 + lane], p + wr);
        }
    }
    cp_async_commit();
}

// The raw words of the lane's two nodes at plane k from the stage (the element of the
// first node in the low half, as the loads of pair_fetch give them).
template <int ST, bool YZW>
__device__ __forceinline__ void march_read(unsigned (&raw)[Q], const unsigned (*stage)[kStageWords], const Geom &g,
                                           int lane, const bool (&yo)[3], int k)
{
    int zs[3];
    bool zo[3];
    axis_sources(k, g.nz, g.wall[2], zs, zo);
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int cx = ex(a) + 1, cy = ey(a) + 1, cz = ez(a) + 1;
        if (cx == 1 || (YZW && (yo[cy] | zo[cz])))
            raw[a] = stage[a][1 + lane];
        else if (cx == 2)   // ex = +1: sources i0 - 1 (high half of the left word), i0
            raw[a] = __byte_perm(stage[a][lane], stage[a][1 + lane], 0x5432);
        else                // ex = -1: sources i0 + 1, i0 + 2 (low half of the right word)
            raw[a] = __byte_perm(stage[a][1 + lane], stage[a][2 + lane], 0x5432);
    }
}

template <int ST, int CORR, bool SR, bool YZW>
__global__ void __launch_bounds__(kBlockThreads, LBC_MARCH_MINBLOCKS)
k_step_march(DirPtrs<typename Codec<ST>::S> ptr, Geom g, Phys<float> P, DirConst<float> D, float F0, float F1,
             float F2s, const float *__restrict__ ff, unsigned sr_key)
{
    using IO = PairIO<ST>;
    static_assert(sizeof(typename Codec<ST>::S) == 2, "k_step_march stages 16-bit storage");
    __shared__ unsigned stage_all[kBlockThreads / kBlockX][Q][kStageWords];
    const int lane = threadIdx.x;   // blockDim.x == kBlockX: one warp per row segment
    const int i0 = 2 * ((int)blockIdx.x * kBlockX + lane);
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = g.kz0 + (int)blockIdx.z * kMarchPlanes;
    if (j >= g.ny) return;          // the whole warp
    const bool on = i0 < g.nx;
    const unsigned act = __ballot_sync(0xffffffffu, on);
    if (!on) return;
    const int last = 31 - __clz(act);   // the active lanes are 0 .. last
    const int kend = min(k0 + kMarchPlanes, g.kz1);
    unsigned (*stage)[kStageWords] = stage_all[threadIdx.y];
    const unsigned nx = (unsigned)g.nx, nxy = (unsigned)g.nx * (unsigned)g.ny;
    int ys[3];
    bool yo[3];
    axis_sources(j, g.ny, g.wall[1], ys, yo);
    const unsigned wi = (unsigned)i0 >> 1;
    const unsigned wl = (i0 == 0 ? nx : (unsigned)i0) / 2u - 1u;   // word of node i0 - 1 (periodic in x)
    const unsigned wr = (i0 + 2 == g.nx) ? 0u : wi + 1u;            // word of node i0 + 2
    march_issue<ST, YZW>(stage, ptr, g, lane, lane == 0, lane == last, wi, wl, wr, ys, yo, k0);
    for (int k = k0; k < kend; ++k) {
        cp_async_wait_all();
        __syncwarp(act);
        unsigned raw[Q];
        march_read<ST, YZW>(raw, stage, g, lane, yo, k);
        __syncwarp(act);
        if (k + 1 < kend) march_issue<ST, YZW>(stage, ptr, g, lane, lane == 0, lane == last, wi, wl, wr, ys, yo, k + 1);
        F2 h[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) h[a] = IO::dec(raw[a], D.w[a], D.iscale[a]);
        const unsigned self = (unsigned)k * nxy + (unsigned)j * nx + (unsigned)i0;
        F2 Fx(F0), Fy(F1), Fz(F2s);
        if (ff) {
            const unsigned N = (unsigned)g.N;
            Fx += F2(__ldg(reinterpret_cast<const float2 *>(ff + self)));
            Fy += F2(__ldg(reinterpret_cast<const float2 *>(ff + N + self)));
            Fz += F2(__ldg(reinterpret_cast<const float2 *>(ff + 2u * N + self)));
        }
        if constexpr (SR) {
            unsigned rs = hash32((self + (unsigned)g.zofs * nxy) * 0x9e3779b1u + sr_key) | 1u;
            collide_pair<CORR>(
                h, [&](int a, F2 v) { IO::st2sr(ptr.dst[a] + self, v, D.w[a], D.scale[a], xorshift32(rs)); }, P, Fx,
                Fy, Fz);
        } else {
            collide_pair<CORR>(h, [&](int a, F2 v) { IO::st2(ptr.dst[a] + self, v, D.w[a], D.scale[a]); }, P, Fx, Fy,
                               Fz);
        }
    }
}

// Density of every node (pre-pass of LB_CORR_FULL).
template <int ST>
__global__ void __launch_bounds__(kBlockThreads)
k_density(const typename Codec<ST>::S *__restrict__ src, Geom g, Phys<typename Codec<ST>::T> P,
          DirConst<typename Codec<ST>::T> D, typename Codec<ST>::T lid_u, typename Codec<ST>::T *__restrict__ rho)
{
    using T = typename Codec<ST>::T;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const Pull q = make_pull(g, i, j, k);
    T h[Q];
    pull_node<ST>(h, src, q, g.N, D, P, lid_u);
    T s = T(0);
#pragma unroll
    for (int a = 0; a < Q; ++a) s += h[a];
    rho[q.base] = T(1) + s;
}

// Density and velocity (Eq. 12) of every node; and/or the pre-collision
// populations f_a = w_a + h_a.  Any output pointer may be null.
template <int ST>
__global__ void __launch_bounds__(kBlockThreads)
k_gather(const typename Codec<ST>::S *__restrict__ src, Geom g, Phys<typename Codec<ST>::T> P,
         DirConst<typename Codec<ST>::T> D, typename Codec<ST>::T F0, typename Codec<ST>::T F1,
         typename Codec<ST>::T F2, const typename Codec<ST>::T *__restrict__ ff, typename Codec<ST>::T lid_u,
         typename Codec<ST>::T *__restrict__ rho, typename Codec<ST>::T *__restrict__ u,
         typename Codec<ST>::T *__restrict__ fout)
{
    using T = typename Codec<ST>::T;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const long long N = g.N;
    const Pull q = make_pull(g, i, j, k);
    T h[Q];
    pull_node<ST>(h, src, q, N, D, P, lid_u);
    if (fout) {
#pragma unroll
        for (int a = 0; a < Q; ++a) fout[(long long)a * N + q.base] = D.w[a] + h[a];
    }
    if (rho || u) {
        const RawMoments<T> m = raw_moments(h, P);
        T Fx = F0, Fy = F1, Fz = F2;
        if (ff) {
            Fx += ff[q.base];
            Fy += ff[N + q.base];
            Fz += ff[2 * N + q.base];
        }
        const T r = T(1) + m.dr;
        if (rho) rho[q.base] = r;
        if (u) {
            u[q.base] = (m.jx + T(0.5) * Fx) / r;
            u[N + q.base] = (m.jy + T(0.5) * Fy) / r;
            u[2 * N + q.base] = (m.jz + T(0.5) * Fz) / r;
        }
    }
}

// Write pre-collision deviations h of node x into the pull layout (inverse of
// pull_node, without lid terms): S_a(x - e_a) or, across a wall, S_opp(a)(x).
template <int ST>
__device__ __forceinline__ void scatter_node(const typename Codec<ST>::T (&h)[Q], typename Codec<ST>::S *__restrict__ dst,
                                             const Pull &q, long long N, const DirConst<typename Codec<ST>::T> &D)
{
    using C = Codec<ST>;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int cx = ex(a) + 1, cy = ey(a) + 1, cz = ez(a) + 1;
        const bool out = q.xo[cx] | q.yo[cy] | q.zo[cz];
        const long long off = out ? (long long)opp(a) * N + q.base
                                  : (long long)a * N + q.zoff[cz] + q.yoff[cy] + q.xs[cx];
        dst[off] = C::store(h[a], D.w[a], D.scale[a]);
    }
}

// f := f^eq(rho, u) (init), or f := given populations (set).
template <int ST>
__global__ void __launch_bounds__(kBlockThreads)
k_scatter(typename Codec<ST>::S *__restrict__ dst, Geom g, Phys<typename Codec<ST>::T> P,
          DirConst<typename Codec<ST>::T> D, const typename Codec<ST>::T *__restrict__ rho,
          const typename Codec<ST>::T *__restrict__ u, const typename Codec<ST>::T *__restrict__ fin)
{
    using T = typename Codec<ST>::T;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const long long N = g.N;
    const Pull q = make_pull(g, i, j, k);
    T h[Q];
    if (fin) {
#pragma unroll
        for (int a = 0; a < Q; ++a) h[a] = fin[(long long)a * N + q.base] - D.w[a];
    } else {
        equilibrium_dev(h, P, rho[q.base], u[q.base], u[N + q.base], u[2 * N + q.base]);
    }
    scatter_node<ST>(h, dst, q, N, D);
}

// First pass of the FP64 reduction: per-block sums of rho and rho u (Eq. 12) in
// a fixed tree order, plus a status bit for non-finite or non-positive density.
constexpr int kReduceThreads = 256;

template <int ST>
__global__ void __launch_bounds__(kReduceThreads)
k_reduce_partial(const typename Codec<ST>::S *__restrict__ src, Geom g, Phys<typename Codec<ST>::T> P,
                 DirConst<typename Codec<ST>::T> D, typename Codec<ST>::T F0, typename Codec<ST>::T F1,
                 typename Codec<ST>::T F2, const typename Codec<ST>::T *__restrict__ ff,
                 typename Codec<ST>::T lid_u, double *__restrict__ partial, unsigned *__restrict__ status)
{
    using T = typename Codec<ST>::T;
    __shared__ double sh[4][kReduceThreads];
    const long long N = g.N;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    unsigned bad = 0;
    // grid-stride over nodes in a fixed order
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(n % g.nx);
        const long long t = n / g.nx;
        const int j = (int)(t % g.ny);
        const int k = (int)(t / g.ny);
        const Pull q = make_pull(g, i, j, k);
        T h[Q];
        pull_node<ST>(h, src, q, N, D, P, lid_u);
        const RawMoments<T> m = raw_moments(h, P);
        T Fx = F0, Fy = F1, Fz = F2;
        if (ff) {
            Fx += ff[n];
            Fy += ff[N + n];
            Fz += ff[2 * N + n];
        }
        const double rho = 1.0 + (double)m.dr;
        const double jx = (double)m.jx + 0.5 * (double)Fx;
        const double jy = (double)m.jy + 0.5 * (double)Fy;
        const double jz = (double)m.jz + 0.5 * (double)Fz;
        if (!(rho > 0.0) || !isfinite(rho) || !isfinite(jx) || !isfinite(jy) || !isfinite(jz)) bad = 1u;
        acc[0] += rho;
        acc[1] += jx;
        acc[2] += jy;
        acc[3] += jz;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int s = kReduceThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < 4; ++c) partial[4 * blockIdx.x + c] = sh[c][0];
    if (bad) atomicOr(status, 1u);
}

// Second pass: one block sums the per-block partials in a fixed order.
__global__ void __launch_bounds__(kReduceThreads)
k_reduce_final(const double *__restrict__ partial, int nblocks, double *__restrict__ out);

}  // namespace lbc
