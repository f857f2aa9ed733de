// ops.cuh -- host-side launchers of the kernels for one storage type.  Each
// step_*.cu instantiates Ops<ST> for one lb_storage value so that the storage
// variants compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "kernels.cuh"
#include "adjoint.cuh"
#include "bulk.cuh"

namespace lbc {

// Everything a launch needs, in double precision; converted per storage type.
struct LaunchArgs {
    Geom g;
    double r, s, cs2, wn, wb;
    double F[3];
    double lid_u;
    double w[Q];
    float scale[Q];
    int corr;
    int model;                // 0 central moments, 1 raw moments (LOCAL corrections only)
    cudaStream_t stream;
    const void *force_field;  // device, compute type, [3][N] or null
    void *rho_field;          // device, compute type, [N] (FULL) or null
    int kernel;               // 0 automatic, 1 one node per thread, 2 two nodes per thread, 3 row-staged,
                              // 4 two nodes per thread marching along z with staged sources, 5 FULL in
                              // one pass
    int *err;                 // device error word of the bounded waits (bulk kernel)
    int sm_count;             // multiprocessors of the device
    unsigned sr_key;          // non-zero: stochastic rounding of 16-bit stores with this step key
};

#ifndef LBC_ADJ_STAGED
#define LBC_ADJ_STAGED 1   // 4-byte storage: the staged z-marching adjoint (0: one node per thread)
#endif

#ifndef LBC_PAIR_PLANES
#define LBC_PAIR_PLANES 1
#endif
// z-planes per thread of the two-node kernel (software pipelining depth).
constexpr int kPairPlanes = LBC_PAIR_PLANES;

// Launch shape of the one-node kernels: every plane of the lattice, or for a step
// launch the planes kz0, kz0 + kzs, ... below kz1.
inline int step_planes(const Geom &g) { return (g.kz1 - g.kz0 + g.kzs - 1) / g.kzs; }

inline void launch_shape(const Geom &g, dim3 &grid, dim3 &block)
{
    int bx = kBlockX;
    while (bx > 1 && bx / 2 >= g.nx) bx /= 2;
    const int by = kBlockThreads / bx;
    block = dim3(bx, by, 1);
    grid = dim3((g.nx + bx - 1) / bx, (g.ny + by - 1) / by, g.nz);
}

template <int ST>
struct Ops {
    using C = Codec<ST>;
    using T = typename C::T;
    using S = typename C::S;

    static DirConst<T> dirs(const LaunchArgs &a)
    {
        DirConst<T> D;
        for (int q = 0; q < Q; ++q) {
            D.w[q] = (T)a.w[q];
            D.scale[q] = a.scale[q];
            D.iscale[q] = 1.0f / a.scale[q];
        }
        return D;
    }
    static Phys<T> phys(const LaunchArgs &a) { return make_phys<T>(a.r, a.s, a.cs2, a.wn, a.wb); }

    static cudaError_t step(const LaunchArgs &a, const void *src, void *dst);
    static bool use_pair(const LaunchArgs &a);
    static bool use_march(const LaunchArgs &a);
    static bool use_full_single_pass(const LaunchArgs &a);
    static cudaError_t step_pair(const LaunchArgs &a, const void *src, void *dst);
    static bool use_bulk(const LaunchArgs &a);
    static cudaError_t step_bulk(const LaunchArgs &a, const void *src, void *dst);
    static const char *step_kernel_name(const LaunchArgs &a);
    static cudaError_t gather(const LaunchArgs &a, const void *src, void *rho, void *u, void *f);
    static cudaError_t scatter(const LaunchArgs &a, void *dst, const void *rho, const void *u, const void *f);
    static cudaError_t reduce_partial(const LaunchArgs &a, const void *src, double *partial, int nblocks,
                                      unsigned *status);
    // adjoint (mean kinetic energy objective); the grid of these launches is
    // launch_shape(a.g), and jpart / wpart hold two doubles per block of it
    static cudaError_t adjoint_seed(const LaunchArgs &a, const void *src, void *lam, void *dJdF, double *jpart);
    static cudaError_t adjoint_step(const LaunchArgs &a, const void *src, const void *lam_in, void *lam_out,
                                    void *dJdF, double *wpart);
    static cudaError_t collide_vjp(const LaunchArgs &a, const void *f, const void *F, const void *L, void *fb,
                                   void *Fb, long long n, double *wpart);
};

inline long long adjoint_blocks(const Geom &g)
{
    dim3 grid, block;
    launch_shape(g, grid, block);
    return (long long)grid.x * grid.y * grid.z;
}

template <int ST>
cudaError_t Ops<ST>::step(const LaunchArgs &a, const void *src, void *dst)
{
    dim3 grid, block;
    launch_shape(a.g, grid, block);
    const Phys<T> P = phys(a);
    const DirConst<T> D = dirs(a);
    const S *s = static_cast<const S *>(src);
    S *d = static_cast<S *>(dst);
    const T *ff = static_cast<const T *>(a.force_field);
    T *rf = static_cast<T *>(a.rho_field);
    if (use_bulk(a)) return step_bulk(a, src, dst);
    if (use_pair(a)) return step_pair(a, src, dst);   // (with its own density pre-pass in FULL mode)
    if (a.corr == LB_CORR_FULL) {
        k_density<ST><<<grid, block, 0, a.stream>>>(s, a.g, P, D, (T)a.lid_u, rf);
    }
    dim3 sgrid = grid;               // the planes this launch updates
    sgrid.z = step_planes(a.g);
    switch (a.corr) {
    case LB_CORR_NONE:
        k_step<ST, LB_CORR_NONE><<<sgrid, block, 0, a.stream>>>(s, d, a.g, P, D, (T)a.F[0], (T)a.F[1], (T)a.F[2],
                                                                ff, rf, (T)a.lid_u, a.sr_key);
        break;
    case LB_CORR_LOWMACH:
        k_step<ST, LB_CORR_LOWMACH><<<sgrid, block, 0, a.stream>>>(s, d, a.g, P, D, (T)a.F[0], (T)a.F[1],
                                                                   (T)a.F[2], ff, rf, (T)a.lid_u, a.sr_key);
        break;
    case LB_CORR_LOCAL:
        if (a.model == 1)
            k_step<ST, LB_CORR_LOCAL | kRawModel><<<sgrid, block, 0, a.stream>>>(
                s, d, a.g, P, D, (T)a.F[0], (T)a.F[1], (T)a.F[2], ff, rf, (T)a.lid_u, a.sr_key);
        else
            k_step<ST, LB_CORR_LOCAL><<<sgrid, block, 0, a.stream>>>(s, d, a.g, P, D, (T)a.F[0], (T)a.F[1],
                                                                     (T)a.F[2], ff, rf, (T)a.lid_u, a.sr_key);
        break;
    default:
        k_step<ST, LB_CORR_FULL><<<sgrid, block, 0, a.stream>>>(s, d, a.g, P, D, (T)a.F[0], (T)a.F[1], (T)a.F[2],
                                                                ff, rf, (T)a.lid_u, a.sr_key);
        break;
    }
    return cudaGetLastError();
}

// The two-node kernel covers the FP32-arithmetic storage forms on lattices with an
// even nx, no walls normal to x, no moving lid and 32-bit offsets (FULL corrections
// with round-to-nearest storage only); everything else takes the one-node kernel.
template <int ST>
bool Ops<ST>::use_pair(const LaunchArgs &a)
{
    if (ST == LB_F64 || a.kernel == 1) return false;   // (kernel 3 falls back here where staging does not apply)
    if (a.model == 1 && a.sr_key != 0) return false;   // raw model with stochastic rounding: one node per thread
    if (a.corr == LB_CORR_FULL && a.sr_key != 0) return false;  // FULL with stochastic rounding: one node per thread
    return (a.g.nx % 2 == 0) && !a.g.wall[0] && a.lid_u == 0.0 &&
           (unsigned long long)Q * (unsigned long long)a.g.N < (1ull << 32);
}

// The z-marching kernel (on request, kernel 4): 16-bit storage on a lattice the
// two-node kernel takes, LOCAL corrections of the central-moment model, contiguous
// planes and rows of at least 64 nodes (one warp per 64-node segment).
template <int ST>
bool Ops<ST>::use_march(const LaunchArgs &a)
{
    return sizeof(S) == 2 && a.kernel == 4 && use_pair(a) && a.corr == LB_CORR_LOCAL && a.model == 0 &&
           a.g.kzs == 1 && a.g.nx >= 2 * kBlockX;
}

// FULL corrections in one pass (on request, kernel 5): the two-node kernel's lattices
// that are periodic in y and z, with rows of a multiple of 64 nodes, stepped whole.  The
// density pre-pass plus two-node step stays the automatic choice: on GB300 it measured
// 19.9 against 19.8 GLUPS (FP32) and 25.0 against 21.7 (BF16) on 512x256x256.
template <int ST>
bool Ops<ST>::use_full_single_pass(const LaunchArgs &a)
{
    return a.kernel == 5 && a.corr == LB_CORR_FULL && a.model == 0 && a.sr_key == 0 && use_pair(a) &&
           !a.g.wall[1] && !a.g.wall[2] && a.g.nx % (2 * kBlockX) == 0 && a.g.kz0 == 0 && a.g.kz1 == a.g.nz &&
           a.g.kzs == 1;
}

#ifndef LBC_OPS_SKIP_PAIR   // defined in the step_*_pair.cu translation units
template <int ST>
cudaError_t Ops<ST>::step_pair(const LaunchArgs &a, const void *src, void *dst)
{
    if constexpr (ST == LB_F64) {
        return cudaErrorInvalidValue;
    } else {
        if constexpr (sizeof(S) == 2) {
            if (use_march(a)) {
                const dim3 block(kBlockX, kBlockThreads / kBlockX, 1);
                const dim3 grid((a.g.nx / 2 + kBlockX - 1) / kBlockX, (a.g.ny + block.y - 1) / block.y,
                                (a.g.kz1 - a.g.kz0 + kMarchPlanes - 1) / kMarchPlanes);
                DirPtrs<S> ptr;
                for (int q = 0; q < Q; ++q) {
                    ptr.src[q] = static_cast<const S *>(src) + (size_t)q * (size_t)a.g.N;
                    ptr.dst[q] = static_cast<S *>(dst) + (size_t)q * (size_t)a.g.N;
                }
                const Phys<float> P = phys(a);
                const DirConst<float> D = dirs(a);
                const float *ff = static_cast<const float *>(a.force_field);
                const float F0 = (float)a.F[0], F1 = (float)a.F[1], F2 = (float)a.F[2];
                const bool sr = a.sr_key != 0, yzw = a.g.wall[1] || a.g.wall[2];
                if (sr && yzw)
                    k_step_march<ST, LB_CORR_LOCAL, true, true><<<grid, block, 0, a.stream>>>(ptr, a.g, P, D, F0, F1,
                                                                                              F2, ff, a.sr_key);
                else if (sr)
                    k_step_march<ST, LB_CORR_LOCAL, true, false><<<grid, block, 0, a.stream>>>(ptr, a.g, P, D, F0, F1,
                                                                                               F2, ff, a.sr_key);
                else if (yzw)
                    k_step_march<ST, LB_CORR_LOCAL, false, true><<<grid, block, 0, a.stream>>>(ptr, a.g, P, D, F0, F1,
                                                                                               F2, ff, 0u);
                else
                    k_step_march<ST, LB_CORR_LOCAL, false, false><<<grid, block, 0, a.stream>>>(ptr, a.g, P, D, F0,
                                                                                                F1, F2, ff, 0u);
                return cudaGetLastError();
            }
        }
        constexpr int ZC = kPairPlanes;
        const int np = a.g.nx / 2;
        int bx = kBlockX;
        while (bx > 1 && bx / 2 >= np) bx /= 2;
        const int by = kBlockThreads / bx;
        if (ZC > 1 && a.g.kzs != 1) return cudaErrorInvalidValue;   // strided planes: one plane per thread
        const dim3 block(bx, by, 1), grid((np + bx - 1) / bx, (a.g.ny + by - 1) / by, (step_planes(a.g) + ZC - 1) / ZC);
        const Phys<float> P = phys(a);
        const DirConst<float> D = dirs(a);
        DirPtrs<S> ptr;
        for (int q = 0; q < Q; ++q) {
            ptr.src[q] = static_cast<const S *>(src) + (size_t)q * (size_t)a.g.N;
            ptr.dst[q] = static_cast<S *>(dst) + (size_t)q * (size_t)a.g.N;
        }
        const float *ff = static_cast<const float *>(a.force_field);
        float *rf = static_cast<float *>(a.rho_field);
        const float F0 = (float)a.F[0], F1 = (float)a.F[1], F2 = (float)a.F[2];
        const bool sr = a.sr_key != 0 && sizeof(S) == 2;
        const bool yzw = a.g.wall[1] || a.g.wall[2];
        if (use_full_single_pass(a)) {
            constexpr int rows = full_rows<ST>();
            constexpr size_t smem = full_smem<ST>();
            static unsigned configured = 0;   // devices whose function attribute is set (bit per device)
            int dev = 0;
            cudaError_t e = cudaGetDevice(&dev);
            if (e != cudaSuccess) return e;
            if (dev < 32 && !(configured & (1u << dev))) {
                e = cudaFuncSetAttribute(k_step_full<ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
                configured |= 1u << dev;
            } else if (dev >= 32) {
                e = cudaFuncSetAttribute(k_step_full<ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
            }
            const dim3 fblock(kBlockX, rows, 1);
            const dim3 fgrid(a.g.nx / (2 * kBlockX), (a.g.ny + rows - 1) / rows, (a.g.nz + kFullPlanes - 1) / kFullPlanes);
            k_step_full<ST><<<fgrid, fblock, smem, a.stream>>>(ptr, a.g, P, D, F0, F1, F2, ff);
            return cudaGetLastError();
        }
        if (a.corr == LB_CORR_FULL) {
            // density pre-pass (one plane per thread), then the step with the gradients
            const dim3 dgrid(grid.x, grid.y, step_planes(a.g));
            if (yzw) {
                k_density_pair<ST, true><<<dgrid, block, 0, a.stream>>>(ptr, a.g, D, rf);
                k_step_pair<ST, LB_CORR_FULL, ZC, false, true><<<grid, block, 0, a.stream>>>(ptr, a.g, P, D, F0, F1, F2,
                                                                                             ff, rf, 0u);
            } else {
                k_density_pair<ST, false><<<dgrid, block, 0, a.stream>>>(ptr, a.g, D, rf);
                k_step_pair<ST, LB_CORR_FULL, ZC, false, false><<<grid, block, 0, a.stream>>>(ptr, a.g, P, D, F0, F1,
                                                                                              F2, ff, rf, 0u);
            }
            return cudaGetLastError();
        }
        switch (a.corr) {
        case LB_CORR_NONE:
            if (sr)
                k_step_pair<ST, LB_CORR_NONE, ZC, true, true><<<grid, block, 0, a.stream>>>(ptr, a.g, P, D, F0, F1, F2, ff, rf,
                                                                                      a.sr_key);
            else
                k_step_pair<ST, LB_CORR_NONE, ZC, false, true><<<grid, block, 0, a.stream>>>(ptr, a.g, P, D, F0, F1, F2, ff, rf,
                                                                                       0u);
            break;
        case LB_CORR_LOWMACH:
            if (sr)
                k_step_pair<ST, LB_CORR_LOWMACH, ZC, true, true><<<grid, block, 0, a.stream>>>(ptr, a.g, P, D, F0, F1, F2,
                                                                                         ff, rf, a.sr_key);
            else
                k_step_pair<ST, LB_CORR_LOWMACH, ZC, false, true><<<grid, block, 0, a.stream>>>(ptr, a.g, P, D, F0, F1, F2,
                                                                                          ff, rf, 0u);
            break;
        default:
            if (a.model == 1)
                k_step_pair<ST, LB_CORR_LOCAL | kRawModel, ZC, false, true><<<grid, block, 0, a.stream>>>(
                    ptr, a.g, P, D, F0, F1, F2, ff, rf, 0u);
            else if (!a.g.wall[1] && !a.g.wall[2] && sr)     // periodic in y and z: no bounce-back tests
                k_step_pair<ST, LB_CORR_LOCAL, ZC, true, false><<<grid, block, 0, a.stream>>>(ptr, a.g, P, D, F0, F1,
                                                                                              F2, ff, rf, a.sr_key);
            else if (!a.g.wall[1] && !a.g.wall[2])
                k_step_pair<ST, LB_CORR_LOCAL, ZC, false, false><<<grid, block, 0, a.stream>>>(ptr, a.g, P, D, F0, F1,
                                                                                               F2, ff, rf, 0u);
            else if (sr)
                k_step_pair<ST, LB_CORR_LOCAL, ZC, true, true><<<grid, block, 0, a.stream>>>(ptr, a.g, P, D, F0, F1, F2, ff, rf,
                                                                                       a.sr_key);
            else
                k_step_pair<ST, LB_CORR_LOCAL, ZC, false, true><<<grid, block, 0, a.stream>>>(ptr, a.g, P, D, F0, F1, F2, ff, rf,
                                                                                        0u);
            break;
        }
        return cudaGetLastError();
    }
}
#endif  // LBC_OPS_SKIP_PAIR

// The staged (bulk-copy) kernel, on request (kernel 3): LOCAL corrections, rows of
// at most 1024 elements whose byte length is a multiple of 16, no walls normal to
// x, no moving lid.  The automatic choice is the two-node kernel: at five CTAs per
// SM it measured 98 % of the copy bandwidth on 512-wide FP32 rows against 93 % for
// this one, and faster for 2-byte storage.
template <int ST>
bool Ops<ST>::use_bulk(const LaunchArgs &a)
{
    if (ST == LB_F64 || a.corr != LB_CORR_LOCAL || a.model != 0 || !a.err) return false;
    if (a.kernel != 3) return false;
    const unsigned elem = (unsigned)sizeof(S);
    return a.g.nx >= 2 && a.g.nx <= 1024 && (a.g.nx * elem) % 16 == 0 && !a.g.wall[0] && a.lid_u == 0.0 &&
           (unsigned long long)Q * (unsigned long long)a.g.N < (1ull << 32);
}

template <int ST, int NXMAX, int NS, int MINB>
cudaError_t launch_bulk(const LaunchArgs &a, const void *src, void *dst)
{
    using S = typename Codec<ST>::S;
    constexpr size_t smem = (size_t)NS * BulkGeom<ST, NXMAX>::stage + NS * (sizeof(uint64_t) + sizeof(unsigned));
    auto kern = k_step_bulk<ST, LB_CORR_LOCAL, NXMAX, NS, MINB>;
    static bool configured = false;   // per instantiation; the attribute is per device function
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    DirPtrs<S> ptr;
    for (int q = 0; q < Q; ++q) {
        ptr.src[q] = static_cast<const S *>(src) + (size_t)q * (size_t)a.g.N;
        ptr.dst[q] = static_cast<S *>(dst) + (size_t)q * (size_t)a.g.N;
    }
    const Phys<float> P = make_phys<float>(a.r, a.s, a.cs2, a.wn, a.wb);
    DirConst<float> D;
    for (int q = 0; q < Q; ++q) {
        D.w[q] = (float)a.w[q];
        D.scale[q] = a.scale[q];
        D.iscale[q] = 1.0f / a.scale[q];
    }
    const long long rows = (long long)a.g.ny * a.g.nz;
    const int grid = (int)std::min<long long>(rows, (long long)a.sm_count * MINB);
    kern<<<grid, kBulkThreads, smem, a.stream>>>(ptr, a.g, P, D, (float)a.F[0], (float)a.F[1], (float)a.F[2],
                                                 static_cast<const float *>(a.force_field), a.err, a.sr_key);
    return cudaGetLastError();
}

// Stage depth and CTAs per multiprocessor: two CTAs of 256 threads per SM
// (<= 128 registers per thread) whenever two sets of stages fit in shared memory.
#ifndef LBC_BULK16_STAGES
#define LBC_BULK16_STAGES 4      // 2-byte storage, rows of up to 512 nodes
#endif
#ifndef LBC_BULK16_MINBLOCKS
#define LBC_BULK16_MINBLOCKS 2
#endif
template <int ST>
cudaError_t Ops<ST>::step_bulk(const LaunchArgs &a, const void *src, void *dst)
{
    if constexpr (ST == LB_F64) {
        return cudaErrorInvalidValue;
    } else if constexpr (sizeof(S) == 4) {
        if (a.g.nx <= 512) return launch_bulk<ST, 512, 2, 2>(a, src, dst);
        return launch_bulk<ST, 1024, 2, 1>(a, src, dst);
    } else {
        if (a.g.nx <= 512) return launch_bulk<ST, 512, LBC_BULK16_STAGES, LBC_BULK16_MINBLOCKS>(a, src, dst);
        return launch_bulk<ST, 1024, 2, 2>(a, src, dst);
    }
}

template <int ST>
cudaError_t Ops<ST>::gather(const LaunchArgs &a, const void *src, void *rho, void *u, void *f)
{
    dim3 grid, block;
    launch_shape(a.g, grid, block);
    k_gather<ST><<<grid, block, 0, a.stream>>>(static_cast<const S *>(src), a.g, phys(a), dirs(a), (T)a.F[0],
                                               (T)a.F[1], (T)a.F[2], static_cast<const T *>(a.force_field),
                                               (T)a.lid_u, static_cast<T *>(rho), static_cast<T *>(u),
                                               static_cast<T *>(f));
    return cudaGetLastError();
}

template <int ST>
cudaError_t Ops<ST>::scatter(const LaunchArgs &a, void *dst, const void *rho, const void *u, const void *f)
{
    dim3 grid, block;
    launch_shape(a.g, grid, block);
    k_scatter<ST><<<grid, block, 0, a.stream>>>(static_cast<S *>(dst), a.g, phys(a), dirs(a),
                                                static_cast<const T *>(rho), static_cast<const T *>(u),
                                                static_cast<const T *>(f));
    return cudaGetLastError();
}

template <int ST>
cudaError_t Ops<ST>::reduce_partial(const LaunchArgs &a, const void *src, double *partial, int nblocks,
                                    unsigned *status)
{
    k_reduce_partial<ST><<<nblocks, kReduceThreads, 0, a.stream>>>(
        static_cast<const S *>(src), a.g, phys(a), dirs(a), (T)a.F[0], (T)a.F[1], (T)a.F[2],
        static_cast<const T *>(a.force_field), (T)a.lid_u, partial, status);
    return cudaGetLastError();
}

#ifndef LBC_OPS_SKIP_ADJOINT   // defined in the step_*_adjoint.cu translation units
template <int ST>
cudaError_t Ops<ST>::adjoint_seed(const LaunchArgs &a, const void *src, void *lam, void *dJdF, double *jpart)
{
    dim3 grid, block;
    launch_shape(a.g, grid, block);
    k_adjoint_seed<ST><<<grid, block, 0, a.stream>>>(static_cast<const S *>(src), a.g, phys(a), dirs(a), (T)a.F[0],
                                                     (T)a.F[1], (T)a.F[2], static_cast<const T *>(a.force_field),
                                                     static_cast<T *>(lam), static_cast<T *>(dJdF), jpart);
    return cudaGetLastError();
}

template <int ST>
cudaError_t Ops<ST>::adjoint_step(const LaunchArgs &a, const void *src, const void *lam_in, void *lam_out,
                                  void *dJdF, double *wpart)
{
    dim3 grid, block;
    launch_shape(a.g, grid, block);
    const S *s = static_cast<const S *>(src);
    const T *li = static_cast<const T *>(lam_in);
    T *lo = static_cast<T *>(lam_out);
    const T *ff = static_cast<const T *>(a.force_field);
    T *dF = static_cast<T *>(dJdF);
    const Phys<T> P = phys(a);
    const DirConst<T> D = dirs(a);
    if constexpr (sizeof(S) == 4 && LBC_ADJ_STAGED) {
        // 4-byte storage: the z-marching adjoint with its state and lambda words staged in
        // shared memory (same grid in x and y, kAdjPlanes planes per thread)
        const dim3 mgrid(grid.x, grid.y, (a.g.nz + kAdjPlanes - 1) / kAdjPlanes);
        // devices on which each kernel's shared-memory attribute is set (bit per device,
        // one word per correction mode: the three kernels share one function type)
        static unsigned configured[3] = {0, 0, 0};
        auto launch = [&](auto kern, int m) -> cudaError_t {
            int dev = 0;
            cudaError_t e = cudaGetDevice(&dev);
            if (e != cudaSuccess) return e;
            if (dev >= 32 || !(configured[m] & (1u << dev))) {
                e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdjStageBytes);
                if (e != cudaSuccess) return e;
                if (dev < 32) configured[m] |= 1u << dev;
            }
            kern<<<mgrid, block, kAdjStageBytes, a.stream>>>(s, li, lo, a.g, P, D, (T)a.F[0], (T)a.F[1], (T)a.F[2], ff,
                                                             dF, wpart);
            return cudaGetLastError();
        };
        switch (a.corr) {
        case LB_CORR_NONE: return launch(k_adjoint_march<ST, LB_CORR_NONE>, 0);
        case LB_CORR_LOWMACH: return launch(k_adjoint_march<ST, LB_CORR_LOWMACH>, 1);
        case LB_CORR_LOCAL: return launch(k_adjoint_march<ST, LB_CORR_LOCAL>, 2);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (a.corr) {
    case LB_CORR_NONE:
        k_adjoint<ST, LB_CORR_NONE><<<grid, block, 0, a.stream>>>(s, li, lo, a.g, P, D, (T)a.F[0], (T)a.F[1],
                                                                   (T)a.F[2], ff, dF, wpart);
        break;
    case LB_CORR_LOWMACH:
        k_adjoint<ST, LB_CORR_LOWMACH><<<grid, block, 0, a.stream>>>(s, li, lo, a.g, P, D, (T)a.F[0], (T)a.F[1],
                                                                      (T)a.F[2], ff, dF, wpart);
        break;
    case LB_CORR_LOCAL:
        k_adjoint<ST, LB_CORR_LOCAL><<<grid, block, 0, a.stream>>>(s, li, lo, a.g, P, D, (T)a.F[0], (T)a.F[1],
                                                                    (T)a.F[2], ff, dF, wpart);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int ST>
cudaError_t Ops<ST>::collide_vjp(const LaunchArgs &a, const void *f, const void *F, const void *L, void *fb,
                                 void *Fb, long long n, double *wpart)
{
    const int blocks = (int)((n + kAdjThreads - 1) / kAdjThreads);
    const T *pf = static_cast<const T *>(f), *pF = static_cast<const T *>(F), *pL = static_cast<const T *>(L);
    T *pfb = static_cast<T *>(fb), *pFb = static_cast<T *>(Fb);
    const Phys<T> P = phys(a);
    const DirConst<T> D = dirs(a);
    switch (a.corr) {
    case LB_CORR_NONE:
        k_collide_vjp<ST, LB_CORR_NONE><<<blocks, kAdjThreads, 0, a.stream>>>(pf, pF, pL, pfb, pFb, n, P, D, wpart);
        break;
    case LB_CORR_LOWMACH:
        k_collide_vjp<ST, LB_CORR_LOWMACH><<<blocks, kAdjThreads, 0, a.stream>>>(pf, pF, pL, pfb, pFb, n, P, D,
                                                                                 wpart);
        break;
    case LB_CORR_LOCAL:
        k_collide_vjp<ST, LB_CORR_LOCAL><<<blocks, kAdjThreads, 0, a.stream>>>(pf, pF, pL, pfb, pFb, n, P, D, wpart);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
#endif  // LBC_OPS_SKIP_ADJOINT

// Name of the kernel that step() launches for these arguments (the same
// decision as step(), spelled with the template arguments).
inline const char *storage_name(int st)
{
    switch (st) {
    case LB_F64: return "F64";
    case LB_F32: return "F32";
    case LB_F32_SHIFTED: return "F32_SHIFTED";
    case LB_F16_SHIFTED: return "F16_SHIFTED";
    default: return "BF16_SHIFTED";
    }
}

inline const char *corr_name(int c)
{
    switch (c) {
    case LB_CORR_NONE: return "NONE";
    case LB_CORR_LOWMACH: return "LOWMACH";
    case LB_CORR_LOCAL: return "LOCAL";
    default: return "FULL";
    }
}

template <int ST>
const char *Ops<ST>::step_kernel_name(const LaunchArgs &a)
{
    static thread_local char buf[96];
    if (use_bulk(a)) {
        const bool wide = sizeof(S) == 4, small = a.g.nx <= 512;
        const int nxmax = small ? 512 : 1024;
        const int ns = wide ? 2 : (small ? LBC_BULK16_STAGES : 2);
        const int minb = (wide && !small) ? 1 : (!wide && small ? LBC_BULK16_MINBLOCKS : 2);
        snprintf(buf, sizeof(buf), "k_step_bulk<%s,%s,%d,%d,%d>", storage_name(ST), corr_name(a.corr), nxmax, ns,
                 minb);
    } else if (use_full_single_pass(a)) {
        snprintf(buf, sizeof(buf), "k_step_full<%s,%d,%d>", storage_name(ST), full_rows<ST>(), kFullPlanes);
    } else if (use_march(a)) {
        snprintf(buf, sizeof(buf), "k_step_march<%s,%s,%d,%s,%s>", storage_name(ST), corr_name(a.corr), kMarchPlanes,
                 a.sr_key != 0 ? "true" : "false", (a.g.wall[1] || a.g.wall[2]) ? "walls" : "periodic");
    } else if (use_pair(a)) {
        const bool yzw = a.g.wall[1] || a.g.wall[2] || a.model == 1 ||
                         (a.corr != LB_CORR_LOCAL && a.corr != LB_CORR_FULL);
        snprintf(buf, sizeof(buf), "k_step_pair<%s,%s%s,%d,%s,%s>", storage_name(ST), corr_name(a.corr),
                 a.model == 1 ? "|RAW" : "", kPairPlanes,
                 (a.sr_key != 0 && sizeof(S) == 2) ? "true" : "false", yzw ? "walls" : "periodic");
    } else {
        snprintf(buf, sizeof(buf), "k_step<%s,%s%s>", storage_name(ST), corr_name(a.corr),
                 a.model == 1 ? "|RAW" : "");
    }
    return buf;
}

}  // namespace lbc
