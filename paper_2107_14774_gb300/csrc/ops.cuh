// ops.cuh -- host-side launchers of the kernels for one storage type.  Each
// step_*.cu instantiates Ops<ST> for one lb_storage value so that the storage
// variants compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include "kernels.cuh"

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
    cudaStream_t stream;
    const void *force_field;  // device, compute type, [3][N] or null
    void *rho_field;          // device, compute type, [N] (FULL) or null
};

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
    static cudaError_t gather(const LaunchArgs &a, const void *src, void *rho, void *u, void *f);
    static cudaError_t scatter(const LaunchArgs &a, void *dst, const void *rho, const void *u, const void *f);
    static cudaError_t reduce_partial(const LaunchArgs &a, const void *src, double *partial, int nblocks,
                                      unsigned *status);
};

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
    if (a.corr == LB_CORR_FULL) {
        k_density<ST><<<grid, block, 0, a.stream>>>(s, a.g, P, D, (T)a.lid_u, rf);
    }
    switch (a.corr) {
    case LB_CORR_NONE:
        k_step<ST, LB_CORR_NONE><<<grid, block, 0, a.stream>>>(s, d, a.g, P, D, (T)a.F[0], (T)a.F[1], (T)a.F[2],
                                                                ff, rf, (T)a.lid_u);
        break;
    case LB_CORR_LOWMACH:
        k_step<ST, LB_CORR_LOWMACH><<<grid, block, 0, a.stream>>>(s, d, a.g, P, D, (T)a.F[0], (T)a.F[1],
                                                                   (T)a.F[2], ff, rf, (T)a.lid_u);
        break;
    case LB_CORR_LOCAL:
        k_step<ST, LB_CORR_LOCAL><<<grid, block, 0, a.stream>>>(s, d, a.g, P, D, (T)a.F[0], (T)a.F[1], (T)a.F[2],
                                                                 ff, rf, (T)a.lid_u);
        break;
    default:
        k_step<ST, LB_CORR_FULL><<<grid, block, 0, a.stream>>>(s, d, a.g, P, D, (T)a.F[0], (T)a.F[1], (T)a.F[2],
                                                                ff, rf, (T)a.lid_u);
        break;
    }
    return cudaGetLastError();
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

}  // namespace lbc
