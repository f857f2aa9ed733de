// bulk.cuh -- persistent, row-staged variant of the fused step: the 27 source
// rows of each lattice row are streamed into shared memory with bulk
// asynchronous copies (cp.async.bulk + mbarrier transaction counts) several rows
// ahead, while all warps of the CTA collide from shared memory and store to
// global memory.
//
// Row-wise staging fits the pull layout exactly: for an x-row (j, k) of the
// destination, direction a needs the whole source row (j - e_ay, k - e_az) of
// array a (periodic y/z wrap folded into the row index; across a y or z wall the
// row (j, k) of array opp(a)), shifted by -e_ax along x with periodic wrap, which
// is an index shift inside shared memory.  Every global byte is read once, the
// copies are 16-byte aligned contiguous rows, and no thread holds registers for
// loads in flight.
//
// Every mbarrier wait is bounded: after kSpinLimit polls the thread records an
// error code in *err and leaves (the issuing thread first waits, again bounded,
// for the copies it has issued), so a lost arrival can never hang the GPU.
#pragma once

#include <stdint.h>

#include "kernels.cuh"

namespace lbc {

constexpr int kBulkThreads = 256;
constexpr unsigned kSpinLimit = 1u << 22;

enum : int { kErrNone = 0, kErrFullWait = 1, kErrEmptyWait = 2 };

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false if the limit ran out.
// Repeated polls back off with a short sleep so that waiting warps leave the
// issue slots to the warps that are computing.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, unsigned limit = kSpinLimit)
{
    for (unsigned it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it >= 2) __nanosleep(64);
    }
    return false;
}

// Asynchronous copy of `bytes` (multiple of 16, 16-byte aligned ends) from global
// memory to shared memory, completing `bytes` transactions on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Shared-memory element of the staged rows: 16-bit words for the half formats.
template <int ST> struct BulkIO;
template <> struct BulkIO<LB_F32> {
    using S = float;
    static __device__ __forceinline__ F2 ld2(const char *row, unsigned xa, unsigned xb, float w, float)
    {
        return F2(*reinterpret_cast<const float *>(row + 4u * xa), *reinterpret_cast<const float *>(row + 4u * xb)) -
               F2(w);
    }
    static __device__ __forceinline__ F2 ld2a(const char *row, unsigned x, float w, float)
    {
        return F2(*reinterpret_cast<const float2 *>(row + 4u * x)) - F2(w);
    }
};
template <> struct BulkIO<LB_F32_SHIFTED> {
    using S = float;
    static __device__ __forceinline__ F2 ld2(const char *row, unsigned xa, unsigned xb, float, float)
    {
        return F2(*reinterpret_cast<const float *>(row + 4u * xa), *reinterpret_cast<const float *>(row + 4u * xb));
    }
    static __device__ __forceinline__ F2 ld2a(const char *row, unsigned x, float, float)
    {
        return F2(*reinterpret_cast<const float2 *>(row + 4u * x));
    }
};
template <> struct BulkIO<LB_F16_SHIFTED> {
    using S = __half;
    static __device__ __forceinline__ F2 ld2(const char *row, unsigned xa, unsigned xb, float, float iscale)
    {
        const __half a = *reinterpret_cast<const __half *>(row + 2u * xa);
        const __half b = *reinterpret_cast<const __half *>(row + 2u * xb);
        return F2(__half2float(a), __half2float(b)) * F2(iscale);
    }
    static __device__ __forceinline__ F2 ld2a(const char *row, unsigned x, float, float iscale)
    {
        return F2(__half22float2(*reinterpret_cast<const __half2 *>(row + 2u * x))) * F2(iscale);
    }
};
template <> struct BulkIO<LB_BF16_SHIFTED> {
    using S = __nv_bfloat16;
    static __device__ __forceinline__ F2 ld2(const char *row, unsigned xa, unsigned xb, float, float)
    {
        const unsigned a = *reinterpret_cast<const unsigned short *>(row + 2u * xa);
        const unsigned b = *reinterpret_cast<const unsigned short *>(row + 2u * xb);
        return F2(__uint_as_float(a << 16), __uint_as_float(b << 16));
    }
    static __device__ __forceinline__ F2 ld2a(const char *row, unsigned x, float, float)
    {
        const unsigned r = *reinterpret_cast<const unsigned *>(row + 2u * x);
        return F2(__uint_as_float(r << 16), __uint_as_float(r & 0xffff0000u));
    }
};

// Bytes of one staged row slot (rows of up to NXMAX elements) and of one stage.
template <int ST, int NXMAX>
struct BulkGeom {
    static constexpr unsigned elem = sizeof(typename Codec<ST>::S);
    static constexpr unsigned row = NXMAX * elem;
    static constexpr unsigned stage = Q * row;
};

// Issue the 27 row copies of lattice row r into one stage (called by one thread).
template <int ST, int NXMAX>
__device__ __forceinline__ void bulk_issue_row(const DirPtrs<typename Codec<ST>::S> &ptr, const Geom &g, long long r,
                                               char *stage, uint64_t *full, unsigned rowbytes)
{
    using G = BulkGeom<ST, NXMAX>;
    const unsigned nx = (unsigned)g.nx;
    const int j = (int)(r % g.ny), k = (int)(r / g.ny);
    int ys[3], zs[3];
    bool yo[3], zo[3];
    axis_sources(j, g.ny, g.wall[1], ys, yo);
    axis_sources(k, g.nz, g.wall[2], zs, zo);
    mbar_arrive_expect_tx(full, Q * rowbytes);
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int cy = ey(a) + 1, cz = ez(a) + 1;
        const typename Codec<ST>::S *src;
        if (yo[cy] | zo[cz])   // half-way bounce-back: row (j, k) of the opposite direction
            src = ptr.src[opp(a)] + ((long long)k * g.ny + j) * nx;
        else
            src = ptr.src[a] + ((long long)zs[cz] * g.ny + ys[cy]) * nx;
        bulk_g2s(stage + a * G::row, src, rowbytes, full);
    }
}

// Shared memory: NS stages of 27 rows, NS mbarriers (data arrived) and NS
// counters of the warps that have finished with a stage.  All kBulkThreads threads
// collide; the last warp to finish with a stage refills it with the row NS ahead,
// so no warp ever waits for another one.
template <int ST, int CORR, int NXMAX, int NS, int MINB>
__global__ void __launch_bounds__(kBulkThreads, MINB)
k_step_bulk(DirPtrs<typename Codec<ST>::S> ptr, Geom g, Phys<float> P, DirConst<float> D, float F0, float F1,
            float F2s, const float *__restrict__ ff, int *__restrict__ err, unsigned sr_key)
{
    using G = BulkGeom<ST, NXMAX>;
    using IO = PairIO<ST>;
    using BI = BulkIO<ST>;
    constexpr int kWarps = kBulkThreads / 32;
    extern __shared__ __align__(128) char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + NS * G::stage);
    unsigned *done = reinterpret_cast<unsigned *>(full + NS);
    const unsigned tid = threadIdx.x, lane = tid & 31;
    const unsigned nx = (unsigned)g.nx;
    const long long nrows = (long long)g.ny * g.nz;
    const unsigned rowbytes = nx * G::elem;
    // rows of this CTA: r(n) = blockIdx.x + n gridDim.x, n = 0 .. nmine - 1
    const long long nmine = (nrows - blockIdx.x + gridDim.x - 1) / gridDim.x;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            done[s] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (long long m = 0; m < NS && m < nmine; ++m)
            bulk_issue_row<ST, NXMAX>(ptr, g, blockIdx.x + m * gridDim.x, smem + m * G::stage, &full[m], rowbytes);
    }
    __syncthreads();
    for (long long n = 0; n < nmine; ++n) {
        const int s = (int)(n % NS);
        if (!mbar_wait_bounded(&full[s], (unsigned)((n / NS) & 1))) {
            atomicExch(err, kErrFullWait);
            return;   // every issued copy completes this barrier before any later one can be issued
        }
        const long long r = blockIdx.x + n * gridDim.x;
        const char *stage = smem + s * G::stage;
        const unsigned rowoff = (unsigned)r * nx;
        // rows that came across a y or z wall hold the opposite direction at the node itself
        int ys[3], zs[3];
        bool yo[3], zo[3];
        axis_sources((int)(r % g.ny), g.ny, g.wall[1], ys, yo);
        axis_sources((int)(r / g.ny), g.nz, g.wall[2], zs, zo);
        for (unsigned i0 = 2 * tid; i0 < nx; i0 += 2 * kBulkThreads) {
            const unsigned xm = (i0 == 0) ? nx - 1u : i0 - 1u;       // source of ex = +1 for node i0
            const unsigned xp = (i0 + 2 == nx) ? 0u : i0 + 2u;       // source of ex = -1 for node i0+1
            F2 h[Q];
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                const char *row = stage + a * G::row;
                if (ex(a) == 0 || (yo[ey(a) + 1] | zo[ez(a) + 1]))
                    h[a] = BI::ld2a(row, i0, D.w[a], D.iscale[a]);
                else if (ex(a) == 1)
                    h[a] = BI::ld2(row, xm, i0, D.w[a], D.iscale[a]);
                else
                    h[a] = BI::ld2(row, i0 + 1, xp, D.w[a], D.iscale[a]);
            }
            const unsigned self = rowoff + i0;
            F2 Fx(F0), Fy(F1), Fz(F2s);
            if (ff) {
                const unsigned N = (unsigned)g.N;
                Fx += F2(__ldg(reinterpret_cast<const float2 *>(ff + self)));
                Fy += F2(__ldg(reinterpret_cast<const float2 *>(ff + N + self)));
                Fz += F2(__ldg(reinterpret_cast<const float2 *>(ff + 2u * N + self)));
            }
            unsigned rs = hash32(self * 0x9e3779b1u + sr_key) | 1u;
            collide_pair<CORR>(h,
                               [&](int a, F2 v) {
                                   if (sr_key)
                                       IO::st2sr(ptr.dst[a] + self, v, D.w[a], D.scale[a], xorshift32(rs));
                                   else
                                       IO::st2(ptr.dst[a] + self, v, D.w[a], D.scale[a]);
                               },
                               P, Fx, Fy, Fz);
        }
        __syncwarp();
        // done[s] only grows (kWarps divides 2^32): the warp that completes a multiple
        // of kWarps is the last one off this stage and refills it with row n + NS
        if (lane == 0 && (atomicAdd(&done[s], 1u) + 1u) % kWarps == 0) {
            const long long m = n + NS;
            if (m < nmine) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                bulk_issue_row<ST, NXMAX>(ptr, g, blockIdx.x + m * gridDim.x, smem + s * G::stage, &full[s], rowbytes);
            }
        }
    }
}

}  // namespace lbc
