// reduce_static.cu -- lb_reduce_populations_noalloc: the FP64 mass/momentum
// reduction for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: allocator-restricted embedding hosts
// (a framework that owns every byte of device memory through its own pool), or a
// real-time loop that must never hit the driver allocator.  This entry point
// takes the populations and returns the sums without allocating anything: the
// per-block partial sums and the status word live in a file-scope __device__
// array that every GPU which loads the library keeps until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "lbcuboid.h"

namespace lbc {
void set_last_error(const std::string &msg);   // lbcuboid.cu: message returned by lb_last_error()
}

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 4096;
// each thread folds at most this many nodes, so n <= kMaxBlocks * kThreads * kNodesPerThread
constexpr long long kNodesPerThread = 128;
constexpr long long kMaxNodes = (long long)kMaxBlocks * kThreads * kNodesPerThread;   // 134,217,728

// Scratch: 4 partial sums per block, then the 4 final sums, then the status word.
constexpr int kScratchDoubles = 4 * kMaxBlocks + 4 + 1;
static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch_ptr[kMaxDevices] = {};

// Velocity components of the cuboid D3Q27 directions in the paper's order (Eq. 1a-1c).
__constant__ signed char c_e[3][27] = {
    {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1},
    {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1, 1, 1, -1, -1},
    {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1}};

// Pass 1: block sums of rho = sum f and rho u = sum f e + F/2 (Eq. 12) over nodes in
// a fixed grid-stride order; a non-finite or non-positive node sets the status word.
template <class T>
__global__ void __launch_bounds__(kThreads)
k_reduce_pop(const T *__restrict__ f, long long n, double r, double s, double F0, double F1, double F2,
             double *__restrict__ scratch)
{
    __shared__ double sh[4][kThreads];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    bool bad = false;
    for (long long x = (long long)blockIdx.x * kThreads + threadIdx.x; x < n; x += (long long)gridDim.x * kThreads) {
        double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
        for (int a = 0; a < 27; ++a) {
            const double v = (double)f[a * n + x];
            rho += v;
            jx += v * c_e[0][a];
            jy += v * c_e[1][a];
            jz += v * c_e[2][a];
        }
        jx += 0.5 * F0;
        jy = r * jy + 0.5 * F1;
        jz = s * jz + 0.5 * F2;
        if (!(rho > 0.0) || !isfinite(rho) || !isfinite(jx) || !isfinite(jy) || !isfinite(jz)) bad = true;
        acc[0] += rho;
        acc[1] += jx;
        acc[2] += jy;
        acc[3] += jz;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int k = kThreads / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k)
#pragma unroll
            for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < 4; ++c) scratch[4 * blockIdx.x + c] = sh[c][0];
    if (bad) atomicOr(reinterpret_cast<unsigned long long *>(scratch + 4 * kMaxBlocks + 4), 1ull);
}

// Pass 2: one block adds the partial sums in a fixed order into scratch[4 kMaxBlocks ..].
__global__ void __launch_bounds__(kThreads) k_reduce_pop_final(double *__restrict__ scratch, int nblocks)
{
    __shared__ double sh[4][kThreads];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += kThreads)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] += scratch[4 * b + c];
#pragma unroll
    for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int k = kThreads / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k)
#pragma unroll
            for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < 4; ++c) scratch[4 * kMaxBlocks + c] = sh[c][0];
}

lb_status fail(lb_status st, const std::string &msg)
{
    lbc::set_last_error(msg);
    return st;
}

// Device address of the scratch array on the current device, looked up once per
// device (the array's name is only a host-side stand-in in host code).  The cached
// address belongs to the device's primary context: after cudaDeviceReset on that
// device it is stale, so the entry point must not be called again in that process.
lb_status scratch_for_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LB_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(LB_EINVAL, "device index beyond the supported range");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return fail(LB_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return LB_OK;
}

}  // namespace

extern "C" lb_status lb_reduce_populations_noalloc(const void *f, int real_size, long long n, double r_y,
                                                   double r_z, const double force[3], double out[4], void *stream)
{
    if (!f || !out || n < 1 || (real_size != 4 && real_size != 8) || !(r_y > 0.0) || !(r_z > 0.0))
        return fail(LB_EINVAL, "lb_reduce_populations_noalloc: bad argument");
    if (n > kMaxNodes)
        return fail(LB_EINVAL, "lb_reduce_populations_noalloc: n = " + std::to_string(n) +
                                   " exceeds the maximum of " + std::to_string(kMaxNodes) +
                                   " nodes served by the fixed scratch array");
    // f must be memory the current device can read: a host or numpy pointer (or
    // another device's memory) would make the kernel fault, so reject it here,
    // before anything is launched (cudaPointerGetAttributes allocates nothing)
    int cur = 0;
    cudaError_t ae = cudaGetDevice(&cur);
    if (ae != cudaSuccess) return fail(LB_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ae));
    cudaPointerAttributes attr;
    ae = cudaPointerGetAttributes(&attr, f);
    if (ae != cudaSuccess) {
        cudaGetLastError();
        return fail(LB_EINVAL, "lb_reduce_populations_noalloc: f is not a CUDA pointer");
    }
    if (attr.type != cudaMemoryTypeManaged && !(attr.type == cudaMemoryTypeDevice && attr.device == cur))
        return fail(LB_EINVAL, "lb_reduce_populations_noalloc: f must be device memory of the current device "
                               "or managed memory (host memory is not accepted)");
    double *scratch = nullptr;
    lb_status st = scratch_for_current_device(&scratch);
    if (st) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double F0 = force ? force[0] : 0.0, F1 = force ? force[1] : 0.0, F2 = force ? force[2] : 0.0;
    long long blocks = (n + (long long)kThreads * kNodesPerThread - 1) / ((long long)kThreads * kNodesPerThread);
    if (blocks < 1) blocks = 1;
    // the status word must start at zero; the partial sums are overwritten by pass 1
    cudaError_t e = cudaMemsetAsync(scratch + 4 * kMaxBlocks + 4, 0, sizeof(double), s);
    if (e == cudaSuccess) {
        if (real_size == 8)
            k_reduce_pop<double><<<(int)blocks, kThreads, 0, s>>>(static_cast<const double *>(f), n, r_y, r_z, F0, F1,
                                                                  F2, scratch);
        else
            k_reduce_pop<float><<<(int)blocks, kThreads, 0, s>>>(static_cast<const float *>(f), n, r_y, r_z, F0, F1,
                                                                 F2, scratch);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_reduce_pop_final<<<1, kThreads, 0, s>>>(scratch, (int)blocks);
        e = cudaGetLastError();
    }
    double res[5];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(res, scratch + 4 * kMaxBlocks, 5 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(LB_ECUDA, std::string("lb_reduce_populations_noalloc: ") + cudaGetErrorString(e));
    for (int c = 0; c < 4; ++c) out[c] = res[c];
    unsigned long long status;
    static_assert(sizeof(status) == sizeof(double), "status word size");
    __builtin_memcpy(&status, &res[4], sizeof(status));
    if (status) return fail(LB_EUNSTABLE, "lb_reduce_populations_noalloc: non-finite or non-positive density");
    return LB_OK;
}
