// lbcuboid.cu -- C ABI of liblbcuboid (declared in include/lbcuboid.h): context
// management, argument checking, host/device staging and dispatch to the
// per-storage launchers of ops.cuh.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <string>
#include <vector>

#include "lbcuboid.h"
#include "ops.cuh"

// The launchers (and with them every kernel) are instantiated once per storage
// form in step_*.cu, which compile in parallel; this file only calls them.
extern template struct lbc::Ops<LB_F64>;
extern template struct lbc::Ops<LB_F32>;
extern template struct lbc::Ops<LB_F32_SHIFTED>;
extern template struct lbc::Ops<LB_F16_SHIFTED>;
extern template struct lbc::Ops<LB_BF16_SHIFTED>;

using namespace lbc;

namespace {

thread_local std::string g_last_error;

lb_status fail(lb_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

lb_status cuda_fail(cudaError_t e, const char *where)
{
    return fail(e == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

#define LB_CUDA(call)                                         \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

size_t storage_bytes(int st)
{
    switch (st) {
    case LB_F64: return 8;
    case LB_F32:
    case LB_F32_SHIFTED: return 4;
    default: return 2;
    }
}

constexpr int kMaxSub = 16;   // most z-slabs of a decomposed lattice

}  // namespace

struct lb_ctx {
    lb_config cfg;
    Geom g;
    double cs2, wn, wb;
    double w[Q];
    float scale[Q];
    cudaStream_t stream;
    void *buf[2];
    int cur;
    size_t sbytes;          // bytes of one stored value
    size_t rbytes;          // bytes of one real
    void *force_field;      // [3][N] real or null
    void *rho_field;        // [N] real (FULL)
    void *stage;            // staging for host pointers
    size_t stage_bytes;
    double *partial;
    double *out4;
    unsigned *status;
    int nred;
    long long t;
    // True while the stored state holds pre-collision populations written by
    // lb_init / lb_set_populations (the moving-lid term belongs to streaming after
    // a collision, so it is not applied when those populations are read).
    bool fresh;
    // Lid velocity of the step whose collision wrote the stored state: the next read
    // streams that state, and the moving-wall term of that streaming belongs to the
    // same step (so a lid changed between lb_step calls acts from the next step on).
    double lid_state;
    // Work buffers of lb_adjoint_ke (checkpoints, segment, adjoint fields, block sums),
    // kept for the next call and grown when a call needs more; freed by lb_destroy
    void *adj_buf[7];
    size_t adj_bytes[7];
    int *err;               // error word of the bounded waits of the staged kernel
    int sm_count;
    // CUDA graphs of kGraphSteps consecutive steps starting from buffer 0 / 1, with
    // the launch arguments they were captured with; graph_off after a failed capture
    cudaGraphExec_t graph[2];
    LaunchArgs graph_key[2];
    bool graph_off;
    // z-slab decomposition (cfg.subdomains > 1): slab p owns the global planes
    // sub_z0[p] .. sub_z0[p + 1] - 1, stored at its local planes 1 .. n_p between the
    // ghost planes 0 and n_p + 1; two buffers per slab with the parity of buf
    int nsub;
    int sub_z0[kMaxSub + 1];
    void *sub_buf[2][kMaxSub];
    int sub_kernel;               // step kernel of the whole lattice (1 or 2), used by every slab
    cudaStream_t side;            // boundary planes and halo exchange, beside the interiors
    cudaEvent_t ev_fork, ev_join;
};

namespace {

// Key of the stochastic-rounding draws of one time step (0 = round to nearest):
// the lowbias32 hash (C. Wellons) of the seed mixed with the step index.
unsigned step_key(const lb_ctx *c);

LaunchArgs launch_args(const lb_ctx *c)
{
    LaunchArgs a;
    std::memset(&a, 0, sizeof(a));   // padding included: graphs are keyed by the bytes of a
    a.g = c->g;
    a.r = c->cfg.r_y;
    a.s = c->cfg.r_z;
    a.cs2 = c->cs2;
    a.wn = c->wn;
    a.wb = c->wb;
    for (int i = 0; i < 3; ++i) a.F[i] = c->cfg.force[i];
    a.lid_u = c->fresh ? 0.0 : c->lid_state;
    for (int q = 0; q < Q; ++q) {
        a.w[q] = c->w[q];
        a.scale[q] = c->scale[q];
    }
    a.corr = c->cfg.corr;
    a.model = c->cfg.model;
    a.stream = c->stream;
    a.force_field = c->force_field;
    a.rho_field = c->rho_field;
    a.kernel = c->cfg.kernel;
    a.err = c->err;
    a.sm_count = c->sm_count;
    a.sr_key = step_key(c);
    return a;
}

unsigned step_key(const lb_ctx *c)
{
    if (c->cfg.rounding != 1) return 0u;
    unsigned x = c->cfg.rounding_seed ^ (unsigned)(c->t * 0x9e3779b97f4a7c15ull) ^ (unsigned)((c->t >> 32) * 0x85ebca6bu);
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x | 1u;
}

// Self-test of the bounded mbarrier wait of the row-staged kernel: one thread
// initialises an mbarrier for one arrival and waits for its first phase with a
// short limit while nothing arrives (the wait must give up and say so), then
// arrives itself and waits again (the wait must succeed).
constexpr unsigned kProbeLimit = 1u << 12;

__global__ void k_wait_probe(int *out)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    out[0] = mbar_wait_bounded(&bar, 0u, kProbeLimit) ? 0 : 1;    // nobody arrives: must time out
    mbar_arrive(&bar);
    out[1] = mbar_wait_bounded(&bar, 0u, kProbeLimit) ? 1 : 0;    // phase 0 completed
}

template <class F>
cudaError_t dispatch(int st, F &&f)
{
    switch (st) {
    case LB_F64: return f(Ops<LB_F64>());
    case LB_F32: return f(Ops<LB_F32>());
    case LB_F32_SHIFTED: return f(Ops<LB_F32_SHIFTED>());
    case LB_F16_SHIFTED: return f(Ops<LB_F16_SHIFTED>());
    default: return f(Ops<LB_BF16_SHIFTED>());
    }
}

// ---------------------------------------------------------------------------
// z-slab decomposition.  Copies move whole planes as words of W bytes (the largest
// of 16, 8, 4, 2 that divides a plane's bytes; plane starts are then aligned).

// Between the whole lattice and slab `slab` for every direction (grid z): to the
// slab, local planes 0 .. n_p + 1 from global planes z0 - 1 .. z0 + n_p (periodic in
// z); from the slab, its owned planes 1 .. n_p.
template <class W>
__global__ void k_slab_copy(W *whole, W *slab, long long nw_whole, long long nw_slab, long long plane_w, int z0,
                            int nz, int to_slab)
{
    const int a = blockIdx.z;
    const int lp = (int)blockIdx.y + (to_slab ? 0 : 1);
    int gz = z0 + lp - 1;
    if (gz < 0) gz += nz;
    if (gz >= nz) gz -= nz;
    W *pw = whole + a * nw_whole + gz * plane_w;
    W *ps = slab + a * nw_slab + lp * plane_w;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < plane_w;
         i += (long long)gridDim.x * blockDim.x) {
        if (to_slab)
            ps[i] = pw[i];
        else
            pw[i] = ps[i];
    }
}

// Halo exchange after a step, on the buffers just written.  Block z = 18 p + d:
// d < 9, the d-th direction with e_z = +1: the last owned plane of slab p goes to the
// lower ghost plane of slab p + 1; d >= 9, a direction with e_z = -1: the first owned
// plane of slab p goes to the upper ghost plane of slab p - 1 (periodic in p).
struct SlabSet {
    void *base[kMaxSub];
    long long nw[kMaxSub];        // words of one direction array of each slab
    int np[kMaxSub];              // owned planes of each slab
    int dir[18];
    int P;
    long long plane_w;            // words of one plane
};

template <class W>
__global__ void k_halo(SlabSet s)
{
    const int p = (int)blockIdx.z / 18, d = (int)blockIdx.z % 18;
    const int a = s.dir[d];
    int q, sp, dp;
    if (d < 9) {
        q = (p + 1) % s.P;
        sp = s.np[p];
        dp = 0;
    } else {
        q = (p + s.P - 1) % s.P;
        sp = 1;
        dp = s.np[q] + 1;
    }
    const W *src = static_cast<const W *>(s.base[p]) + a * s.nw[p] + sp * s.plane_w;
    W *dst = static_cast<W *>(s.base[q]) + a * s.nw[q] + dp * s.plane_w;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < s.plane_w;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// Word size for moving planes of `plane_bytes` bytes.
int plane_word(size_t plane_bytes)
{
    for (int w : {16, 8, 4})
        if (plane_bytes % w == 0) return w;
    return 2;
}

template <class F>
cudaError_t with_word(int w, F &&f)
{
    switch (w) {
    case 16: return f(uint4());
    case 8: return f(uint2());
    case 4: return f(0u);
    default: return f((unsigned short)0);
    }
}

// Launch arguments of slab p: its local geometry (owned planes between two ghost
// planes, z periodic across the ghosts), and the planes to update: the first and the
// last owned plane (boundary) or those between them (interior).
LaunchArgs slab_args(const lb_ctx *c, const LaunchArgs &a, int p, bool boundary)
{
    LaunchArgs b = a;
    const int np = c->sub_z0[p + 1] - c->sub_z0[p];
    b.g.nz = np + 2;
    b.g.N = (long long)c->g.nx * c->g.ny * (np + 2);
    b.g.zofs = c->sub_z0[p] - 1;
    if (boundary) {
        b.g.kz0 = 1;
        b.g.kz1 = np + 1;
        b.g.kzs = np > 1 ? np - 1 : 1;
    } else {
        b.g.kz0 = 2;
        b.g.kz1 = np;
        b.g.kzs = 1;
    }
    b.kernel = c->sub_kernel;
    return b;
}

// Whole lattice <-> slabs (parity p) on the main stream.
cudaError_t slab_transfer(lb_ctx *c, int p, bool to_slab)
{
    const long long plane = (long long)c->g.nx * c->g.ny;
    const size_t plane_bytes = (size_t)plane * c->sbytes;
    return with_word(plane_word(plane_bytes), [&](auto word) {
        using W = decltype(word);
        const long long plane_w = (long long)(plane_bytes / sizeof(W));
        for (int s = 0; s < c->nsub; ++s) {
            const int np = c->sub_z0[s + 1] - c->sub_z0[s];
            const dim3 grid((unsigned)std::min<long long>((plane_w + 255) / 256, 64), to_slab ? np + 2 : np, Q);
            k_slab_copy<W><<<grid, 256, 0, c->stream>>>(static_cast<W *>(c->buf[p]), static_cast<W *>(c->sub_buf[p][s]),
                                                        plane_w * c->g.nz, plane_w * (np + 2), plane_w, c->sub_z0[s],
                                                        c->g.nz, to_slab ? 1 : 0);
        }
        return cudaGetLastError();
    });
}

// One time step of the decomposed lattice from slab parity p to p ^ 1: the side stream
// updates every slab's boundary planes and then exchanges the halos while the main
// stream updates the interiors; the main stream then waits for the side stream.
cudaError_t slab_step(lb_ctx *c, const LaunchArgs &a, int p)
{
    cudaError_t e = cudaEventRecord(c->ev_fork, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->ev_fork, 0);
    for (int s = 0; s < c->nsub && e == cudaSuccess; ++s) {
        LaunchArgs b = slab_args(c, a, s, true);
        b.stream = c->side;
        const void *src = c->sub_buf[p][s];
        void *dst = c->sub_buf[p ^ 1][s];
        e = dispatch(c->cfg.storage, [&](auto ops) { return decltype(ops)::step(b, src, dst); });
    }
    if (e == cudaSuccess) {
        SlabSet set;
        std::memset(&set, 0, sizeof(set));
        const size_t plane_bytes = (size_t)c->g.nx * c->g.ny * c->sbytes;
        const int word = plane_word(plane_bytes);
        set.P = c->nsub;
        set.plane_w = (long long)(plane_bytes / word);
        int nu = 0, nd = 9;
        for (int q = 0; q < Q; ++q) {
            if (ez(q) == 1) set.dir[nu++] = q;
            if (ez(q) == -1) set.dir[nd++] = q;
        }
        for (int s = 0; s < c->nsub; ++s) {
            set.np[s] = c->sub_z0[s + 1] - c->sub_z0[s];
            set.base[s] = c->sub_buf[p ^ 1][s];
            set.nw[s] = set.plane_w * (set.np[s] + 2);
        }
        e = with_word(word, [&](auto w) {
            using W = decltype(w);
            const dim3 grid((unsigned)std::min<long long>((set.plane_w + 255) / 256, 32), 1, 18 * c->nsub);
            k_halo<W><<<grid, 256, 0, c->side>>>(set);
            return cudaGetLastError();
        });
    }
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, c->side);
    for (int s = 0; s < c->nsub && e == cudaSuccess; ++s) {
        if (c->sub_z0[s + 1] - c->sub_z0[s] < 3) continue;
        const LaunchArgs b = slab_args(c, a, s, false);
        const void *src = c->sub_buf[p][s];
        void *dst = c->sub_buf[p ^ 1][s];
        e = dispatch(c->cfg.storage, [&](auto ops) { return decltype(ops)::step(b, src, dst); });
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_join, 0);
    return e;
}

// One time step from buffer parity p (whole lattice or slabs).
cudaError_t one_step(lb_ctx *c, const LaunchArgs &a, int p)
{
    if (c->nsub > 1) return slab_step(c, a, p);
    const void *src = c->buf[p];
    void *dst = c->buf[p ^ 1];
    return dispatch(c->cfg.storage, [&](auto ops) { return decltype(ops)::step(a, src, dst); });
}

// Slab buffers, the side stream and its events, made on the first decomposed step.
lb_status ensure_slabs(lb_ctx *c)
{
    if (c->side) return LB_OK;
    for (int s = 0; s < c->nsub; ++s) {
        const size_t bytes = (size_t)Q * c->g.nx * c->g.ny * (c->sub_z0[s + 1] - c->sub_z0[s] + 2) * c->sbytes;
        for (int p = 0; p < 2; ++p) {
            LB_CUDA(cudaMalloc(&c->sub_buf[p][s], bytes));
            LB_CUDA(cudaMemsetAsync(c->sub_buf[p][s], 0, bytes, c->stream));
        }
    }
    LB_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    LB_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    LB_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    return LB_OK;
}

// Steps per CUDA graph.  On small lattices one step takes less time than a kernel
// launch, so lb_step replays a captured run of kGraphSteps launches (an even number:
// the ping-pong buffers end where they started) while the launch arguments stay the
// same.  Graphs are used on a non-default stream with round-to-nearest storage (the
// stochastic-rounding key changes every step) once a step has run with the same
// arguments outside the capture.
constexpr int kGraphSteps = 64;

void drop_graph(lb_ctx *c, int p)
{
    if (c->graph[p]) cudaGraphExecDestroy(c->graph[p]);
    c->graph[p] = nullptr;
}

// The graph for the current buffer and arguments, captured on first use; null when
// capture is not possible (graphs are then off for this context).
cudaGraphExec_t graph_for(lb_ctx *c, const LaunchArgs &a)
{
    const int p = c->cur;
    if (c->graph[p] && std::memcmp(&c->graph_key[p], &a, sizeof(a)) == 0) return c->graph[p];
    drop_graph(c, p);
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        c->graph_off = true;
        return nullptr;
    }
    cudaError_t e = cudaSuccess;
    int cur = p;
    for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k) {
        e = one_step(c, a, cur);
        cur ^= 1;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    cudaGraphExec_t x = nullptr;
    if (e == cudaSuccess && e2 == cudaSuccess && g) e = cudaGraphInstantiate(&x, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess || e2 != cudaSuccess || !x) {
        cudaGetLastError();
        c->graph_off = true;
        return nullptr;
    }
    c->graph[p] = x;
    c->graph_key[p] = a;
    return x;
}


bool is_device_pointer(const void *p)
{
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

lb_status ensure_stage(lb_ctx *c, size_t bytes)
{
    if (c->stage_bytes >= bytes) return LB_OK;
    if (c->stage) LB_CUDA(cudaFree(c->stage));
    c->stage = nullptr;
    c->stage_bytes = 0;
    LB_CUDA(cudaMalloc(&c->stage, bytes));
    c->stage_bytes = bytes;
    return LB_OK;
}

// Device view of a caller input of `bytes` bytes placed at `offset` in the stage.
lb_status device_input(lb_ctx *c, const void *p, size_t bytes, size_t offset, const void **dev)
{
    if (is_device_pointer(p)) {
        *dev = p;
        return LB_OK;
    }
    char *s = static_cast<char *>(c->stage) + offset;
    LB_CUDA(cudaMemcpyAsync(s, p, bytes, cudaMemcpyHostToDevice, c->stream));
    *dev = s;
    return LB_OK;
}

// 1-D rest weight of velocity index v (-1, 0, 1) on an axis with speed c.
double w1(int v, double c, double cs2) { return v == 0 ? 1.0 - cs2 / (c * c) : 0.5 * cs2 / (c * c); }

}  // namespace

extern "C" {

void lb_config_default(lb_config *cfg, int nx, int ny, int nz, double r_y, double r_z, double nu)
{
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->nx = nx;
    cfg->ny = ny;
    cfg->nz = nz;
    cfg->r_y = r_y;
    cfg->r_z = r_z;
    cfg->nu = nu;
    cfg->zeta = 0.0;
    cfg->cs2 = 0.0;
    cfg->storage = LB_F32;
    cfg->corr = LB_CORR_LOCAL;
}

lb_status lb_create(int nx, int ny, int nz, double r_y, double r_z, double nu, double zeta, lb_ctx **out)
{
    lb_config cfg;
    lb_config_default(&cfg, nx, ny, nz, r_y, r_z, nu);
    cfg.zeta = zeta;
    return lb_create_ex(&cfg, out);
}

lb_status lb_create_ex(const lb_config *cfg, lb_ctx **out)
{
    if (!cfg || !out) return fail(LB_EINVAL, "lb_create_ex: null argument");
    *out = nullptr;
    if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1) return fail(LB_EINVAL, "lb_create_ex: dimensions must be >= 1");
    if (cfg->nz > 65535 || (cfg->ny + 127) / 128 > 65535)
        return fail(LB_EINVAL, "lb_create_ex: ny or nz exceeds the launch-grid limit (nz <= 65535)");
    if (!(cfg->r_y > 0.0) || !(cfg->r_z > 0.0) || !std::isfinite(cfg->r_y) || !std::isfinite(cfg->r_z))
        return fail(LB_EINVAL, "lb_create_ex: aspect ratios must be positive and finite");
    if (cfg->storage < LB_F64 || cfg->storage > LB_BF16_SHIFTED) return fail(LB_EINVAL, "lb_create_ex: bad storage");
    if (cfg->corr < LB_CORR_NONE || cfg->corr > LB_CORR_FULL) return fail(LB_EINVAL, "lb_create_ex: bad corr");
    if (cfg->wall_mask & ~7u) return fail(LB_EINVAL, "lb_create_ex: bad wall_mask");
    if (cfg->kernel < 0 || cfg->kernel > 5) return fail(LB_EINVAL, "lb_create_ex: bad kernel selector");
    if (cfg->rounding < 0 || cfg->rounding > 1) return fail(LB_EINVAL, "lb_create_ex: bad rounding mode");
    if (cfg->rounding == 1 && cfg->storage != LB_F16_SHIFTED && cfg->storage != LB_BF16_SHIFTED)
        return fail(LB_EINVAL, "lb_create_ex: stochastic rounding applies to FP16/BF16 storage only");
    if (cfg->model < 0 || cfg->model > 1) return fail(LB_EINVAL, "lb_create_ex: bad collision model");
    if (cfg->model == 1 && cfg->corr != LB_CORR_LOCAL)
        return fail(LB_EINVAL, "lb_create_ex: the raw-moment model runs with LB_CORR_LOCAL only");
    if (cfg->lid_u != 0.0 && !(cfg->wall_mask & LB_WALL_Y))
        return fail(LB_EINVAL, "lb_create_ex: a moving lid needs walls normal to y");
    const double r = cfg->r_y, s = cfg->r_z;
    const double cmin = std::fmin(1.0, std::fmin(r * r, s * s));
    const double cs2 = cfg->cs2 > 0.0 ? cfg->cs2 : cmin / 3.0;
    if (!(cs2 > 0.0) || !(cs2 < cmin))
        return fail(LB_EINVAL, "lb_create_ex: cs2 must satisfy 0 < cs2 < min(1, r^2, s^2) (positive rest weights)");
    if (!(cfg->nu > 0.0) || !std::isfinite(cfg->nu)) return fail(LB_EINVAL, "lb_create_ex: nu must be > 0");
    const double wn = 1.0 / (cfg->nu / cs2 + 0.5);
    const double wb = cfg->zeta > 0.0 ? 1.0 / (1.5 * cfg->zeta / cs2 + 0.5) : 1.0;
    if (!(wn > 0.0 && wn < 2.0) || !(wb > 0.0 && wb < 2.0))
        return fail(LB_EINVAL, "lb_create_ex: relaxation rates must lie in (0, 2)");
    const long long N = (long long)cfg->nx * cfg->ny * cfg->nz;
    const int nsub = cfg->subdomains > 1 ? cfg->subdomains : 1;
    if (nsub > 1) {
        if (nsub > kMaxSub || nsub > cfg->nz)
            return fail(LB_EINVAL, "lb_create_ex: subdomains must lie in 1..16 and not exceed nz");
        if ((cfg->wall_mask & LB_WALL_Z) || cfg->corr == LB_CORR_FULL || cfg->kernel == 3)
            return fail(LB_EINVAL, "lb_create_ex: subdomains need z periodic, corrections other than FULL and "
                                   "a kernel other than the row-staged one");
    }

    lb_ctx *c = new lb_ctx();
    std::memset(static_cast<void *>(c), 0, sizeof(*c));
    c->cfg = *cfg;
    c->lid_state = cfg->lid_u;
    c->cfg.cs2 = cs2;
    c->cs2 = cs2;
    c->wn = wn;
    c->wb = wb;
    c->g.nx = cfg->nx;
    c->g.ny = cfg->ny;
    c->g.nz = cfg->nz;
    for (int i = 0; i < 3; ++i) c->g.wall[i] = (cfg->wall_mask >> i) & 1u;
    c->g.N = N;
    c->g.kz0 = 0;
    c->g.kz1 = cfg->nz;
    c->g.kzs = 1;
    c->g.zofs = 0;
    c->nsub = nsub;
    for (int s = 0; s <= nsub; ++s) c->sub_z0[s] = (int)((long long)cfg->nz * s / nsub);
    c->stream = static_cast<cudaStream_t>(cfg->stream);
    c->sbytes = storage_bytes(cfg->storage);
    c->rbytes = cfg->storage == LB_F64 ? 8 : 4;
    const double cc[3] = {1.0, r, s};
    for (int a = 0; a < Q; ++a) {
        const double wa = w1(ex(a), cc[0], cs2) * w1(ey(a), cc[1], cs2) * w1(ez(a), cc[2], cs2);
        c->w[a] = wa;
        // FP16: scale direction a by 2^E so that h_a / w_a ~ O(1) lands near 2^10,
        // far from both the subnormal range and the 65504 limit.
        c->scale[a] = cfg->storage == LB_F16_SHIFTED ? std::ldexp(1.0f, 10 - std::ilogb(wa)) : 1.0f;
    }
    const size_t bytes = (size_t)Q * N * c->sbytes;
    cudaError_t e = cudaMalloc(&c->buf[0], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->buf[1], bytes);
    c->nred = 2 * 152;
    if (e == cudaSuccess) e = cudaMalloc(&c->partial, sizeof(double) * 4 * c->nred);
    if (e == cudaSuccess) e = cudaMalloc(&c->out4, sizeof(double) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c->status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&c->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) {
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
    }
    if (e == cudaSuccess && cfg->corr == LB_CORR_FULL) e = cudaMalloc(&c->rho_field, N * c->rbytes);
    if (e == cudaSuccess && nsub > 1) {
        // every slab runs the kernel the whole lattice would (bit-identical results)
        const LaunchArgs a = launch_args(c);
        bool pair = false;
        switch (cfg->storage) {
        case LB_F64: pair = Ops<LB_F64>::use_pair(a); break;
        case LB_F32: pair = Ops<LB_F32>::use_pair(a); break;
        case LB_F32_SHIFTED: pair = Ops<LB_F32_SHIFTED>::use_pair(a); break;
        case LB_F16_SHIFTED: pair = Ops<LB_F16_SHIFTED>::use_pair(a); break;
        default: pair = Ops<LB_BF16_SHIFTED>::use_pair(a); break;
        }
        c->sub_kernel = pair ? 2 : 1;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(c->buf[0], 0, bytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->buf[1], 0, bytes, c->stream);
    if (e != cudaSuccess) {
        lb_destroy(c);
        return cuda_fail(e, "lb_create_ex: allocation");
    }
    *out = c;
    return LB_OK;
}

void lb_destroy(lb_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    cudaFree(c->buf[0]);
    cudaFree(c->buf[1]);
    cudaFree(c->force_field);
    cudaFree(c->rho_field);
    cudaFree(c->stage);
    cudaFree(c->partial);
    cudaFree(c->out4);
    cudaFree(c->status);
    cudaFree(c->err);
    for (int b = 0; b < 7; ++b) cudaFree(c->adj_buf[b]);
    drop_graph(c, 0);
    drop_graph(c, 1);
    for (int s = 0; s < kMaxSub; ++s)
        for (int p = 0; p < 2; ++p) cudaFree(c->sub_buf[p][s]);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    delete c;
}

int lb_real_size(const lb_ctx *c) { return c ? (int)c->rbytes : 0; }

size_t lb_num_nodes(const lb_ctx *c) { return c ? (size_t)c->g.N : 0; }

lb_status lb_get_params(const lb_ctx *c, double out[3])
{
    if (!c || !out) return fail(LB_EINVAL, "lb_get_params: null argument");
    out[0] = c->wn;
    out[1] = c->wb;
    out[2] = c->cs2;
    return LB_OK;
}

long long lb_time_step(const lb_ctx *c) { return c ? c->t : -1; }

lb_status lb_init(lb_ctx *c, const void *rho, const void *u)
{
    if (!c || !rho || !u) return fail(LB_EINVAL, "lb_init: null argument");
    const size_t nb = (size_t)c->g.N * c->rbytes;
    lb_status st = LB_OK;
    if (!is_device_pointer(rho) || !is_device_pointer(u)) st = ensure_stage(c, 4 * nb);
    if (st) return st;
    const void *drho, *du;
    if ((st = device_input(c, rho, nb, 0, &drho))) return st;
    if ((st = device_input(c, u, 3 * nb, nb, &du))) return st;
    const LaunchArgs a = launch_args(c);
    void *dst = c->buf[c->cur];
    LB_CUDA(dispatch(c->cfg.storage, [&](auto ops) { return decltype(ops)::scatter(a, dst, drho, du, nullptr); }));
    c->t = 0;
    c->fresh = true;
    return LB_OK;
}

lb_status lb_set_force_field(lb_ctx *c, const void *force)
{
    if (!c) return fail(LB_EINVAL, "lb_set_force_field: null context");
    if (force && c->nsub > 1) return fail(LB_EINVAL, "lb_set_force_field: not available with subdomains > 1");
    const size_t nb = 3 * (size_t)c->g.N * c->rbytes;
    if (!force) {
        LB_CUDA(cudaStreamSynchronize(c->stream));
        LB_CUDA(cudaFree(c->force_field));
        c->force_field = nullptr;
        return LB_OK;
    }
    if (!c->force_field) LB_CUDA(cudaMalloc(&c->force_field, nb));
    LB_CUDA(cudaMemcpyAsync(c->force_field, force, nb, cudaMemcpyDefault, c->stream));
    return LB_OK;
}

lb_status lb_step(lb_ctx *c, int n)
{
    if (!c) return fail(LB_EINVAL, "lb_step: null context");
    if (n < 0) return fail(LB_EINVAL, "lb_step: n must be >= 0");
    if (n == 0) return LB_OK;
    if (c->nsub > 1) {
        lb_status st = ensure_slabs(c);
        if (st) return st;
        LB_CUDA(slab_transfer(c, c->cur, true));
    }
    bool plain_done = false;   // one step with these arguments ran outside a capture
    for (int i = 0; i < n;) {
        const LaunchArgs a = launch_args(c);
        if (plain_done && n - i >= kGraphSteps && !c->graph_off && c->stream != nullptr && c->cfg.rounding == 0 &&
            c->lid_state == c->cfg.lid_u) {
            cudaGraphExec_t x = graph_for(c, a);
            if (x) {
                LB_CUDA(cudaGraphLaunch(x, c->stream));
                i += kGraphSteps;
                c->t += kGraphSteps;
                continue;
            }
        }
        LB_CUDA(one_step(c, a, c->cur));
        c->cur ^= 1;
        ++c->t;
        plain_done = !c->fresh;
        c->fresh = false;
        c->lid_state = c->cfg.lid_u;
        ++i;
    }
    if (c->nsub > 1) LB_CUDA(slab_transfer(c, c->cur, false));
    return LB_OK;
}

lb_status lb_moments(lb_ctx *c, void *rho, void *u)
{
    if (!c || (!rho && !u)) return fail(LB_EINVAL, "lb_moments: null argument");
    const size_t nb = (size_t)c->g.N * c->rbytes;
    const bool dr = !rho || is_device_pointer(rho), du = !u || is_device_pointer(u);
    if (!dr || !du) {
        lb_status st = ensure_stage(c, 4 * nb);
        if (st) return st;
    }
    char *stage = static_cast<char *>(c->stage);
    void *trho = rho ? (dr ? rho : stage) : nullptr;
    void *tu = u ? (du ? u : stage + nb) : nullptr;
    const LaunchArgs a = launch_args(c);
    const void *src = c->buf[c->cur];
    LB_CUDA(dispatch(c->cfg.storage, [&](auto ops) { return decltype(ops)::gather(a, src, trho, tu, nullptr); }));
    if (rho && !dr) LB_CUDA(cudaMemcpyAsync(rho, trho, nb, cudaMemcpyDeviceToHost, c->stream));
    if (u && !du) LB_CUDA(cudaMemcpyAsync(u, tu, 3 * nb, cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

lb_status lb_reduce(lb_ctx *c, double out[4])
{
    if (!c || !out) return fail(LB_EINVAL, "lb_reduce: null argument");
    const LaunchArgs a = launch_args(c);
    const void *src = c->buf[c->cur];
    LB_CUDA(cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream));
    LB_CUDA(dispatch(c->cfg.storage, [&](auto ops) {
        return decltype(ops)::reduce_partial(a, src, c->partial, c->nred, c->status);
    }));
    k_reduce_final<<<1, kReduceThreads, 0, c->stream>>>(c->partial, c->nred, c->out4);
    LB_CUDA(cudaGetLastError());
    unsigned status = 0;
    LB_CUDA(cudaMemcpyAsync(out, c->out4, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(cudaMemcpyAsync(&status, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    int err = 0;
    LB_CUDA(cudaMemcpyAsync(&err, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(cudaStreamSynchronize(c->stream));
    if (err) return fail(LB_ETIMEOUT, "lb_reduce: a bounded wait of the staged step kernel ran out (code " +
                                          std::to_string(err) + "); the state is not valid");
    if (status) return fail(LB_EUNSTABLE, "lb_reduce: non-finite or non-positive density/velocity found");
    return LB_OK;
}

lb_status lb_get_populations(lb_ctx *c, void *dst)
{
    if (!c || !dst) return fail(LB_EINVAL, "lb_get_populations: null argument");
    const size_t nb = (size_t)Q * c->g.N * c->rbytes;
    const bool dev = is_device_pointer(dst);
    if (!dev) {
        lb_status st = ensure_stage(c, nb);
        if (st) return st;
    }
    void *t = dev ? dst : c->stage;
    const LaunchArgs a = launch_args(c);
    const void *src = c->buf[c->cur];
    LB_CUDA(dispatch(c->cfg.storage, [&](auto ops) { return decltype(ops)::gather(a, src, nullptr, nullptr, t); }));
    if (!dev) LB_CUDA(cudaMemcpyAsync(dst, t, nb, cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

lb_status lb_set_populations(lb_ctx *c, const void *src)
{
    if (!c || !src) return fail(LB_EINVAL, "lb_set_populations: null argument");
    const size_t nb = (size_t)Q * c->g.N * c->rbytes;
    const bool dev = is_device_pointer(src);
    if (!dev) {
        lb_status st = ensure_stage(c, nb);
        if (st) return st;
    }
    const void *dsrc;
    lb_status st = device_input(c, src, nb, 0, &dsrc);
    if (st) return st;
    const LaunchArgs a = launch_args(c);
    void *dst = c->buf[c->cur];
    LB_CUDA(dispatch(c->cfg.storage, [&](auto ops) { return decltype(ops)::scatter(a, dst, nullptr, nullptr, dsrc); }));
    LB_CUDA(cudaStreamSynchronize(c->stream));
    c->t = 0;
    c->fresh = true;
    return LB_OK;
}

size_t lb_state_bytes(const lb_ctx *c) { return c ? (size_t)Q * c->g.N * c->sbytes : 0; }

lb_status lb_get_state(lb_ctx *c, void *dst)
{
    if (!c || !dst) return fail(LB_EINVAL, "lb_get_state: null argument");
    LB_CUDA(cudaMemcpyAsync(dst, c->buf[c->cur], lb_state_bytes(c), cudaMemcpyDefault, c->stream));
    LB_CUDA(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

lb_status lb_set_state(lb_ctx *c, const void *src, long long time_step)
{
    if (!c || !src) return fail(LB_EINVAL, "lb_set_state: null argument");
    LB_CUDA(cudaMemcpyAsync(c->buf[c->cur], src, lb_state_bytes(c), cudaMemcpyDefault, c->stream));
    LB_CUDA(cudaStreamSynchronize(c->stream));
    c->t = time_step;
    c->fresh = false;
    c->lid_state = c->cfg.lid_u;
    return LB_OK;
}

lb_status lb_set_force(lb_ctx *c, const double force[3])
{
    if (!c || !force) return fail(LB_EINVAL, "lb_set_force: null argument");
    for (int i = 0; i < 3; ++i) {
        if (!std::isfinite(force[i])) return fail(LB_EINVAL, "lb_set_force: non-finite force");
        c->cfg.force[i] = force[i];
    }
    return LB_OK;
}

lb_status lb_set_rates(lb_ctx *c, double omega_nu, double omega_xi)
{
    if (!c) return fail(LB_EINVAL, "lb_set_rates: null context");
    if (!(omega_nu > 0.0 && omega_nu < 2.0) || !(omega_xi > 0.0 && omega_xi < 2.0))
        return fail(LB_EINVAL, "lb_set_rates: relaxation rates must lie in (0, 2)");
    c->wn = omega_nu;
    c->wb = omega_xi;
    return LB_OK;
}

lb_status lb_set_lid(lb_ctx *c, double lid_u)
{
    if (!c) return fail(LB_EINVAL, "lb_set_lid: null context");
    if (!std::isfinite(lid_u)) return fail(LB_EINVAL, "lb_set_lid: non-finite velocity");
    if (lid_u != 0.0 && !(c->cfg.wall_mask & LB_WALL_Y))
        return fail(LB_EINVAL, "lb_set_lid: a moving lid needs walls normal to y");
    c->cfg.lid_u = lid_u;
    return LB_OK;
}

namespace {

// Device scratch owned by one adjoint / objective call (freed on every exit path).
struct Scratch {
    std::vector<void *> ptrs;
    ~Scratch()
    {
        for (void *p : ptrs) cudaFree(p);
    }
    cudaError_t alloc(void **p, size_t bytes)
    {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};

// Work buffer `slot` of lb_adjoint_ke with at least `bytes` bytes (reused across calls).
cudaError_t adjoint_buffer(lb_ctx *c, int slot, size_t bytes, void **p)
{
    if (c->adj_bytes[slot] < bytes) {
        cudaError_t e = cudaFree(c->adj_buf[slot]);
        c->adj_buf[slot] = nullptr;
        c->adj_bytes[slot] = 0;
        if (e != cudaSuccess) return e;
        if ((e = cudaMalloc(&c->adj_buf[slot], bytes)) != cudaSuccess) {
            c->adj_buf[slot] = nullptr;
            return e;
        }
        c->adj_bytes[slot] = bytes;
    }
    *p = c->adj_buf[slot];
    return cudaSuccess;
}

lb_status sum_pairs(lb_ctx *c, const double *dev, long long nblocks, double out[2])
{
    std::vector<double> h(2 * (size_t)nblocks);
    LB_CUDA(cudaMemcpyAsync(h.data(), dev, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(cudaStreamSynchronize(c->stream));
    out[0] = out[1] = 0.0;
    for (long long b = 0; b < nblocks; ++b) {
        out[0] += h[2 * b];
        out[1] += h[2 * b + 1];
    }
    return LB_OK;
}

}  // namespace

lb_status lb_objective_ke(lb_ctx *c, double *J)
{
    if (!c || !J) return fail(LB_EINVAL, "lb_objective_ke: null argument");
    Scratch s;
    const long long nb = adjoint_blocks(c->g);
    double *jpart = nullptr;
    LB_CUDA(s.alloc((void **)&jpart, 2 * nb * sizeof(double)));
    LB_CUDA(cudaMemsetAsync(jpart, 0, 2 * nb * sizeof(double), c->stream));
    const LaunchArgs a = launch_args(c);
    const void *src = c->buf[c->cur];
    LB_CUDA(dispatch(c->cfg.storage, [&](auto ops) {
        return decltype(ops)::adjoint_seed(a, src, nullptr, nullptr, jpart);
    }));
    double out[2];
    lb_status st = sum_pairs(c, jpart, nb, out);
    if (st) return st;
    *J = out[0];
    return LB_OK;
}

lb_status lb_adjoint_ke(lb_ctx *c, int T, int K, void *dJdF, double dJdomega[2], double *J)
{
    if (!c || !dJdF || !dJdomega) return fail(LB_EINVAL, "lb_adjoint_ke: null argument");
    if (T < 1 || K < 1) return fail(LB_EINVAL, "lb_adjoint_ke: T and K must be >= 1");
    if (c->cfg.corr == LB_CORR_FULL) return fail(LB_EINVAL, "lb_adjoint_ke: corrections FULL are not supported");
    if (c->cfg.model != 0) return fail(LB_EINVAL, "lb_adjoint_ke: the raw-moment model is not supported");
    if (c->cfg.lid_u != 0.0 || c->lid_state != 0.0)
        return fail(LB_EINVAL, "lb_adjoint_ke: a moving lid is not supported");
    if (c->cfg.rounding != 0) return fail(LB_EINVAL, "lb_adjoint_ke: needs round-to-nearest storage");
    if (K > T) K = T;
    const size_t sb = lb_state_bytes(c);
    const long long N = c->g.N;
    const int nck = (T + K - 1) / K;
    const long long nb = adjoint_blocks(c->g);
    char *ck = nullptr, *seg = nullptr;
    void *lam[2] = {nullptr, nullptr}, *dF = nullptr;
    double *jpart = nullptr, *wpart = nullptr;
    LB_CUDA(adjoint_buffer(c, 0, (size_t)nck * sb, (void **)&ck));
    if (K > 1) LB_CUDA(adjoint_buffer(c, 1, (size_t)(K - 1) * sb, (void **)&seg));
    LB_CUDA(adjoint_buffer(c, 2, (size_t)Q * N * c->rbytes, &lam[0]));
    LB_CUDA(adjoint_buffer(c, 3, (size_t)Q * N * c->rbytes, &lam[1]));
    LB_CUDA(adjoint_buffer(c, 4, 3 * (size_t)N * c->rbytes, &dF));
    LB_CUDA(adjoint_buffer(c, 5, 2 * nb * sizeof(double), (void **)&jpart));
    LB_CUDA(adjoint_buffer(c, 6, 2 * nb * sizeof(double), (void **)&wpart));
    LB_CUDA(cudaMemsetAsync(jpart, 0, 2 * nb * sizeof(double), c->stream));
    LB_CUDA(cudaMemsetAsync(wpart, 0, 2 * nb * sizeof(double), c->stream));
    const int storage = c->cfg.storage;
    const LaunchArgs a = launch_args(c);
    auto step = [&](const void *src, void *dst) {
        return dispatch(storage, [&](auto ops) { return decltype(ops)::step(a, src, dst); });
    };

    // forward sweep: state 0 is copied into checkpoint 0; each step writes the next state
    // straight into its checkpoint slot (states K, 2K, ...) or into the context's two
    // buffers, which end up holding state T as lb_step(T) would leave it.  With K = 1 all
    // states stay resident and nothing is recomputed below.
    LB_CUDA(cudaMemcpyAsync(ck, c->buf[c->cur], sb, cudaMemcpyDeviceToDevice, c->stream));
    const void *src = ck;
    int w = 0;
    for (int n = 0; n < T; ++n) {
        void *dst;
        if ((n + 1) % K == 0 && (n + 1) / K < nck) {
            dst = ck + (size_t)((n + 1) / K) * sb;
        } else {
            dst = c->buf[w];
            w ^= 1;
        }
        LB_CUDA(step(src, dst));
        src = dst;
    }
    c->cur = (src == c->buf[0]) ? 0 : 1;   // the last step always writes a context buffer
    c->t += T;
    c->fresh = false;
    c->lid_state = c->cfg.lid_u;
    LB_CUDA(dispatch(storage, [&](auto ops) {
        return decltype(ops)::adjoint_seed(a, c->buf[c->cur], lam[0], dF, jpart);
    }));
    // backward sweep: recompute each segment's states n0 + 1 .. n1 - 1 from its
    // checkpoint (state n0), then walk the segment back
    int li = 0;
    for (int sgm = nck - 1; sgm >= 0; --sgm) {
        const int n0 = sgm * K, n1 = std::min(T, n0 + K);
        const char *base = ck + (size_t)sgm * sb;
        auto state = [&](int n) -> const void * { return n == n0 ? base : seg + (size_t)(n - n0 - 1) * sb; };
        for (int n = n0 + 1; n < n1; ++n) LB_CUDA(step(state(n - 1), seg + (size_t)(n - n0 - 1) * sb));
        for (int n = n1 - 1; n >= n0; --n) {
            const void *sn = state(n);
            const void *lin = lam[li];
            void *lout = lam[li ^ 1];
            LB_CUDA(dispatch(storage, [&](auto ops) {
                return decltype(ops)::adjoint_step(a, sn, lin, lout, dF, wpart);
            }));
            li ^= 1;
        }
    }
    LB_CUDA(cudaMemcpyAsync(dJdF, dF, 3 * (size_t)N * c->rbytes, cudaMemcpyDefault, c->stream));
    double jj[2];
    lb_status st = sum_pairs(c, jpart, nb, jj);
    if (st) return st;
    st = sum_pairs(c, wpart, nb, dJdomega);
    if (st) return st;
    if (J) *J = jj[0];
    return LB_OK;
}

lb_status lb_adjoint(lb_ctx *c, int T, int K, void *dJdF, double dJdomega[2])
{
    return lb_adjoint_ke(c, T, K, dJdF, dJdomega, nullptr);
}

lb_status lb_collide_vjp(lb_ctx *c, long long n, const void *f, const void *F, const void *lam, void *f_bar,
                         void *F_bar, double w_bar[2])
{
    if (!c || !f || !F || !lam || !f_bar || !F_bar || !w_bar || n < 1)
        return fail(LB_EINVAL, "lb_collide_vjp: bad argument");
    if (c->cfg.corr == LB_CORR_FULL) return fail(LB_EINVAL, "lb_collide_vjp: corrections FULL are not supported");
    if (c->cfg.model != 0) return fail(LB_EINVAL, "lb_collide_vjp: the raw-moment model is not supported");
    for (const void *p : {f, F, lam, (const void *)f_bar, (const void *)F_bar})
        if (!is_device_pointer(p)) return fail(LB_EINVAL, "lb_collide_vjp: device pointers required");
    Scratch s;
    const long long nb = (n + kAdjThreads - 1) / kAdjThreads;
    double *wpart = nullptr;
    LB_CUDA(s.alloc((void **)&wpart, 2 * nb * sizeof(double)));
    LB_CUDA(cudaMemsetAsync(wpart, 0, 2 * nb * sizeof(double), c->stream));
    const LaunchArgs a = launch_args(c);
    LB_CUDA(dispatch(c->cfg.storage, [&](auto ops) {
        return decltype(ops)::collide_vjp(a, f, F, lam, f_bar, F_bar, n, wpart);
    }));
    return sum_pairs(c, wpart, nb, w_bar);
}

lb_status lb_selftest_bounded_wait(int out[2])
{
    if (!out) return fail(LB_EINVAL, "lb_selftest_bounded_wait: null argument");
    int *d = nullptr;
    LB_CUDA(cudaMalloc(&d, 2 * sizeof(int)));
    cudaError_t e = cudaMemset(d, 0xff, 2 * sizeof(int));
    if (e == cudaSuccess) {
        k_wait_probe<<<1, 32>>>(d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, d, 2 * sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    LB_CUDA(e);
    return LB_OK;
}

const char *lb_step_kernel(const lb_ctx *c)
{
    if (!c) return "";
    const LaunchArgs a = launch_args(c);
    switch (c->cfg.storage) {
    case LB_F64: return Ops<LB_F64>::step_kernel_name(a);
    case LB_F32: return Ops<LB_F32>::step_kernel_name(a);
    case LB_F32_SHIFTED: return Ops<LB_F32_SHIFTED>::step_kernel_name(a);
    case LB_F16_SHIFTED: return Ops<LB_F16_SHIFTED>::step_kernel_name(a);
    default: return Ops<LB_BF16_SHIFTED>::step_kernel_name(a);
    }
}

const char *lb_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace lbc {

void set_last_error(const std::string &msg) { g_last_error = msg; }

__global__ void __launch_bounds__(kReduceThreads)
k_reduce_final(const double *__restrict__ partial, int nblocks, double *__restrict__ out)
{
    __shared__ double sh[4][kReduceThreads];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] += partial[4 * b + c];
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
        for (int c = 0; c < 4; ++c) out[c] = sh[c][0];
}

}  // namespace lbc
