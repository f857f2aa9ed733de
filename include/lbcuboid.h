/*
 * lbcuboid.h -- C ABI of the GB300 (sm_103a) implementation of the fused
 * collide-and-stream update of the cuboid-lattice D3Q27 central-moment lattice
 * Boltzmann method (3DCCM-LBM) of Yahia, Schupbach & Premnath,
 * arXiv:2107.14774.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice units (Sec. 2.1): dx = dt = 1, dy = r_y, dz = r_z.  The 27 particle
 * velocities are e_a = (ex, r_y ey, r_z ez) with (ex, ey, ez) the integer D3Q27
 * stencil in the paper's ordering (Eq. 1a-1c).
 * Node (i, j, k), 0 <= i < nx, ... is stored at index n = i + nx (j + ny k);
 * N = nx ny nz.  Populations are [27][N] (direction-major), density [N],
 * velocity and force [3][N].
 * "real" below is double when the context stores LB_F64 populations and float
 * otherwise (see lb_real_size).
 * A pointer argument may point to device memory or to host memory (pageable or
 * pinned): the library inspects it (cudaPointerGetAttributes) and copies
 * through the context's stream when it is a host pointer.  Caller pointers are
 * only borrowed for the duration of the call; the library copies what it keeps.
 * All work is issued on the context's CUDA stream.  Calls that return host
 * data synchronise that stream.
 *
 * Errors: every call returns an lb_status; nothing aborts or throws.  Parameter
 * errors are reported synchronously (LB_EINVAL); asynchronous CUDA errors
 * surface as LB_ECUDA at the next call that synchronises.  lb_last_error()
 * returns a thread-local message for the last failure.
 *
 * Ownership: the context owns its two population buffers and scratch memory
 * (cudaMalloc at creation, cudaFree at lb_destroy).
 */
#ifndef LBCUBOID_H
#define LBCUBOID_H

#include <stddef.h>

/* The library is built with hidden symbol visibility; the entry points declared here are
 * the only symbols it exports. */
#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_ctx lb_ctx;

typedef enum {
    LB_OK = 0,
    LB_EINVAL = 1,     /* bad argument (sizes, rates, pointer, state) */
    LB_ENOMEM = 2,     /* device allocation failed */
    LB_ECUDA = 3,      /* CUDA runtime error (message in lb_last_error) */
    LB_EUNSTABLE = 4,  /* non-finite or non-positive density found */
    LB_ETIMEOUT = 5,   /* a bounded wait ran out */
    LB_ESTATE = 6      /* call not valid in the context's current state */
} lb_status;

/* Population storage.  Arithmetic is FP64 for LB_F64 and FP32 for the others.
 * The shifted forms store g_a = f_a - w_a rho0 (rho0 = 1, w_a the rest weights
 * f^eq_a(1, 0)); LB_F16_SHIFTED scales each direction by an exact power of two
 * before rounding to binary16 (round to nearest even), LB_BF16_SHIFTED rounds to
 * bfloat16 (round to nearest even). */
typedef enum {
    LB_F64 = 0,
    LB_F32 = 1,
    LB_F32_SHIFTED = 2,
    LB_F16_SHIFTED = 3,
    LB_BF16_SHIFTED = 4
} lb_storage;

/* Second-order equilibrium corrections (Eq. 29-30, 38-40; App. D).
 * NONE: uncorrected cuboid scheme.  LOWMACH: anisotropy terms only (the
 * low-Mach coefficients of Sec. 2.5; no 3u^2 terms, no density gradients).
 * LOCAL: full theta coefficients from the locally recovered diagonal strain
 * rates (Eq. 44-49) with the density-gradient terms dropped.  FULL: LOCAL plus
 * the lambda and e-terms with grad(rho) from second-order central differences
 * of the current density (one-sided next to walls). */
typedef enum {
    LB_CORR_NONE = 0,
    LB_CORR_LOWMACH = 1,
    LB_CORR_LOCAL = 2,
    LB_CORR_FULL = 3
} lb_corr;

#define LB_WALL_X 1u   /* walls normal to x at i = -1/2 and i = nx - 1/2 */
#define LB_WALL_Y 2u
#define LB_WALL_Z 4u

typedef struct {
    int nx, ny, nz;        /* >= 1 each */
    double r_y, r_z;       /* grid aspect ratios r = dy/dx, s = dz/dx (> 0) */
    double nu;             /* shear viscosity > 0: omega_nu = 1/(nu/cs2 + 1/2) (Eq. 53) */
    double zeta;           /* bulk viscosity > 0: omega_xi = 1/(3 zeta/(2 cs2) + 1/2) (Eq. 53);
                              zeta <= 0 selects omega_xi = 1 */
    double cs2;            /* squared sound speed; 0 selects min(1, r^2, s^2)/3 (Sec. 2.6);
                              must satisfy 0 < cs2 < min(1, r^2, s^2) */
    int storage;           /* lb_storage */
    int corr;              /* lb_corr */
    unsigned wall_mask;    /* LB_WALL_* bits: half-way bounce-back walls (Sec. 4); other axes periodic */
    double force[3];       /* uniform body force (lattice units), Eq. 11c */
    double lid_u;          /* velocity along x of the wall at j = ny - 1/2 (needs LB_WALL_Y);
                              momentum-augmented bounce-back (Sec. 4, Eq. 69); 0 = at rest */
    void *stream;          /* cudaStream_t to issue all work on; NULL = the legacy default stream */
    int rounding;          /* 16-bit storage only: 0 = round to nearest even, 1 = stochastic
                              rounding (hardware cvt.rs, random bits from a counter-based hash
                              of (node, direction, time step, rounding_seed)) */
    unsigned rounding_seed;
    int kernel;            /* 0: automatic (two nodes per thread where the lattice allows it,
                              else one node per thread); 1: one node per thread; 2: two nodes
                              per thread; 3: row-staged through shared memory with bulk copies
                              (4- and 2-byte storage, rows of up to 1024 nodes); 4: two nodes per
                              thread marching along z, the next plane's sources copied into
                              shared memory while the current plane is collided (16-bit storage,
                              LOCAL corrections, rows of at least 64 nodes; else as 0); 5: FULL
                              corrections in one pass, the densities of the next plane and of
                              the tile's halo computed on chip instead of by a pre-pass (lattices
                              periodic in y and z with rows of a multiple of 64 nodes; else as 0) */
    int model;             /* collision model: 0 = central moments (3DCCM, Sec. 3.2), 1 = raw
                              moments with the same corrected equilibria (3DCRM, Sec. 3.1 raw
                              formulation and Sec. 7); model 1 needs LB_CORR_LOCAL and is not
                              differentiated by lb_adjoint_ke / lb_collide_vjp */
    int subdomains;        /* 0 or 1: one domain.  P in 2..16 (and <= nz): lb_step updates the
                              lattice as P slabs along z, each with one ghost plane on either
                              side, exchanging after every step the 9 populations with e_z = +1
                              (-1) of a slab's last (first) plane with the next (previous)
                              slab through device memory while the slab interiors update on
                              a second stream -- the slab decomposition a multi-GPU run
                              distributes, on one device; results are bit-identical to one
                              domain.  Needs z periodic, corrections other than FULL, no
                              per-node force field and kernel != 3 (LB_EINVAL otherwise).
                              Every lb_step call copies the state into the slabs and back
                              (two extra state copies per call, not per step). */
} lb_config;

/* Fill *cfg with defaults: FP32 storage, LOCAL corrections, periodic, no
 * force, omega_xi = 1, cs2 = min(1, r^2, s^2)/3. */
void lb_config_default(lb_config *cfg, int nx, int ny, int nz, double r_y, double r_z, double nu);

/* Create a context with the defaults above (lb_create(nx,ny,nz,r_y,r_z,nu,zeta)).
 * zeta <= 0 selects omega_xi = 1.  *out receives the context. */
lb_status lb_create(int nx, int ny, int nz, double r_y, double r_z, double nu, double zeta,
                    lb_ctx **out);

/* Create a context from a full configuration. */
lb_status lb_create_ex(const lb_config *cfg, lb_ctx **out);

/* Release every resource of the context (synchronises its stream).  NULL is ignored. */
void lb_destroy(lb_ctx *ctx);

/* Bytes of one "real" of this context: 8 (LB_F64) or 4. */
int lb_real_size(const lb_ctx *ctx);

/* Nodes N = nx ny nz. */
size_t lb_num_nodes(const lb_ctx *ctx);

/* Relaxation rates and sound speed in use: out[0] = omega_nu, out[1] = omega_xi, out[2] = cs2. */
lb_status lb_get_params(const lb_ctx *ctx, double out[3]);

/* Initialise the populations to the equilibrium f^eq(rho, u) (Eq. 9, 10) at every
 * node; rho [N] and u [3][N] in the context's real type.  The density and
 * velocity returned by lb_moments right after lb_init are rho and u + F/(2 rho). */
lb_status lb_init(lb_ctx *ctx, const void *rho, const void *u);

/* Optional per-node body force [3][N] (real), added to the uniform force; copied
 * into the context.  NULL removes it. */
lb_status lb_set_force_field(lb_ctx *ctx, const void *force);

/* Enqueue n fused collide-and-stream steps (Sec. 3.2 algorithm; Apps. A-G) on the
 * context's stream.  Asynchronous; errors of the launches are reported here,
 * errors during execution at the next synchronising call. */
lb_status lb_step(lb_ctx *ctx, int n);

/* Density [N] and velocity [3][N] (real) of the current populations:
 * rho = sum f, rho u = sum f e + F/2 (Eq. 12).  Synchronises. */
lb_status lb_moments(lb_ctx *ctx, void *rho, void *u);

/* FP64 global sums out[0] = sum rho, out[1..3] = sum rho u (host array), computed
 * with a deterministic two-pass reduction.  Returns LB_EUNSTABLE (with the sums
 * still written) if any node has a non-finite or non-positive density or a
 * non-finite velocity, and LB_ETIMEOUT if a bounded wait inside a step kernel ran
 * out since the context was created (the state is then not valid).  Synchronises. */
lb_status lb_reduce(lb_ctx *ctx, double out_mass_momentum[4]);

/* Copy the pre-collision populations f_a(x, t) [27][N] (real) out of / into the
 * context.  Exact for LB_F64 and LB_F32; the shifted forms convert between f and
 * the stored g = f - w rho0 in the real type. */
lb_status lb_get_populations(lb_ctx *ctx, void *dst);
lb_status lb_set_populations(lb_ctx *ctx, const void *src);

/* Raw checkpoint of the stored state: lb_state_bytes() bytes in the library's
 * internal layout (27 N stored values), copied out of / into the context.
 * Resuming from it is bit-identical to an uninterrupted run. */
size_t lb_state_bytes(const lb_ctx *ctx);
lb_status lb_get_state(lb_ctx *ctx, void *dst);
lb_status lb_set_state(lb_ctx *ctx, const void *src, long long time_step);

/* Number of completed time steps since the last lb_init / lb_set_populations. */
long long lb_time_step(const lb_ctx *ctx);

/* Replace the uniform body force (Eq. 11c) for the steps enqueued after this call
 * (a time-dependent forcing such as the pulsatile duct of Sec. 5.2 updates it
 * between lb_step calls; the step from t to t + 1 uses the force set before it).
 * force: host array of 3 doubles, read during the call.  LB_EINVAL on a null
 * pointer or a non-finite component. */
lb_status lb_set_force(lb_ctx *ctx, const double force[3]);

/* Set the relaxation rates of the shear and bulk parts of the second-order moments
 * directly (App. D; they map to nu and xi through Eq. 53) for the steps enqueued
 * after this call.  LB_EINVAL unless 0 < omega < 2 for both. */
lb_status lb_set_rates(lb_ctx *ctx, double omega_nu, double omega_xi);

/* Replace the lid velocity (the x velocity of the wall at j = ny - 1/2 in the
 * momentum-augmented bounce-back of Sec. 4, Eq. 69) for the steps enqueued after this
 * call: the step from t to t + 1 (collision at t, then streaming with the wall term into
 * t + 1) uses the velocity set before the lb_step call that runs it, as lb_set_force
 * does for the force.  A lid started from rest and brought up to speed over many steps
 * is set this way between lb_step calls.  LB_EINVAL on a non-finite value, or on a
 * non-zero one without walls normal to y. */
lb_status lb_set_lid(lb_ctx *ctx, double lid_u);

/* Mean kinetic energy J = (1/N) sum_x rho |u|^2 / 2 of the current populations,
 * u including the F/2 shift (Eq. 12); FP64 sum, deterministic.  Synchronises. */
lb_status lb_objective_ke(lb_ctx *ctx, double *J);

/* Discrete adjoint of T fused steps (Sec. 3.2 update, transposed) for the mean
 * kinetic energy J after T steps, starting from the current state.  Returns J,
 * dJ/dF [3][N] (real; the gradient with respect to the per-node body force field,
 * i.e. to the total force at each node) and dJ/domega = (dJ/domega_nu,
 * dJ/domega_xi) on the host.  The forward states are kept every K steps
 * (checkpoints, written there by the step kernels themselves) and each K-step segment
 * is recomputed once during the backward sweep, so device memory grows as
 * (ceil(T/K) + K - 1) stored states of lb_state_bytes each.  K = 1 keeps all T states
 * resident and recomputes nothing (a 128x64x64 FP32 lattice takes 57 MB per state).
 * These work buffers are allocated by the first call that needs them and kept by the
 * context for later calls (grown when a call needs more); lb_destroy frees them.  If
 * the call returns an error, the context's state is undefined until lb_init,
 * lb_set_populations or lb_set_state sets it again.  On return the context holds
 * the state after the T steps (as after lb_step(ctx, T)).  Corrections NONE,
 * LOWMACH or LOCAL; no moving lid (LB_EINVAL otherwise).  Synchronises. */
lb_status lb_adjoint_ke(lb_ctx *ctx, int T, int K, void *dJdF, double dJdomega[2], double *J);
/* (lb_adjoint_ke also requires round-to-nearest storage: rounding = 0.) */

/* The same adjoint without returning J (the objective is the mean kinetic energy). */
lb_status lb_adjoint(lb_ctx *ctx, int T, int K, void *dJdF, double dJdomega[2]);

/* Self-test of failure detection without a GPU fault (no counterpart in the paper):
 * runs one thread that waits, with the bounded mbarrier wait of the row-staged kernel
 * and a short limit, on a phase nothing completes, then completes it and waits again.
 * out[0] = 1 if the first wait gave up (as it must), out[1] = 1 if the second
 * succeeded.  Uses the current device and the legacy default stream; synchronises. */
lb_status lb_selftest_bounded_wait(int out[2]);

/* Vector-Jacobian product of the per-node collision alone, for n independent
 * nodes (device pointers, real type): f [27][n] pre-collision populations,
 * F [3][n] body force, lam [27][n] = dJ/d(post-collision populations).  Writes
 * f_bar [27][n] = dJ/df, F_bar [3][n] = dJ/dF and w_bar = (dJ/domega_nu,
 * dJ/domega_xi) summed over the nodes (host).  Synchronises. */
lb_status lb_collide_vjp(lb_ctx *ctx, long long n, const void *f, const void *F, const void *lam, void *f_bar,
                         void *F_bar, double w_bar[2]);

/* FP64 sums out[0] = sum rho and out[1..3] = sum rho u (rho u = sum f e + F/2)
 * of n nodes, from pre-collision populations f [27][n] (device memory of the
 * current device or managed memory -- anything else, host memory included, returns
 * LB_EINVAL before any launch; natural layout as returned by lb_get_populations;
 * real_size 4 = float, 8 = double), for a lattice with aspect ratios r_y, r_z and
 * the uniform body force `force` (NULL = none).  A per-node force field
 * (lb_set_force_field) is not included: with one, the momentum differs from
 * lb_reduce's by half the summed field.  This entry point has no counterpart in the paper: it is the reduction of
 * lb_reduce for callers that cannot allocate device memory -- hosts whose
 * framework owns all device memory through its own pool, real-time loops that
 * must never enter the driver allocator.  It calls no cudaMalloc or cudaFree: its per-block partial sums and
 * status word live in one fixed array in the library's device globals (about
 * 131 KB, held by every GPU that loads the library until the process exits), so
 * n is limited to 134,217,728 nodes (LB_EINVAL beyond).  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with the
 * device current and keeps it for the life of the process (a cudaDeviceReset of that
 * device makes it stale: do not call this entry point after one); make that first
 * call before any stream capture.  All calls
 * share the array: calls that overlap on the GPU (other streams, other threads)
 * race and must be serialised by the caller; the array keeps the last call's
 * contents.  Work is issued on `stream` (cudaStream_t, NULL = default stream) and
 * the call synchronises it.  Returns LB_EUNSTABLE (sums still written) if a node
 * has a non-finite or non-positive density. */
lb_status lb_reduce_populations_noalloc(const void *f, int real_size, long long n, double r_y, double r_z,
                                        const double force[3], double out[4], void *stream);

/* Name (with template arguments) of the step kernel lb_step launches for this
 * context, e.g. "k_step_pair<F32,LOCAL,1,false,periodic>"; thread-local storage, valid
 * until the next call on the same thread.  No counterpart in the paper. */
const char *lb_step_kernel(const lb_ctx *ctx);

/* Message of the last error on this thread ("" if none). */
const char *lb_last_error(void);

#ifdef __cplusplus
}
#endif

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#endif /* LBCUBOID_H */
