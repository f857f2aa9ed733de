/*
 * lbref.c -- FP64 CPU oracle of the cuboid-lattice D3Q27 central-moment
 * lattice Boltzmann scheme (3DCCM-LBM) of Yahia, Schupbach & Premnath,
 * "Three-Dimensional Central Moment Lattice Boltzmann Method on a Cuboid
 * Lattice for Anisotropic and Inhomogeneous Flows" (arXiv:2107.14774).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load it.  It shares no code, header, table
 * or constant with the CUDA library, and the library never calls it.
 *
 * Everything is double precision.  Build with -ffp-contract=off so that no
 * multiply-add is fused behind the reader's back.
 *
 * Two independent forms of the per-node collision are provided:
 *   form 0 ("factored"):     m = P f; m <- S m; m^c = F(u) m; relax (App. D);
 *                            m~ = F(-u) m~^c; m~ <- S^-1 m~; f~ = P^-1 m~
 *                            (Secs. 3.1-3.2, the central-moment update of Sec. 3.1,
 *                            Apps. A-G).  P^-1 is obtained by Gauss-Jordan.
 *   form 1 ("definitional"): k_mnp = sum_a f_a (e_ax-ux)^m (e_ay-uy)^n
 *                            (e_az-uz)^p with the cuboid velocities (Eq. 3a);
 *                            relax (App. D); f~ solves M(u) f~ = k~ by LU.
 * Streaming follows Sec. 3.2 (f_a(x,t+1) = f~_a(x - e_a, t)); walls are the
 * link-wise half-way bounce-back of Sec. 4 (its momentum-augmented form),
 * with the wall-velocity term of the moving lid when a lid is configured.
 *
 * Readings of points where the paper is silent or garbled (all listed in the
 * design notes of the repository):
 *   - c_s^2 is a parameter (Table 1 uses values other than min(r^2,s^2)/3);
 *   - corrections mode LOCAL drops the density-gradient terms (grad rho := 0),
 *     LOWMACH additionally drops the 3u^2 aliasing parts of theta and of the
 *     C coefficients (Sec. 2.5, last remark), NONE uses no correction, FULL
 *     takes grad rho from second-order central differences of the current
 *     density field (one-sided second-order differences next to a wall);
 *   - every relaxation rate other than omega_nu, omega_xi is 1 (App. D);
 *   - the initial state is f = f^eq(rho, u) = Q^-1 m^eq (Eq. 10);
 *   - the optional storage emulation rounds what a reduced-precision store
 *     keeps: the deviation g_a = f_a - w_a from the rest weights w_a =
 *     f^eq_a(1, 0), after the collision (and after initialisation), to
 *     binary16 scaled per direction by 2^(10 - ilogb w_a), or to bfloat16,
 *     rounding to nearest with ties to even.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NQ 27

/* Cubic D3Q27 velocities in the paper's ordering (Sec. 3.1, cubic lattice
 * velocities); the cuboid velocities of Eq. 1a-1c are (ex, r*ey, s*ez). */
static const int EX[NQ] = {0,1,-1,0,0,0,0,1,-1,1,-1,1,-1,1,-1,0,0,0,0,1,-1,1,-1,1,-1,1,-1};
static const int EY[NQ] = {0,0,0,1,-1,0,0,1,1,-1,-1,0,0,0,0,1,-1,1,-1,1,1,-1,-1,1,1,-1,-1};
static const int EZ[NQ] = {0,0,0,0,0,1,-1,0,0,0,0,1,1,-1,-1,1,1,-1,-1,1,1,1,1,-1,-1,-1,-1};

/* Exponents (m,n,p) of the moments in the order of the raw-moment list m
 * (Sec. 3.1, the list of raw moments) and of the central-moment list m^c. */
static const int MM[NQ] = {0,1,0,0,1,1,0,2,0,0,1,1,2,0,2,0,1,2,2,0,2,1,1,1,2,2,2};
static const int MN[NQ] = {0,0,1,0,1,0,1,0,2,0,2,0,1,1,0,2,1,2,0,2,1,2,1,2,1,2,2};
static const int MP[NQ] = {0,0,0,1,0,1,1,0,0,2,0,2,0,2,1,1,1,0,2,2,1,1,2,2,2,1,2};

enum { CORR_NONE = 0, CORR_LOWMACH = 1, CORR_LOCAL = 2, CORR_FULL = 3 };

typedef struct {
    int nx, ny, nz;
    unsigned wall_mask;        /* bit0: walls normal to x, bit1: y, bit2: z; else periodic */
    double r, s;               /* grid aspect ratios dy/dx, dz/dx (Sec. 2.1) */
    double cs2;                /* speed of sound squared */
    double omega_nu, omega_xi; /* shear and bulk relaxation rates (App. D) */
    int corr;                  /* CORR_* */
    int form;                  /* 0 factored, 1 definitional */
    double force[3];           /* uniform body force */
    const double *force_field; /* optional per-node force [3][nz][ny][nx], added to force */
    double lid_u;              /* velocity (along x) of the wall at y = ny-1/2; 0 = at rest */
    int model;                 /* 0 central moments (3DCCM), 1 raw moments (3DCRM, Sec. 7) */
    int storage_emulation;     /* 0 none; 1 or 2: round every stored deviation g = f - w to
                                  binary16 (times 2^(10 - ilogb w_a)) or to bfloat16 */
} or_params;

/* ------------------------------------------------------------------------ */
/* Small dense linear algebra                                                */

static double ipow(double x, int k)
{
    double v = 1.0;
    for (int i = 0; i < k; ++i) v *= x;
    return v;
}

/* Gauss-Jordan inversion with partial pivoting; returns 0 on success. */
static int invert27(const double A[NQ][NQ], double Ainv[NQ][NQ])
{
    double a[NQ][2 * NQ];
    for (int i = 0; i < NQ; ++i)
        for (int j = 0; j < NQ; ++j) {
            a[i][j] = A[i][j];
            a[i][NQ + j] = (i == j) ? 1.0 : 0.0;
        }
    for (int c = 0; c < NQ; ++c) {
        int piv = c;
        for (int i = c + 1; i < NQ; ++i)
            if (fabs(a[i][c]) > fabs(a[piv][c])) piv = i;
        if (a[piv][c] == 0.0) return -1;
        if (piv != c)
            for (int j = 0; j < 2 * NQ; ++j) {
                double t = a[c][j]; a[c][j] = a[piv][j]; a[piv][j] = t;
            }
        double d = a[c][c];
        for (int j = 0; j < 2 * NQ; ++j) a[c][j] /= d;
        for (int i = 0; i < NQ; ++i) {
            if (i == c || a[i][c] == 0.0) continue;
            double m = a[i][c];
            for (int j = 0; j < 2 * NQ; ++j) a[i][j] -= m * a[c][j];
        }
    }
    for (int i = 0; i < NQ; ++i)
        for (int j = 0; j < NQ; ++j) Ainv[i][j] = a[i][NQ + j];
    return 0;
}

/* Solve A x = b by LU decomposition with partial pivoting; returns 0 on success. */
static int lu_solve27(const double A[NQ][NQ], const double b[NQ], double x[NQ])
{
    double a[NQ][NQ], y[NQ];
    int perm[NQ];
    memcpy(a, A, sizeof(a));
    for (int i = 0; i < NQ; ++i) perm[i] = i;
    for (int c = 0; c < NQ; ++c) {
        int piv = c;
        for (int i = c + 1; i < NQ; ++i)
            if (fabs(a[i][c]) > fabs(a[piv][c])) piv = i;
        if (a[piv][c] == 0.0) return -1;
        if (piv != c) {
            for (int j = 0; j < NQ; ++j) { double t = a[c][j]; a[c][j] = a[piv][j]; a[piv][j] = t; }
            int t = perm[c]; perm[c] = perm[piv]; perm[piv] = t;
        }
        for (int i = c + 1; i < NQ; ++i) {
            a[i][c] /= a[c][c];
            for (int j = c + 1; j < NQ; ++j) a[i][j] -= a[i][c] * a[c][j];
        }
    }
    for (int i = 0; i < NQ; ++i) {               /* forward: L y = P b */
        double v = b[perm[i]];
        for (int j = 0; j < i; ++j) v -= a[i][j] * y[j];
        y[i] = v;
    }
    for (int i = NQ - 1; i >= 0; --i) {          /* backward: U x = y */
        double v = y[i];
        for (int j = i + 1; j < NQ; ++j) v -= a[i][j] * x[j];
        x[i] = v / a[i][i];
    }
    return 0;
}

static void matvec27(const double A[NQ][NQ], const double x[NQ], double y[NQ])
{
    for (int i = 0; i < NQ; ++i) {
        double v = 0.0;
        for (int j = 0; j < NQ; ++j) v += A[i][j] * x[j];
        y[i] = v;
    }
}

/* ------------------------------------------------------------------------ */
/* Matrices of Sec. 3.1                                                      */

static double g_P[NQ][NQ], g_Pinv[NQ][NQ];
static int g_ready = 0;
static int g_KI[3][3][3];   /* (m,n,p) -> position in the moment list */
static int g_OPP[NQ];       /* opposite direction: e_opp = -e */

/* P: moment basis of the cubic lattice, P[j][a] = ex^m ey^n ez^p with the
 * cubic velocities (Sec. 3.1, the moment basis of the cubic lattice). */
static void setup(void)
{
    if (g_ready) return;
    for (int j = 0; j < NQ; ++j)
        for (int a = 0; a < NQ; ++a)
            g_P[j][a] = ipow(EX[a], MM[j]) * ipow(EY[a], MN[j]) * ipow(EZ[a], MP[j]);
    invert27(g_P, g_Pinv);
    for (int j = 0; j < NQ; ++j) g_KI[MM[j]][MN[j]][MP[j]] = j;
    for (int a = 0; a < NQ; ++a)
        for (int b = 0; b < NQ; ++b)
            if (EX[b] == -EX[a] && EY[b] == -EY[a] && EZ[b] == -EZ[a]) g_OPP[a] = b;
    g_ready = 1;
}

/* S: diagonal scaling of the raw moments by r^n s^p (Eq. 58-59, App. B). */
static void scaling_S(double r, double s, double S[NQ])
{
    for (int j = 0; j < NQ; ++j) S[j] = ipow(r, MN[j]) * ipow(s, MP[j]);
}

static double binom(int n, int k)
{
    static const double C[3][3] = {{1, 0, 0}, {1, 1, 0}, {1, 2, 1}};
    return C[n][k];
}

/* Frame transformation F(u): central moments from raw moments by the binomial
 * expansion of (e_x-u_x)^m (e_y-u_y)^n (e_z-u_z)^p (Eq. 3a vs Eq. 3b,
 * Sec. 3.1 mapping of raw to central moments, App. C):
 *   k_mnp = sum_{a<=m, b<=n, c<=p} C(m,a) C(n,b) C(p,c)
 *           (-u_x)^(m-a) (-u_y)^(n-b) (-u_z)^(p-c) k'_abc.
 * F(-u) is its inverse (App. E). */
static void frame_F(const double u[3], double F[NQ][NQ])
{
    for (int i = 0; i < NQ; ++i) {
        int m = MM[i], n = MN[i], p = MP[i];
        for (int j = 0; j < NQ; ++j) {
            int a = MM[j], b = MN[j], c = MP[j];
            if (a > m || b > n || c > p) { F[i][j] = 0.0; continue; }
            F[i][j] = binom(m, a) * binom(n, b) * binom(p, c)
                    * ipow(-u[0], m - a) * ipow(-u[1], n - b) * ipow(-u[2], p - c);
        }
    }
}

/* M(u): central-moment matrix of the cuboid lattice by its definition (Eq. 3a):
 * M[j][a] = (e_ax-u_x)^m (r e_ay-u_y)^n (s e_az-u_z)^p. */
static void central_M(double r, double s, const double u[3], double M[NQ][NQ])
{
    for (int j = 0; j < NQ; ++j)
        for (int a = 0; a < NQ; ++a)
            M[j][a] = ipow(EX[a] - u[0], MM[j]) * ipow(r * EY[a] - u[1], MN[j])
                    * ipow(s * EZ[a] - u[2], MP[j]);
}

/* ------------------------------------------------------------------------ */
/* Collision in central moments (App. D)                                     */

#define K(m, n, p) k[g_KI[m][n][p]]
#define KS(m, n, p) sig[g_KI[m][n][p]]
#define KT(m, n, p) kt[g_KI[m][n][p]]

/* Diagonal strain rates recovered locally from the non-equilibrium second
 * order central moments (Eq. 44-49, written with the shear/bulk subscripts of
 * App. D).  The inputs are the non-equilibrium combinations n2s = k_2s - 3 cs2 rho,
 * k2d1 = k_200 - k_020, k2d2 = k_200 - k_002.  gr = density gradient (zero unless
 * mode FULL).  al = 1 keeps the 3u^2 aliasing terms, 0 drops them (low-Mach form). */
static void strain_rates_n(const or_params *p, double n2s, double k2d1, double k2d2, double rho,
                           const double u[3], const double gr[3], double al, double d[3])
{
    const double cs2 = p->cs2, r2 = p->r * p->r, s2 = p->s * p->s;
    const double wn = p->omega_nu, wb = p->omega_xi;
    const double ux = u[0], uy = u[1], uz = u[2];
    double A = 0.5 * (3.0 * cs2 - 1.0) * ux;
    double B = 0.5 * (3.0 * cs2 - r2) * uy;
    double C = 0.5 * (3.0 * cs2 - s2) * uz;
    double e_sr1 = -A * gr[0] + B * gr[1];
    double e_sr2 = -A * gr[0] + C * gr[2];
    double e_br = -A * gr[0] - B * gr[1] - C * gr[2];
    double R_b = n2s + e_br;
    double R_s1 = k2d1 + e_sr1;
    double R_s2 = k2d2 + e_sr2;
    double C_sx = (-2.0 * cs2 / wn + 0.5 * (3.0 * cs2 - 1.0) + al * 1.5 * ux * ux) * rho;
    double C_bx = (-2.0 * cs2 / wb + 0.5 * (3.0 * cs2 - 1.0) + al * 1.5 * ux * ux) * rho;
    double C_sy = (2.0 * cs2 / wn - 0.5 * (3.0 * cs2 - r2) - al * 1.5 * uy * uy) * rho;
    double C_by = (-2.0 * cs2 / wb + 0.5 * (3.0 * cs2 - r2) + al * 1.5 * uy * uy) * rho;
    double C_sz = (2.0 * cs2 / wn - 0.5 * (3.0 * cs2 - s2) - al * 1.5 * uz * uz) * rho;
    double C_bz = (-2.0 * cs2 / wb + 0.5 * (3.0 * cs2 - s2) + al * 1.5 * uz * uz) * rho;
    double num = -C_sz * C_by * R_s1 - C_sy * (C_bz * R_s2 - C_sz * R_b);
    double den = -C_sx * C_sz * C_by - C_sy * (C_sx * C_bz - C_sz * C_bx);
    d[0] = num / den;
    d[1] = (R_s1 - C_sx * d[0]) / C_sy;
    d[2] = (R_s2 - C_sx * d[0]) / C_sz;
}

static void strain_rates(const or_params *p, const double k[NQ], double rho, const double u[3],
                         const double gr[3], double al, double d[3])
{
    double k2s = K(2,0,0) + K(0,2,0) + K(0,0,2);
    strain_rates_n(p, k2s - 3.0 * p->cs2 * rho, K(2,0,0) - K(0,2,0), K(2,0,0) - K(0,0,2), rho, u, gr, al, d);
}

/* Effective equilibria of the combined second-order moments (Eq. 63 of App. D;
 * corrections of Eq. 30 with the coefficients of Eq. 38-40): eq = base + the
 * theta terms times the local strain rates + the lambda terms times grad rho.
 * base = the uncorrected equilibria of (k_2s, k_2d1, k_2d2); n2s, k2d1, k2d2 =
 * the non-equilibrium parts handed to the strain-rate recovery. */
static void corrected_equilibria(const or_params *p, double n2s, double k2d1, double k2d2, double rho,
                                 const double u[3], const double grad_rho[3], const double base[3],
                                 double eq[3])
{
    const double cs2 = p->cs2, r2 = p->r * p->r, s2 = p->s * p->s;
    const double wn = p->omega_nu, wb = p->omega_xi;
    const double ux = u[0], uy = u[1], uz = u[2];
    eq[0] = base[0]; eq[1] = base[1]; eq[2] = base[2];
    if (p->corr == CORR_NONE) return;
    double gr[3] = {0.0, 0.0, 0.0};
    double al = (p->corr == CORR_LOWMACH) ? 0.0 : 1.0;
    if (p->corr == CORR_FULL) { gr[0] = grad_rho[0]; gr[1] = grad_rho[1]; gr[2] = grad_rho[2]; }
    double d[3];
    strain_rates_n(p, n2s, k2d1, k2d2, rho, u, gr, al, d);
    double tn = 1.0 / wn - 0.5, tb = 1.0 / wb - 0.5;
    double th_sx = -rho * (al * 3.0 * ux * ux + 3.0 * cs2 - 1.0) * tn;
    double th_sy = -rho * (al * 3.0 * uy * uy + 3.0 * cs2 - r2) * tn;
    double th_sz = -rho * (al * 3.0 * uz * uz + 3.0 * cs2 - s2) * tn;
    double th_bx = -rho * (al * 3.0 * ux * ux + 3.0 * cs2 - 1.0) * tb;
    double th_by = -rho * (al * 3.0 * uy * uy + 3.0 * cs2 - r2) * tb;
    double th_bz = -rho * (al * 3.0 * uz * uz + 3.0 * cs2 - s2) * tb;
    double la_sx = -(3.0 * cs2 - 1.0) * tn * ux;
    double la_sy = +(3.0 * cs2 - r2) * tn * uy;
    double la_sz = +(3.0 * cs2 - s2) * tn * uz;
    double la_bx = -(3.0 * cs2 - 1.0) * tb * ux;
    double la_by = -(3.0 * cs2 - r2) * tb * uy;
    double la_bz = -(3.0 * cs2 - s2) * tb * uz;
    eq[0] = base[0] + th_bx * d[0] + th_by * d[1] + th_bz * d[2]
          + la_bx * gr[0] + la_by * gr[1] + la_bz * gr[2];
    eq[1] = base[1] + th_sx * d[0] - th_sy * d[1] + la_sx * gr[0] + la_sy * gr[1];
    eq[2] = base[2] + th_sx * d[0] - th_sz * d[2] + la_sx * gr[0] + la_sz * gr[2];
}

/* Post-collision central moments kt from pre-collision central moments k. */
static void relax_central(const or_params *p, const double k[NQ], double rho, const double u[3],
                          const double F[3], const double grad_rho[3], double kt[NQ])
{
    const double cs2 = p->cs2, cs4 = cs2 * cs2, cs6 = cs4 * cs2;
    const double wn = p->omega_nu, wb = p->omega_xi;
    /* every other relaxation rate is unity (App. D) */
    const double w1 = 1.0, w3 = 1.0, w111 = 1.0, w211 = 1.0, w4 = 1.0, w122 = 1.0, w222 = 1.0;

    /* B: combine selected moments (App. D, combined pre-collision central moments) */
    double k2s = K(2,0,0) + K(0,2,0) + K(0,0,2);
    double k2d1 = K(2,0,0) - K(0,2,0);
    double k2d2 = K(2,0,0) - K(0,0,2);
    double k3s1 = K(1,2,0) + K(1,0,2), k3m1 = K(1,2,0) - K(1,0,2);
    double k3s2 = K(2,1,0) + K(0,1,2), k3m2 = K(2,1,0) - K(0,1,2);
    double k3s3 = K(2,0,1) + K(0,2,1), k3m3 = K(2,0,1) - K(0,2,1);
    double k4s = K(2,2,0) + K(2,0,2) + K(0,2,2);
    double k4d1 = K(2,2,0) + K(2,0,2) - K(0,2,2);
    double k4d2 = K(2,2,0) - K(2,0,2);

    /* effective equilibria of the combined second-order moments (App. D) */
    const double base[3] = {3.0 * cs2 * rho, 0.0, 0.0};
    double eq[3];
    corrected_equilibria(p, k2s - 3.0 * cs2 * rho, k2d1, k2d2, rho, u, grad_rho, base, eq);
    const double k2s_eq = eq[0], k2d1_eq = eq[1], k2d2_eq = eq[2];

    /* relaxation (App. D); source central moments: sigma_100 = F (Eq. 11c) */
    double t100 = K(1,0,0) + w1 * (0.0 - K(1,0,0)) + (1.0 - 0.5 * w1) * F[0];
    double t010 = K(0,1,0) + w1 * (0.0 - K(0,1,0)) + (1.0 - 0.5 * w1) * F[1];
    double t001 = K(0,0,1) + w1 * (0.0 - K(0,0,1)) + (1.0 - 0.5 * w1) * F[2];
    double t110 = K(1,1,0) + wn * (0.0 - K(1,1,0));
    double t101 = K(1,0,1) + wn * (0.0 - K(1,0,1));
    double t011 = K(0,1,1) + wn * (0.0 - K(0,1,1));
    double t2d1 = k2d1 + wn * (k2d1_eq - k2d1);
    double t2d2 = k2d2 + wn * (k2d2_eq - k2d2);
    double t2s = k2s + wb * (k2s_eq - k2s);
    double t3s1 = k3s1 + w3 * (0.0 - k3s1), t3m1 = k3m1 + w3 * (0.0 - k3m1);
    double t3s2 = k3s2 + w3 * (0.0 - k3s2), t3m2 = k3m2 + w3 * (0.0 - k3m2);
    double t3s3 = k3s3 + w3 * (0.0 - k3s3), t3m3 = k3m3 + w3 * (0.0 - k3m3);
    double t111 = K(1,1,1) + w111 * (0.0 - K(1,1,1));
    double t211 = K(2,1,1) + w211 * (0.0 - K(2,1,1));
    double t121 = K(1,2,1) + w211 * (0.0 - K(1,2,1));
    double t112 = K(1,1,2) + w211 * (0.0 - K(1,1,2));
    double t4s = k4s + w4 * (3.0 * cs4 * rho - k4s);
    double t4d1 = k4d1 + w4 * (cs4 * rho - k4d1);
    double t4d2 = k4d2 + w4 * (0.0 - k4d2);
    double t122 = K(1,2,2) + w122 * (0.0 - K(1,2,2));
    double t212 = K(2,1,2) + w122 * (0.0 - K(2,1,2));
    double t221 = K(2,2,1) + w122 * (0.0 - K(2,2,1));
    double t222 = K(2,2,2) + w222 * (cs6 * rho - K(2,2,2));

    /* B^-1: segregate the combined moments again (end of App. D) */
    KT(0,0,0) = K(0,0,0);
    KT(1,0,0) = t100; KT(0,1,0) = t010; KT(0,0,1) = t001;
    KT(1,1,0) = t110; KT(1,0,1) = t101; KT(0,1,1) = t011;
    KT(2,0,0) = (t2s + t2d1 + t2d2) / 3.0;
    KT(0,2,0) = (t2s - 2.0 * t2d1 + t2d2) / 3.0;
    KT(0,0,2) = (t2s + t2d1 - 2.0 * t2d2) / 3.0;
    KT(1,2,0) = 0.5 * (t3s1 + t3m1); KT(1,0,2) = 0.5 * (t3s1 - t3m1);
    KT(2,1,0) = 0.5 * (t3s2 + t3m2); KT(0,1,2) = 0.5 * (t3s2 - t3m2);
    KT(2,0,1) = 0.5 * (t3s3 + t3m3); KT(0,2,1) = 0.5 * (t3s3 - t3m3);
    KT(1,1,1) = t111;
    KT(2,2,0) = 0.25 * (t4s + t4d1 + 2.0 * t4d2);
    KT(2,0,2) = 0.25 * (t4s + t4d1 - 2.0 * t4d2);
    KT(0,2,2) = 0.5 * (t4s - t4d1);
    KT(2,1,1) = t211; KT(1,2,1) = t121; KT(1,1,2) = t112;
    KT(1,2,2) = t122; KT(2,1,2) = t212; KT(2,2,1) = t221;
    KT(2,2,2) = t222;
}

/* Raw-moment equilibria (Eq. 10): the binomial transform of Eq. 9, which is the
 * product rho mu_m(u_x) mu_n(u_y) mu_p(u_z) with mu_0 = 1, mu_1 = u, mu_2 = cs2 + u^2. */
static void raw_equilibrium(double cs2, double rho, const double u[3], double meq[NQ])
{
    for (int j = 0; j < NQ; ++j) {
        double v = rho;
        const int e[3] = {MM[j], MN[j], MP[j]};
        for (int i = 0; i < 3; ++i) {
            if (e[i] == 1) v *= u[i];
            else if (e[i] == 2) v *= cs2 + u[i] * u[i];
        }
        meq[j] = v;
    }
}

/* Raw moments of the source term (Eq. 11). */
static void raw_source(const double F[3], const double u[3], double sig[NQ])
{
    for (int j = 0; j < NQ; ++j) sig[j] = 0.0;
    KS(1,0,0) = F[0]; KS(0,1,0) = F[1]; KS(0,0,1) = F[2];
    KS(1,1,0) = F[0] * u[1] + F[1] * u[0];
    KS(1,0,1) = F[0] * u[2] + F[2] * u[0];
    KS(0,1,1) = F[1] * u[2] + F[2] * u[1];
    KS(2,0,0) = 2.0 * F[0] * u[0];
    KS(0,2,0) = 2.0 * F[1] * u[1];
    KS(0,0,2) = 2.0 * F[2] * u[2];
}

/* Post-collision raw moments mt of the raw-moment scheme (3DCRM: the cuboid
 * raw-moment formulation of Sec. 3.1 (its raw-moment update), with the
 * corrected equilibria of the central scheme, Sec. 7):
 *   mt = m + B^-1 { Lambda (B m^eq - B m) + (I - Lambda/2) B Phi },
 * m^eq from Eq. 10, Phi from Eq. 11, Lambda = omega_nu on the off-diagonal and
 * deviatoric second-order moments, omega_xi on their trace, 1 elsewhere.  For
 * the groups that B combines above second order all rates are 1, so B and B^-1
 * cancel there.  The strain rates of the corrections take the second-order
 * non-equilibrium moments m - m^eq + Phi/2, the quantity that equals the central
 * non-equilibrium moments (Sec. 2.6 equates the two; with a body force they
 * differ by Phi/2). */
static void relax_raw(const or_params *p, const double m[NQ], double rho, const double u[3],
                      const double F[3], const double grad_rho[3], double mt[NQ])
{
    const double wn = p->omega_nu, wb = p->omega_xi;
    double meq[NQ], sig[NQ];
    raw_equilibrium(p->cs2, rho, u, meq);
    raw_source(F, u, sig);
    /* rate 1 everywhere first: mt = m + (m^eq - m) + Phi/2 */
    for (int j = 0; j < NQ; ++j) mt[j] = m[j] + 1.0 * (meq[j] - m[j]) + (1.0 - 0.5) * sig[j];
    mt[g_KI[0][0][0]] = m[g_KI[0][0][0]];
    /* off-diagonal second-order moments at omega_nu */
    const int off[3][3] = {{1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
    for (int i = 0; i < 3; ++i) {
        const int j = g_KI[off[i][0]][off[i][1]][off[i][2]];
        mt[j] = m[j] + wn * (meq[j] - m[j]) + (1.0 - 0.5 * wn) * sig[j];
    }
    /* B: trace and the two deviatoric combinations of the diagonal moments */
    const int jx = g_KI[2][0][0], jy = g_KI[0][2][0], jz = g_KI[0][0][2];
    double c2s = m[jx] + m[jy] + m[jz], c2d1 = m[jx] - m[jy], c2d2 = m[jx] - m[jz];
    const double base[3] = {meq[jx] + meq[jy] + meq[jz], meq[jx] - meq[jy], meq[jx] - meq[jz]};
    const double s2s = sig[jx] + sig[jy] + sig[jz], s2d1 = sig[jx] - sig[jy], s2d2 = sig[jx] - sig[jz];
    const double nx = m[jx] - meq[jx] + 0.5 * sig[jx];
    const double ny = m[jy] - meq[jy] + 0.5 * sig[jy];
    const double nz = m[jz] - meq[jz] + 0.5 * sig[jz];
    double eq[3];
    corrected_equilibria(p, nx + ny + nz, nx - ny, nx - nz, rho, u, grad_rho, base, eq);
    const double t2s = c2s + wb * (eq[0] - c2s) + (1.0 - 0.5 * wb) * s2s;
    const double t2d1 = c2d1 + wn * (eq[1] - c2d1) + (1.0 - 0.5 * wn) * s2d1;
    const double t2d2 = c2d2 + wn * (eq[2] - c2d2) + (1.0 - 0.5 * wn) * s2d2;
    /* B^-1 */
    mt[jx] = (t2s + t2d1 + t2d2) / 3.0;
    mt[jy] = (t2s - 2.0 * t2d1 + t2d2) / 3.0;
    mt[jz] = (t2s + t2d1 - 2.0 * t2d2) / 3.0;
}

/* Central-moment equilibria matched to the Maxwellian (Eq. 9). */
static void central_equilibrium(double cs2, double rho, double keq[NQ])
{
    for (int j = 0; j < NQ; ++j) {
        double v = rho;
        int e[3] = {MM[j], MN[j], MP[j]};
        for (int i = 0; i < 3; ++i) {
            if (e[i] == 1) v = 0.0;
            else if (e[i] == 2) v *= cs2;
        }
        keq[j] = v;
    }
}

/* Hydrodynamic fields of one node (Eq. 12): rho = sum f, rho u = sum f e + F/2. */
static void node_moments(const or_params *p, const double f[NQ], const double F[3],
                         double *rho, double u[3])
{
    double m0 = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    for (int a = 0; a < NQ; ++a) {
        m0 += f[a];
        jx += f[a] * EX[a];
        jy += f[a] * (p->r * EY[a]);
        jz += f[a] * (p->s * EZ[a]);
    }
    *rho = m0;
    u[0] = (jx + 0.5 * F[0]) / m0;
    u[1] = (jy + 0.5 * F[1]) / m0;
    u[2] = (jz + 0.5 * F[2]) / m0;
}

/* Map post-collision central moments back to populations. */
static int central_to_populations(const or_params *p, const double u[3], const double kt[NQ],
                                  double ft[NQ])
{
    if (p->form == 1) {
        double M[NQ][NQ];
        central_M(p->r, p->s, u, M);
        return lu_solve27(M, kt, ft);
    }
    double Fm[NQ][NQ], S[NQ], mt[NQ], mu[3] = {-u[0], -u[1], -u[2]};
    frame_F(mu, Fm);                     /* F^-1 = F(-u), App. E */
    matvec27(Fm, kt, mt);
    scaling_S(p->r, p->s, S);            /* S^-1, App. F */
    for (int j = 0; j < NQ; ++j) mt[j] /= S[j];
    matvec27(g_Pinv, mt, ft);            /* P^-1, App. G */
    return 0;
}

/* One collision at one node.  F is the body force at the node, grad_rho the
 * density gradient (used by mode FULL only). */
static int collide_node(const or_params *p, const double f[NQ], const double F[3],
                        const double grad_rho[3], double ft[NQ])
{
    double rho, u[3], k[NQ], kt[NQ];
    node_moments(p, f, F, &rho, u);
    if (p->model == 1) {
        /* raw moments with the cuboid velocities, relaxed in place of central ones */
        double m[NQ], mt[NQ], S[NQ];
        const double zero[3] = {0.0, 0.0, 0.0};
        if (p->form == 1) {
            double M[NQ][NQ];
            central_M(p->r, p->s, zero, M);     /* Eq. 3b: moments about zero velocity */
            matvec27(M, f, m);
            relax_raw(p, m, rho, u, F, grad_rho, mt);
            return lu_solve27(M, mt, ft);
        }
        matvec27(g_P, f, m);                    /* m = S P f */
        scaling_S(p->r, p->s, S);
        for (int j = 0; j < NQ; ++j) m[j] *= S[j];
        relax_raw(p, m, rho, u, F, grad_rho, mt);
        for (int j = 0; j < NQ; ++j) mt[j] /= S[j];   /* f~ = P^-1 S^-1 m~ */
        matvec27(g_Pinv, mt, ft);
        return 0;
    }
    if (p->form == 1) {
        double M[NQ][NQ];
        central_M(p->r, p->s, u, M);     /* Eq. 3a */
        matvec27(M, f, k);
    } else {
        double m[NQ], S[NQ], Fm[NQ][NQ];
        matvec27(g_P, f, m);             /* m = P f, App. A */
        scaling_S(p->r, p->s, S);        /* m <- S m, App. B */
        for (int j = 0; j < NQ; ++j) m[j] *= S[j];
        frame_F(u, Fm);                  /* m^c = F(u) m, App. C */
        matvec27(Fm, m, k);
    }
    relax_central(p, k, rho, u, F, grad_rho, kt);
    return central_to_populations(p, u, kt, ft);
}

/* ------------------------------------------------------------------------ */
/* Whole-lattice operations.  Arrays are [27][nz][ny][nx], x fastest.          */

static size_t nodes(const or_params *p) { return (size_t)p->nx * p->ny * p->nz; }

static void node_force(const or_params *p, size_t x, double F[3])
{
    size_t N = nodes(p);
    for (int i = 0; i < 3; ++i) {
        F[i] = p->force[i];
        if (p->force_field) F[i] += p->force_field[i * N + x];
    }
}

/* Second-order central difference of the density along one axis; one-sided
 * second-order differences next to a wall; h is the grid spacing. */
static double diff_axis(const double *rho, size_t x, size_t stride, int i, int n, int wall, double h)
{
    if (n == 1) return 0.0;
    if (!wall) {
        size_t xp = (i == n - 1) ? x - (size_t)(n - 1) * stride : x + stride;
        size_t xm = (i == 0) ? x + (size_t)(n - 1) * stride : x - stride;
        return (rho[xp] - rho[xm]) / (2.0 * h);
    }
    if (n == 2) return (i == 0 ? rho[x + stride] - rho[x] : rho[x] - rho[x - stride]) / h;
    if (i == 0) return (-3.0 * rho[x] + 4.0 * rho[x + stride] - rho[x + 2 * stride]) / (2.0 * h);
    if (i == n - 1) return (3.0 * rho[x] - 4.0 * rho[x - stride] + rho[x - 2 * stride]) / (2.0 * h);
    return (rho[x + stride] - rho[x - stride]) / (2.0 * h);
}

int or_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Collide every node: ft[a][x] = post-collision population (Sec. 3.2). */
int or_collide_all(const or_params *p, const double *f, double *ft)
{
    setup();
    const size_t N = nodes(p);
    double *rho = NULL;
    int err = 0;
    if (p->corr == CORR_FULL) {
        rho = (double *)malloc(N * sizeof(double));
        if (!rho) return -2;
        for (size_t x = 0; x < N; ++x) {
            double v = 0.0;
            for (int a = 0; a < NQ; ++a) v += f[a * N + x];
            rho[x] = v;
        }
    }
#pragma omp parallel for schedule(static) reduction(| : err)
    for (long z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int xx = 0; xx < p->nx; ++xx) {
                size_t x = ((size_t)z * p->ny + y) * p->nx + xx;
                double fl[NQ], out[NQ], F[3], gr[3] = {0.0, 0.0, 0.0};
                for (int a = 0; a < NQ; ++a) fl[a] = f[a * N + x];
                node_force(p, x, F);
                if (rho) {
                    gr[0] = diff_axis(rho, x, 1, xx, p->nx, p->wall_mask & 1u, 1.0);
                    gr[1] = diff_axis(rho, x, (size_t)p->nx, y, p->ny, p->wall_mask & 2u, p->r);
                    gr[2] = diff_axis(rho, x, (size_t)p->nx * p->ny, (int)z, p->nz,
                                      p->wall_mask & 4u, p->s);
                }
                err |= collide_node(p, fl, F, gr, out) ? 1 : 0;
                for (int a = 0; a < NQ; ++a) ft[a * N + x] = out[a];
            }
    free(rho);
    return err ? -1 : 0;
}

/* Equilibrium populations f^eq(rho, u) = Q^-1 m^eq (Eq. 9, 10; Sec. 4). */
static int equilibrium_node(const or_params *p, double rho, const double u[3], double feq[NQ])
{
    double keq[NQ];
    central_equilibrium(p->cs2, rho, keq);
    return central_to_populations(p, u, keq, feq);
}

/* Streaming f_a(x, t+1) = ft_a(x - e_a, t) on the integer lattice (Sec. 3.2);
 * a link whose source lies beyond a wall returns as the reflected population
 * of the same node: f_a(x, t+1) = ft_opp(a)(x, t) - [f^eq_opp(a) - f^eq_a](x_w)
 * (Sec. 4, momentum-augmented bounce-back; the bracket vanishes at a wall at rest). */
int or_stream(const or_params *p, const double *ft, double *fout)
{
    setup();
    const size_t N = nodes(p);
    const int n[3] = {p->nx, p->ny, p->nz};
#pragma omp parallel for schedule(static)
    for (long z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int xx = 0; xx < p->nx; ++xx) {
                size_t x = ((size_t)z * p->ny + y) * p->nx + xx;
                int c[3] = {xx, y, (int)z};
                for (int a = 0; a < NQ; ++a) {
                    int e[3] = {EX[a], EY[a], EZ[a]}, src[3], out = 0, lid = 0;
                    for (int i = 0; i < 3; ++i) {
                        src[i] = c[i] - e[i];
                        if (src[i] < 0 || src[i] >= n[i]) {
                            if (p->wall_mask & (1u << i)) {
                                out = 1;
                                if (i == 1 && src[i] >= n[i]) lid = 1;
                            } else {
                                src[i] = (src[i] + n[i]) % n[i];
                            }
                        }
                    }
                    if (out) {
                        int b = g_OPP[a];
                        double v = ft[b * N + x];
                        if (lid && p->lid_u != 0.0) {
                            /* wall node density approximated by the fluid node's */
                            double rho = 0.0, uw[3] = {p->lid_u, 0.0, 0.0}, feq[NQ];
                            for (int q = 0; q < NQ; ++q) rho += ft[q * N + x];
                            equilibrium_node(p, rho, uw, feq);
                            v -= feq[b] - feq[a];
                        }
                        fout[a * N + x] = v;
                    } else {
                        size_t s = ((size_t)src[2] * p->ny + src[1]) * p->nx + src[0];
                        fout[a * N + x] = ft[a * N + s];
                    }
                }
            }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Reduced-precision storage emulation                                       */

/* Round x to the nearest value of a binary floating-point format with p
 * significand bits and minimum normal exponent emin, ties to even (IEEE 754
 * roundTiesToEven).  Around |x| in [2^e, 2^(e+1)) the format's values are
 * spaced 2^(e-p+1); below 2^emin (subnormals) the spacing stays 2^(emin-p+1).
 * Dividing by a power of two is exact, and rint() rounds ties to even in the
 * default rounding mode.  Results above the largest finite value become inf. */
static double round_format(double x, int p, int emin, double maxfinite)
{
    if (x == 0.0 || !isfinite(x)) return x;
    int e = ilogb(x);
    if (e < emin) e = emin;
    const double q = ldexp(1.0, e - (p - 1));
    const double r = rint(x / q) * q;
    return fabs(r) > maxfinite ? copysign(INFINITY, x) : r;
}

/* binary16: 11 significand bits, emin = -14, largest finite 65504. */
double or_round_binary16(double x) { return round_format(x, 11, -14, 65504.0); }

/* bfloat16: 8 significand bits, emin = -126, largest finite (2 - 2^-7) 2^127. */
double or_round_bfloat16(double x) { return round_format(x, 8, -126, ldexp(255.0, 120)); }

/* f_a := w_a + round(f_a - w_a) at every node, per p->storage_emulation. */
int or_quantize(const or_params *p, double *f)
{
    if (!p->storage_emulation) return 0;
    if (p->storage_emulation != 1 && p->storage_emulation != 2) return -1;
    const size_t N = nodes(p);
    const double zero[3] = {0.0, 0.0, 0.0};
    double w[NQ];
    if (equilibrium_node(p, 1.0, zero, w)) return -1;
    for (int a = 0; a < NQ; ++a) {
        const double sc = ldexp(1.0, 10 - ilogb(w[a]));
        double *fa = f + a * N;
#pragma omp parallel for schedule(static)
        for (long x = 0; x < (long)N; ++x) {
            const double g = fa[x] - w[a];
            const double q = p->storage_emulation == 1 ? or_round_binary16(g * sc) / sc : or_round_bfloat16(g);
            fa[x] = w[a] + q;
        }
    }
    return 0;
}

/* One full time step: collide then stream.  f and fout must not alias. */
int or_step(const or_params *p, const double *f, double *fout)
{
    const size_t N = nodes(p);
    double *ft = (double *)malloc(NQ * N * sizeof(double));
    if (!ft) return -2;
    int err = or_collide_all(p, f, ft);
    if (!err) err = or_quantize(p, ft);       /* the store keeps the rounded post-collision state */
    if (!err) err = or_stream(p, ft, fout);
    free(ft);
    return err;
}

int or_run(const or_params *p, double *f, int steps)
{
    const size_t N = nodes(p);
    double *g = (double *)malloc(NQ * N * sizeof(double));
    if (!g) return -2;
    int err = 0;
    for (int t = 0; t < steps && !err; ++t) {
        err = or_step(p, f, g);
        memcpy(f, g, NQ * N * sizeof(double));
    }
    free(g);
    return err;
}

/* f := f^eq(rho(x), u(x)) at every node. */
int or_init(const or_params *p, const double *rho, const double *u, double *f)
{
    setup();
    const size_t N = nodes(p);
    int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
    for (long x = 0; x < (long)N; ++x) {
        double uu[3] = {u[x], u[N + x], u[2 * N + x]}, feq[NQ];
        err |= equilibrium_node(p, rho[x], uu, feq) ? 1 : 0;
        for (int a = 0; a < NQ; ++a) f[a * N + x] = feq[a];
    }
    return err ? -1 : or_quantize(p, f);
}

/* rho(x) and u(x) (including the F/2 shift) of every node (Eq. 12). */
int or_moments(const or_params *p, const double *f, double *rho, double *u)
{
    setup();
    const size_t N = nodes(p);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < (long)N; ++x) {
        double fl[NQ], F[3], rr, uu[3];
        for (int a = 0; a < NQ; ++a) fl[a] = f[a * N + x];
        node_force(p, (size_t)x, F);
        node_moments(p, fl, F, &rr, uu);
        rho[x] = rr;
        u[x] = uu[0]; u[N + x] = uu[1]; u[2 * N + x] = uu[2];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Single-node entry points and matrices, for the tests                      */

int or_collide_node(const or_params *p, const double *f, const double *F, const double *grad_rho,
                    double *ft)
{
    setup();
    return collide_node(p, f, F, grad_rho, ft);
}

int or_equilibrium(const or_params *p, double rho, const double *u, double *feq)
{
    setup();
    return equilibrium_node(p, rho, u, feq);
}

/* Post-collision central moments for given pre-collision central moments. */
void or_relax_central(const or_params *p, const double *k, double rho, const double *u,
                      const double *F, const double *grad_rho, double *kt)
{
    setup();
    relax_central(p, k, rho, u, F, grad_rho, kt);
}

void or_strain_rates(const or_params *p, const double *k, double rho, const double *u,
                     const double *grad_rho, int aliasing, double *d)
{
    setup();
    strain_rates(p, k, rho, u, grad_rho, aliasing ? 1.0 : 0.0, d);
}

void or_matrix_P(double *out) { setup(); memcpy(out, g_P, sizeof(g_P)); }
void or_matrix_Pinv(double *out) { setup(); memcpy(out, g_Pinv, sizeof(g_Pinv)); }
void or_matrix_S(double r, double s, double *out) { scaling_S(r, s, out); }
void or_matrix_F(const double *u, double *out) { frame_F(u, (double (*)[NQ])out); }
void or_matrix_M(double r, double s, const double *u, double *out)
{
    central_M(r, s, u, (double (*)[NQ])out);
}
void or_velocities(int *ex, int *ey, int *ez)
{
    memcpy(ex, EX, sizeof(EX)); memcpy(ey, EY, sizeof(EY)); memcpy(ez, EZ, sizeof(EZ));
}
void or_moment_exponents(int *m, int *n, int *p)
{
    memcpy(m, MM, sizeof(MM)); memcpy(n, MN, sizeof(MN)); memcpy(p, MP, sizeof(MP));
}
void or_central_equilibrium(double cs2, double rho, double *keq) { central_equilibrium(cs2, rho, keq); }
void or_raw_equilibrium(double cs2, double rho, const double *u, double *meq) { setup(); raw_equilibrium(cs2, rho, u, meq); }
