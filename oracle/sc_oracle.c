/*
 * Two-component Shan-Chen lattice Boltzmann step -- plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark load this library.  It shares no
 * code, header, table or constant with the CUDA path: the velocity set is
 * built here by enumeration (in a different order from the GPU tables), the
 * populations are stored node-major (array of structures) and streaming is
 * done by pushing, where the GPU path pulls.
 *
 * What it computes, step by step, in the paper's order (Sec. 2.1):
 *   densities      rho_s = sum_i f_is                               (Sec. 2.1, moments)
 *   common velocity u' = sum_s (1/tau_s) sum_i f_is c_i
 *                        / sum_s rho_s / tau_s                       (Sec. 2.1, moments)
 *   force          F_s(x) = -G rho_s(x) sum_i w_i rho_s'(x + c_i) c_i (Eq. FORCE)
 *                  plus, when A != 0, the Kolmogorov body force of Eq. kolmo
 *                  (Sec. 4.2), F_x = rho A sin(2 pi y / L_y), shared between
 *                  the species in proportion to their densities:
 *                  F_s,x(x) += rho_s(x) A sin(2 pi y / L_y)
 *   collision      f*_is = f_is - (f_is - f^eq_is(rho_s, u' + tau_s F_s / rho_s)) / tau_s
 *                                                                   (Eq. eq:be, dt = 1)
 *   streaming      f_is(x + c_i, t + 1) = f*_is(x), periodic box    (Eq. eq:be; Sec. 4)
 * Alternative forcing (forcing = 1): the discrete-forcing cure of Guo, Zheng
 * and Shi that Sec. 2.3 names as the way to remove the tau-dependent coupling
 * g_tau (the paper gives no formulas; the standard form, for each species):
 *   u_G  = sum_s (j_s + F_s / 2) / tau_s / sum_s rho_s / tau_s
 *   f*_is = f_is - (f_is - f^eq_is(rho_s, u_G)) / tau_s
 *           + (1 - 1 / (2 tau_s)) w_i [(c_i - u_G) / cs2 + (c_i.u_G) c_i / cs2^2] . F_s
 * (u_G is the barycentric velocity for equal tau_s; the 1/tau_s weights make
 * the collision add exactly sum_s F_s to the momentum for any tau_s.)
 * The equilibrium is the Maxwellian truncated at second order in u, which
 * the paper names without printing (Sec. 2.1):
 *   f^eq_i(rho, u) = w_i rho [1 + c.u / cs2 + (c.u)^2 / (2 cs2^2) - u.u / (2 cs2)],
 * cs2 = 1/3, with weights that satisfy the isotropy sums of Sec. 2.1.
 * Reported fields (Sec. 2.3, momentum shifted by F dt / 2):
 *   u_phys = (sum_s j_s + (1/2) sum_s F_s) / (rho_A + rho_B)
 *   p      = cs2 (rho_A + rho_B) + cs2 G rho_A rho_B   (bulk part of the SC
 *                                                       pressure tensor, Sec. 2.1)
 *
 * Parity status: every function here is pinned by the CPU tests (lattice
 * sums in exact rationals, equilibrium moments, conservation laws, exact
 * rational one-step trace, shear-wave and diffusion decay rates, the paper's
 * linear spinodal rate, the paper's coexistence example, Laplace's law; the
 * body force by an exact rational trace with the force, the closed-form
 * first step of a forced uniform fluid and the steady Kolmogorov profile).
 *
 * Node index n = x + nx * (y + ny * z).  Populations: f[(n * 2 + s) * Q + i].
 * Built with -O2 -ffp-contract=off so no fused multiply-add changes rounding;
 * the OpenMP loops run over independent nodes, so results do not depend on
 * the thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXQ 19

typedef struct {
    int lattice;      /* 0: D2Q9 (nz must be 1), 1: D3Q19 */
    int nx, ny, nz;
    double tau_A, tau_B;
    double G;         /* coupling G_AB = G_BA, one value (Eq. FORCE) */
    double body_A;    /* amplitude A of the Kolmogorov force (Eq. kolmo); 0 = none */
    int body_y0;      /* global y of row 0 (a window cut from a larger lattice) */
    int body_ly;      /* period L_y of the forcing; 0 = ny */
    int forcing;      /* 0: velocity shift of Sec. 2.1; 1: Guo et al. source term (Sec. 2.3) */
} oracle_params;

typedef struct {
    int q;
    int c[MAXQ][3];
    double w[MAXQ];
} velocity_set;

/* Velocity set by enumeration of {-1,0,1}^d in z-major, then y, then x
 * order, keeping |c|^2 <= 2 in 3D.  Weights by speed shell: D2Q9 4/9, 1/9,
 * 1/36; D3Q19 1/3, 1/18, 1/36.  Both satisfy the second- and fourth-order
 * isotropy conditions of Sec. 2.1 with cs2 = 1/3 (pinned in the tests). */
static void make_velocity_set(int lattice, velocity_set* vs)
{
    int zr = (lattice == 1) ? 1 : 0;
    int q = 0;
    for (int cz = -zr; cz <= zr; ++cz)
        for (int cy = -1; cy <= 1; ++cy)
            for (int cx = -1; cx <= 1; ++cx) {
                int n2 = cx * cx + cy * cy + cz * cz;
                if (n2 == 3) continue;
                vs->c[q][0] = cx;
                vs->c[q][1] = cy;
                vs->c[q][2] = cz;
                if (lattice == 0)
                    vs->w[q] = (n2 == 0) ? 4.0 / 9.0 : (n2 == 1) ? 1.0 / 9.0 : 1.0 / 36.0;
                else
                    vs->w[q] = (n2 == 0) ? 1.0 / 3.0 : (n2 == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
                ++q;
            }
    vs->q = q;
}

static const double CS2 = 1.0 / 3.0;

static long wrap(long a, long n)
{
    long r = a % n;
    return r < 0 ? r + n : r;
}

/* Index of the node at x + c (periodic). */
static long neighbour(const oracle_params* p, long n, const int c[3])
{
    long nx = p->nx, ny = p->ny, nz = p->nz;
    long x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
    return wrap(x + c[0], nx) + nx * (wrap(y + c[1], ny) + ny * wrap(z + c[2], nz));
}

static void equilibrium(const velocity_set* vs, double rho, const double u[3], double* feq)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < vs->q; ++i) {
        double cu = vs->c[i][0] * u[0] + vs->c[i][1] * u[1] + vs->c[i][2] * u[2];
        feq[i] = vs->w[i] * rho * (1.0 + cu / CS2 + (cu * cu) / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

static int check_params(const oracle_params* p)
{
    if (p->lattice != 0 && p->lattice != 1) return -1;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return -1;
    if (p->lattice == 0 && p->nz != 1) return -1;
    if (!(p->tau_A > 0.5) || !(p->tau_B > 0.5)) return -1;
    if (p->body_ly < 0) return -1;
    if (p->forcing != 0 && p->forcing != 1) return -1;
    return 0;
}

/* ---- public functions (called through ctypes) ---------------------------- */

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Copy the velocity set out: c as q x 3 ints, w as q doubles.  Returns q. */
int oracle_lattice(int lattice, int* c, double* w)
{
    velocity_set vs;
    make_velocity_set(lattice, &vs);
    for (int i = 0; i < vs.q; ++i) {
        for (int a = 0; a < 3; ++a) c[i * 3 + a] = vs.c[i][a];
        w[i] = vs.w[i];
    }
    return vs.q;
}

/* Equilibrium of one node (second-order truncated Maxwellian, Sec. 2.1). */
int oracle_equilibrium(int lattice, double rho, const double* u3, double* feq)
{
    velocity_set vs;
    make_velocity_set(lattice, &vs);
    equilibrium(&vs, rho, u3, feq);
    return vs.q;
}

/* f_is(x, 0) = f^eq(rho_s(x), u(x)); u is N x 3 or NULL for rest. */
int oracle_init(const oracle_params* p, const double* rhoA, const double* rhoB,
                const double* u, double* f)
{
    if (check_params(p)) return -1;
    velocity_set vs;
    make_velocity_set(p->lattice, &vs);
    const int Q = vs.q;
    const long N = (long)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        double u3[3] = {0.0, 0.0, 0.0};
        if (u) { u3[0] = u[n * 3 + 0]; u3[1] = u[n * 3 + 1]; u3[2] = u[n * 3 + 2]; }
        equilibrium(&vs, rhoA[n], u3, f + (n * 2 + 0) * Q);
        equilibrium(&vs, rhoB[n], u3, f + (n * 2 + 1) * Q);
    }
    return 0;
}

/* Densities rho[s][n] and momenta j[s][n][3] of the current populations. */
static void compute_moments(const oracle_params* p, const velocity_set* vs, const double* f,
                            double* rho, double* j)
{
    const int Q = vs->q;
    const long N = (long)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n)
        for (int s = 0; s < 2; ++s) {
            const double* fn = f + (n * 2 + s) * Q;
            double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
            for (int i = 0; i < Q; ++i) {
                r += fn[i];
                jx += fn[i] * vs->c[i][0];
                jy += fn[i] * vs->c[i][1];
                jz += fn[i] * vs->c[i][2];
            }
            rho[s * N + n] = r;
            j[(s * N + n) * 3 + 0] = jx;
            j[(s * N + n) * 3 + 1] = jy;
            j[(s * N + n) * 3 + 2] = jz;
        }
}

/* F_s(x) = -G rho_s(x) sum_i w_i rho_s'(x + c_i) c_i, s' the other species (Eq. FORCE),
 * plus rho_s(x) A sin(2 pi y / L_y) along x (Eq. kolmo). */
static void compute_force(const oracle_params* p, const velocity_set* vs, const double* rho,
                          double* F)
{
    const int Q = vs->q;
    const long N = (long)p->nx * p->ny * p->nz;
    const double two_pi = 2.0 * acos(-1.0);
    const double ly = p->body_ly > 0 ? (double)p->body_ly : (double)p->ny;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n)
        for (int s = 0; s < 2; ++s) {
            const double* rho_other = rho + (1 - s) * N;
            double sum[3] = {0.0, 0.0, 0.0};
            for (int i = 0; i < Q; ++i) {
                double r = rho_other[neighbour(p, n, vs->c[i])];
                for (int a = 0; a < 3; ++a) sum[a] += vs->w[i] * r * vs->c[i][a];
            }
            for (int a = 0; a < 3; ++a) F[(s * N + n) * 3 + a] = -p->G * rho[s * N + n] * sum[a];
            if (p->body_A != 0.0) {
                const long y = (n / p->nx) % p->ny + p->body_y0;
                F[(s * N + n) * 3 + 0] += rho[s * N + n] * p->body_A * sin(two_pi * (double)y / ly);
            }
        }
}

/* nsteps of collide-then-push-stream; f is updated in place (f_tmp is work space of
 * the same size as f). */
int oracle_step(const oracle_params* p, double* f, double* f_tmp, int nsteps)
{
    if (check_params(p) || nsteps < 0) return -1;
    velocity_set vs;
    make_velocity_set(p->lattice, &vs);
    const int Q = vs.q;
    const long N = (long)p->nx * p->ny * p->nz;
    const double tau[2] = {p->tau_A, p->tau_B};
    double* rho = (double*)malloc(sizeof(double) * 2 * N);
    double* j = (double*)malloc(sizeof(double) * 2 * N * 3);
    double* F = (double*)malloc(sizeof(double) * 2 * N * 3);
    if (!rho || !j || !F) { free(rho); free(j); free(F); return -2; }

    for (int t = 0; t < nsteps; ++t) {
        compute_moments(p, &vs, f, rho, j);
        compute_force(p, &vs, rho, F);
#pragma omp parallel for schedule(static)
        for (long n = 0; n < N; ++n) {
            /* common velocity u' (Sec. 2.1) */
            double num[3] = {0.0, 0.0, 0.0}, den = 0.0;
            for (int s = 0; s < 2; ++s) {
                for (int a = 0; a < 3; ++a) num[a] += j[(s * N + n) * 3 + a] / tau[s];
                den += rho[s * N + n] / tau[s];
            }
            if (p->forcing == 1) {
                /* Guo forcing: f^eq at u_G, plus the discrete source term */
                double uG[3];
                for (int a = 0; a < 3; ++a) {
                    double m = 0.0;
                    for (int s = 0; s < 2; ++s)
                        m += (j[(s * N + n) * 3 + a] + 0.5 * F[(s * N + n) * 3 + a]) / tau[s];
                    uG[a] = m / den;
                }
                for (int s = 0; s < 2; ++s) {
                    double feq[MAXQ];
                    equilibrium(&vs, rho[s * N + n], uG, feq);
                    const double* Fs = F + (s * N + n) * 3;
                    const double* fn = f + (n * 2 + s) * Q;
                    for (int i = 0; i < Q; ++i) {
                        double cu = 0.0, src = 0.0;
                        for (int a = 0; a < 3; ++a) cu += vs.c[i][a] * uG[a];
                        for (int a = 0; a < 3; ++a)
                            src += ((vs.c[i][a] - uG[a]) / CS2 + cu * vs.c[i][a] / (CS2 * CS2)) * Fs[a];
                        double post = fn[i] - (fn[i] - feq[i]) / tau[s] + (1.0 - 0.5 / tau[s]) * vs.w[i] * src;
                        long m = neighbour(p, n, vs.c[i]);
                        f_tmp[(m * 2 + s) * Q + i] = post;
                    }
                }
                continue;
            }
            for (int s = 0; s < 2; ++s) {
                double r = rho[s * N + n];
                double ueq[3], feq[MAXQ];
                for (int a = 0; a < 3; ++a)
                    ueq[a] = num[a] / den + tau[s] * F[(s * N + n) * 3 + a] / r;
                equilibrium(&vs, r, ueq, feq);
                const double* fn = f + (n * 2 + s) * Q;
                for (int i = 0; i < Q; ++i) {
                    double post = fn[i] - (fn[i] - feq[i]) / tau[s];
                    long m = neighbour(p, n, vs.c[i]);
                    f_tmp[(m * 2 + s) * Q + i] = post;
                }
            }
        }
        memcpy(f, f_tmp, sizeof(double) * 2 * N * Q);
    }
    free(rho);
    free(j);
    free(F);
    return 0;
}

/* Macroscopic fields of the current populations: rho_A, rho_B (N each),
 * u_phys (N x 3) and bulk pressure p (N).  Any output may be NULL. */
int oracle_moments(const oracle_params* p, const double* f, double* rhoA, double* rhoB,
                   double* u, double* pres)
{
    if (check_params(p)) return -1;
    velocity_set vs;
    make_velocity_set(p->lattice, &vs);
    const long N = (long)p->nx * p->ny * p->nz;
    double* rho = (double*)malloc(sizeof(double) * 2 * N);
    double* j = (double*)malloc(sizeof(double) * 2 * N * 3);
    double* F = (double*)malloc(sizeof(double) * 2 * N * 3);
    if (!rho || !j || !F) { free(rho); free(j); free(F); return -2; }
    compute_moments(p, &vs, f, rho, j);
    compute_force(p, &vs, rho, F);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        double ra = rho[n], rb = rho[N + n];
        if (rhoA) rhoA[n] = ra;
        if (rhoB) rhoB[n] = rb;
        if (u)
            for (int a = 0; a < 3; ++a)
                u[n * 3 + a] = (j[n * 3 + a] + j[(N + n) * 3 + a]
                                + 0.5 * (F[n * 3 + a] + F[(N + n) * 3 + a])) / (ra + rb);
        if (pres) pres[n] = CS2 * (ra + rb) + CS2 * p->G * ra * rb;
    }
    free(rho);
    free(j);
    free(F);
    return 0;
}

/* Total momentum sum_x sum_s j_s of the current populations (3 doubles). */
int oracle_total_momentum(const oracle_params* p, const double* f, double* out3)
{
    if (check_params(p)) return -1;
    velocity_set vs;
    make_velocity_set(p->lattice, &vs);
    const int Q = vs.q;
    const long N = (long)p->nx * p->ny * p->nz;
    double m[3] = {0.0, 0.0, 0.0};
    for (long n = 0; n < N; ++n)
        for (int s = 0; s < 2; ++s)
            for (int i = 0; i < Q; ++i)
                for (int a = 0; a < 3; ++a) m[a] += f[(n * 2 + s) * Q + i] * vs.c[i][a];
    for (int a = 0; a < 3; ++a) out3[a] = m[a];
    return 0;
}

/* ==== Free-energy (FE) two-population model, Sec. 2.2 ======================
 *
 * Populations f_i (density and momentum) and g_i (order parameter), stored like
 * the two SC species: f[(n * 2 + 0) * Q + i] = f_i, f[(n * 2 + 1) * Q + i] = g_i.
 *   rho = sum_i f_i, u = sum_i f_i c_i / rho, phi = sum_i g_i       (Sec. 2.2)
 *   f_i(x + c_i, t + 1) = f_i - (f_i - f_i^eq) / tau                 (Eq. FE1)
 *   g_i(x + c_i, t + 1) = g_i - (g_i - g_i^eq) / tau_g               (Eq. FE2)
 * Free energy: the tau-dependent SC-matching functional of Eq. FEtau with
 * coupling g (pass g_tau to match an SC run), bulk density
 *   V(phi, rho) = cs2 (rho+phi)/2 ln((rho+phi)/2) + cs2 (rho-phi)/2 ln((rho-phi)/2)
 *                 + g cs2 (rho^2 - phi^2)/4,
 * gradient coefficient kappa (g cs2^2 / 4 in Eq. FEtau), so that
 *   mu  = dV/dphi - kappa lap(phi) = cs2/2 ln((rho+phi)/(rho-phi)) - g cs2 phi/2 - kappa lap(phi)
 *   P   = (p_b - kappa phi lap(phi) - kappa/2 |grad phi|^2) delta + kappa grad(phi) grad(phi),
 *   p_b = phi dV/dphi + rho dV/drho - V = cs2 rho + g cs2 (rho^2 - phi^2)/4   (Sec. 2.2)
 * The equilibria are the second-order Hermite forms that meet the moment
 * conditions of Eq. EQFE1 and Eq. EQFE2 exactly (the paper states only the
 * conditions):
 *   f_i^eq = w_i [rho + rho c.u / cs2 + (c_a c_b - cs2 d_ab)(P_ab - rho cs2 d_ab + rho u_a u_b) / (2 cs2^2)]
 *   g_i^eq = w_i [phi + phi c.u / cs2 + (c_a c_b - cs2 d_ab)((Gamma mu - phi cs2) d_ab + phi u_a u_b) / (2 cs2^2)]
 * Derivatives by the isotropic lattice stencils
 *   grad(phi) = (1/cs2) sum_i w_i c_i phi(x + c_i),  lap(phi) = (2/cs2) sum_i w_i (phi(x + c_i) - phi(x)).
 * Reported fields: rho_A = (rho + phi)/2, rho_B = (rho - phi)/2 (phi = rho_A - rho_B,
 * Sec. 2.1), u = sum_i f_i c_i / rho, p = p_b.
 */
typedef struct {
    int lattice;
    int nx, ny, nz;
    double tau, tau_g;  /* relaxation times of f and g (Eqs. FE1, FE2) */
    double g;           /* coupling of the functional */
    double kappa;       /* gradient coefficient */
    double gamma;       /* Gamma of Eq. EQFE2: mobility M = Gamma (tau_g - 1/2) */
} fe_params;

static int fe_check(const fe_params* p)
{
    if (p->lattice != 0 && p->lattice != 1) return -1;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return -1;
    if (p->lattice == 0 && p->nz != 1) return -1;
    if (!(p->tau > 0.5) || !(p->tau_g > 0.5)) return -1;
    return 0;
}

static long fe_neighbour(const fe_params* p, long n, const int c[3])
{
    long nx = p->nx, ny = p->ny, nz = p->nz;
    long x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
    return wrap(x + c[0], nx) + nx * (wrap(y + c[1], ny) + ny * wrap(z + c[2], nz));
}

/* Equilibria of one node from rho, phi, u (3), grad phi (3), lap phi. */
static void fe_equilibria(const velocity_set* vs, int D, double g, double kappa, double gamma, double rho,
                          double phi, const double u[3], const double gp[3], double lp, double* feq, double* geq)
{
    const double mu = 0.5 * CS2 * log((rho + phi) / (rho - phi)) - 0.5 * g * CS2 * phi - kappa * lp;
    const double pb = CS2 * rho + 0.25 * g * CS2 * (rho * rho - phi * phi);
    const double gg = gp[0] * gp[0] + gp[1] * gp[1] + gp[2] * gp[2];
    double Mf[3][3], Mg[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const double d = (a == b) ? 1.0 : 0.0;
            const double P = (pb - kappa * phi * lp - 0.5 * kappa * gg) * d + kappa * gp[a] * gp[b];
            Mf[a][b] = P - rho * CS2 * d + rho * u[a] * u[b];
            Mg[a][b] = (gamma * mu - phi * CS2) * d + phi * u[a] * u[b];
        }
    for (int i = 0; i < vs->q; ++i) {
        double cu = 0.0, hf = 0.0, hg = 0.0;
        for (int a = 0; a < D; ++a) cu += vs->c[i][a] * u[a];
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) {
                const double h = vs->c[i][a] * vs->c[i][b] - ((a == b) ? CS2 : 0.0);
                hf += h * Mf[a][b];
                hg += h * Mg[a][b];
            }
        feq[i] = vs->w[i] * (rho + rho * cu / CS2 + hf / (2.0 * CS2 * CS2));
        geq[i] = vs->w[i] * (phi + phi * cu / CS2 + hg / (2.0 * CS2 * CS2));
    }
}

/* Both equilibria of one node (for the moment pins of Eqs. EQFE1, EQFE2). */
int oracle_fe_equilibria(int lattice, double g, double kappa, double gamma, double rho, double phi,
                         const double* u3, const double* gp3, double lp, double* feq, double* geq)
{
    velocity_set vs;
    make_velocity_set(lattice, &vs);
    fe_equilibria(&vs, lattice == 0 ? 2 : 3, g, kappa, gamma, rho, phi, u3, gp3, lp, feq, geq);
    return vs.q;
}

/* The t = 0 state from rho_A, rho_B: f_i = w_i rho, g_i = w_i phi with rho = rho_A + rho_B,
 * phi = rho_A - rho_B (the rest populations; the first collision relaxes them to the
 * equilibria above). */
int oracle_fe_init(const fe_params* p, const double* rhoA, const double* rhoB, double* f)
{
    if (fe_check(p)) return -1;
    velocity_set vs;
    make_velocity_set(p->lattice, &vs);
    const int Q = vs.q;
    const long N = (long)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n)
        for (int i = 0; i < Q; ++i) {
            f[(n * 2 + 0) * Q + i] = vs.w[i] * (rhoA[n] + rhoB[n]);
            f[(n * 2 + 1) * Q + i] = vs.w[i] * (rhoA[n] - rhoB[n]);
        }
    return 0;
}

/* rho, phi, u (N x 3), grad phi (N x 3) and lap phi of the current populations. */
static void fe_fields(const fe_params* p, const velocity_set* vs, const double* f, double* rho, double* phi,
                      double* u, double* gp, double* lp)
{
    const int Q = vs->q;
    const long N = (long)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        double r = 0.0, ph = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; ++i) {
            const double fi = f[(n * 2 + 0) * Q + i];
            r += fi;
            ph += f[(n * 2 + 1) * Q + i];
            for (int a = 0; a < 3; ++a) j[a] += fi * vs->c[i][a];
        }
        rho[n] = r;
        phi[n] = ph;
        for (int a = 0; a < 3; ++a) u[n * 3 + a] = j[a] / r;
    }
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        double g3[3] = {0.0, 0.0, 0.0}, l = 0.0;
        for (int i = 0; i < Q; ++i) {
            const double pn = phi[fe_neighbour(p, n, vs->c[i])];
            for (int a = 0; a < 3; ++a) g3[a] += vs->w[i] * vs->c[i][a] * pn;
            l += vs->w[i] * (pn - phi[n]);
        }
        for (int a = 0; a < 3; ++a) gp[n * 3 + a] = g3[a] / CS2;
        lp[n] = 2.0 * l / CS2;
    }
}

/* nsteps of collide-then-push-stream of Eqs. FE1, FE2. */
int oracle_fe_step(const fe_params* p, double* f, double* f_tmp, int nsteps)
{
    if (fe_check(p) || nsteps < 0) return -1;
    velocity_set vs;
    make_velocity_set(p->lattice, &vs);
    const int Q = vs.q, D = p->lattice == 0 ? 2 : 3;
    const long N = (long)p->nx * p->ny * p->nz;
    double* rho = (double*)malloc(sizeof(double) * N);
    double* phi = (double*)malloc(sizeof(double) * N);
    double* u = (double*)malloc(sizeof(double) * N * 3);
    double* gp = (double*)malloc(sizeof(double) * N * 3);
    double* lp = (double*)malloc(sizeof(double) * N);
    if (!rho || !phi || !u || !gp || !lp) { free(rho); free(phi); free(u); free(gp); free(lp); return -2; }
    const double tau[2] = {p->tau, p->tau_g};
    for (int t = 0; t < nsteps; ++t) {
        fe_fields(p, &vs, f, rho, phi, u, gp, lp);
#pragma omp parallel for schedule(static)
        for (long n = 0; n < N; ++n) {
            double eq[2][MAXQ];
            fe_equilibria(&vs, D, p->g, p->kappa, p->gamma, rho[n], phi[n], u + n * 3, gp + n * 3, lp[n], eq[0],
                          eq[1]);
            for (int s = 0; s < 2; ++s)
                for (int i = 0; i < Q; ++i) {
                    const double fi = f[(n * 2 + s) * Q + i];
                    f_tmp[(fe_neighbour(p, n, vs.c[i]) * 2 + s) * Q + i] = fi - (fi - eq[s][i]) / tau[s];
                }
        }
        memcpy(f, f_tmp, sizeof(double) * 2 * N * Q);
    }
    free(rho); free(phi); free(u); free(gp); free(lp);
    return 0;
}

/* rho_A = (rho + phi)/2, rho_B = (rho - phi)/2, u (N x 3), p_b; any output may be NULL. */
int oracle_fe_moments(const fe_params* p, const double* f, double* rhoA, double* rhoB, double* u, double* pres)
{
    if (fe_check(p)) return -1;
    velocity_set vs;
    make_velocity_set(p->lattice, &vs);
    const long N = (long)p->nx * p->ny * p->nz;
    double* rho = (double*)malloc(sizeof(double) * N);
    double* phi = (double*)malloc(sizeof(double) * N);
    double* uu = (double*)malloc(sizeof(double) * N * 3);
    double* gp = (double*)malloc(sizeof(double) * N * 3);
    double* lp = (double*)malloc(sizeof(double) * N);
    if (!rho || !phi || !uu || !gp || !lp) { free(rho); free(phi); free(uu); free(gp); free(lp); return -2; }
    fe_fields(p, &vs, f, rho, phi, uu, gp, lp);
    for (long n = 0; n < N; ++n) {
        if (rhoA) rhoA[n] = 0.5 * (rho[n] + phi[n]);
        if (rhoB) rhoB[n] = 0.5 * (rho[n] - phi[n]);
        if (u) for (int a = 0; a < 3; ++a) u[n * 3 + a] = uu[n * 3 + a];
        if (pres) pres[n] = CS2 * rho[n] + 0.25 * p->g * CS2 * (rho[n] * rho[n] - phi[n] * phi[n]);
    }
    free(rho); free(phi); free(uu); free(gp); free(lp);
    return 0;
}

/* rho, phi (N each), u, grad phi (N x 3 each) and lap phi (N) of the current populations. */
int oracle_fe_fields(const fe_params* p, const double* f, double* rho, double* phi, double* u, double* gp,
                     double* lp)
{
    if (fe_check(p)) return -1;
    velocity_set vs;
    make_velocity_set(p->lattice, &vs);
    fe_fields(p, &vs, f, rho, phi, u, gp, lp);
    return 0;
}
