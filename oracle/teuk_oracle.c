/*
 * teuk_oracle.c -- plain FP64 CPU oracle for the Teukolsky time step.
 *
 * TEST INFRASTRUCTURE: see teuk_oracle.h.  Only tests/, the smoke entry and
 * the bench's CPU legs may use this file.  It is deliberately slow and
 * plain: every coefficient is recomputed from its defining formula at every
 * point of every step, and every loop follows the order of the equation it
 * implements.  The only concession to speed is an OpenMP loop over r* rows
 * (the paper's own CPU code was OpenMP-parallel, Sec. 5.2).
 *
 * Paper: G. Khanna & J. McKennon, arXiv:0909.4039.
 *   Eq. 1            Teukolsky master equation (Boyer-Lindquist)
 *   Eqs. 2-3         tortoise coordinate r*, azimuthal coordinate phi~
 *   Eq. 4            mode ansatz Psi = e^{i m phi~} r^3 Phi
 *   Eqs. 5-7         Pi, b, Sigma^2
 *   Eqs. 8-12        first-order system; D/S split
 *   Eqs. 13-14       two-step Lax-Wendroff
 *   Sec. 2.2 (end)   centred angular differences, boundary conditions
 */
#include "teuk_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define OR_PI 3.14159265358979323846

/* ---------------------------------------------------------------- grid -- */

static void horizons(double M, double a, double *rp, double *rm)
{
    double d = sqrt(M * M - a * a);
    *rp = M + d;
    *rm = M - d;
}

static double drs_of(const or_grid *g)
{
    return (g->rs_max - g->rs_min) / (double)(g->Nr - 1);
}

static double dth_of(const or_grid *g) { return OR_PI / (double)g->Nth; }

static double theta_of(const or_grid *g, long j)
{
    return ((double)j + 0.5) * dth_of(g);
}

/* Parity of the angular ghost cells (Sec. 2.2, last paragraph): even |m|
 * has d Phi/d theta = 0 at the poles (symmetric ghost), odd |m| has Phi = 0
 * at the poles (antisymmetric ghost). */
static double ghost_parity(const or_grid *g)
{
    return (abs(g->m) % 2 == 0) ? 1.0 : -1.0;
}

/* ------------------------------------------------------ tortoise map ---- */

/* Eq. 2, dr* = (r^2+a^2)/Delta dr, integrated with partial fractions:
 *   r* = r + 2M r+/(r+ - r-) ln((r - r+)/2M) - 2M r-/(r+ - r-) ln((r - r-)/2M)
 * written in x = r - r+ so that Delta = x (x + r+ - r-) carries no
 * cancellation near the horizon. */
double or_rstar_of_x(double M, double a, double x)
{
    double rp, rm;
    horizons(M, a, &rp, &rm);
    double kp = 2.0 * M * rp / (rp - rm);
    double km = 2.0 * M * rm / (rp - rm);
    return rp + x + kp * log(x / (2.0 * M)) - km * log((x + rp - rm) / (2.0 * M));
}

/* Inverse of or_rstar_of_x by Newton's method on xi = ln x, kept inside a
 * bisection bracket.  The derivative of r* in xi is x (r^2+a^2)/Delta = (r^2+a^2)/(x+r+-r-). */
int or_x_of_rstar(double M, double a, double rs, double *x_out)
{
    double rp, rm;
    horizons(M, a, &rp, &rm);
    if (!(rp > rm)) return -1;
    double lo = -700.0, hi = 60.0;
    if (or_rstar_of_x(M, a, exp(lo)) > rs) return -2;
    if (or_rstar_of_x(M, a, exp(hi)) < rs) return -3;
    double kp = 2.0 * M * rp / (rp - rm);
    double xi = (rs > rp + 4.0 * M) ? log(rs) : (rs - rp) / kp;
    if (xi < lo || xi > hi) xi = 0.5 * (lo + hi);
    for (int it = 0; it < 400; ++it) {
        double x = exp(xi);
        double r = rp + x;
        double f = or_rstar_of_x(M, a, x) - rs;
        if (f > 0) hi = xi; else lo = xi;
        double fp = (r * r + a * a) / (x + rp - rm);
        double step = f / fp;
        double xn = xi - step;
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        if (fabs(xn - xi) <= 1e-16 * (1.0 + fabs(xi)) || hi - lo < 1e-300) {
            xi = xn;
            break;
        }
        xi = xn;
    }
    *x_out = exp(xi);
    return 0;
}

/* Prograde circular equatorial orbit: Omega = M^{1/2}/(r0^{3/2} + a M^{1/2}). */
double or_kepler_omega(double M, double a, double r0)
{
    return sqrt(M) / (pow(r0, 1.5) + a * sqrt(M));
}

/* ------------------------------------------------------ coefficients ---- */

/* Coefficients of  Phi_tt - b^2 Phi_{r*r*} + c_t Phi_t + c_* Phi_{r*}
 *                  + c_0 Phi - q (Phi_thth + cot th Phi_th) = F,
 * which is Eq. 1 after Eqs. 2-4 (Psi = e^{i m phi~} r^3 Phi) and division by
 * -Sigma^2 r^3/Delta (Sigma^2 of Eq. 7).  The first-order form with
 * Pi = Phi_t + b Phi_{r*} (Eq. 5) is
 *     Phi_t + b Phi_{r*} = Pi
 *     Pi_t  - b Pi_{r*}  = F - c_t Pi + K Phi_{r*} - c_0 Phi + q L_th Phi
 * with K = b c_t - c_* - b b_{,r*}; this is Eq. 9 with D of Eq. 11.
 * Symbols: R = r^2 + a^2, h = dr/dr* = Delta/R, P = 2r + 2s(r-M)R/Delta
 * + 2 i a m R/Delta (coefficient of psi_{r*} in Eq. 1 after Eqs. 2-3). */
void or_point_coef(const or_grid *g, double x, double th, or_coef *c)
{
    const double M = g->M, a = g->a;
    const double s = (double)g->s, m = (double)g->m;
    double rp, rm;
    horizons(M, a, &rp, &rm);
    double r = rp + x;
    double delta = x * (x + rp - rm);
    double R = r * r + a * a;
    double sn = sin(th), cs = cos(th), sn2 = sn * sn;

    double sigma2 = R * R - a * a * delta * sn2;             /* Eq. 7 */
    double Sig = sqrt(sigma2);
    double b = R / Sig;                                       /* Eq. 6 */
    double h = delta / R;                                     /* Eq. 2 */
    double q = delta / sigma2;

    /* b_{,r*} = h d b/dr at fixed theta */
    double dR = 2.0 * r;
    double dsig2 = 2.0 * R * dR - a * a * sn2 * 2.0 * (r - M);
    double dbdr = dR / Sig - R * dsig2 / (2.0 * Sig * sigma2);
    double b_rs = h * dbdr;

    /* c_t = (Delta/Sigma^2)[4iMamr/Delta + 2s(r - M(r^2-a^2)/Delta) + 2isa cos th] */
    cplx ct = (2.0 * s * (r * delta - M * (r * r - a * a))
               + I * (4.0 * M * a * m * r + 2.0 * s * a * delta * cs)) / sigma2;

    /* q P, written without 1/Delta */
    cplx qP = (2.0 * r * delta + 2.0 * s * (r - M) * R + I * 2.0 * a * m * R) / sigma2;

    /* c_* = -b^2 (6h/r) - q P */
    cplx cstar = -b * b * 6.0 * h / r - qP;

    /* c_0 = -b^2 (3 r^2 h)_{,r*}/r^3 - q (3h/r) P - q[s - V_th]
     *       - 4 i s m a (r-M)/Sigma^2,  V_th = (m + s cos th)^2/sin^2 th */
    double d3 = h * (6.0 * r * delta / R + 6.0 * r * r * (r - M) / R
                     - 6.0 * r * r * r * delta / (R * R));
    cplx c0rad = -b * b * d3 / (r * r * r) - (3.0 * h / r) * qP
                 - I * 4.0 * s * m * a * (r - M) / sigma2;
    double V = (m + s * cs) * (m + s * cs) / sn2;
    double c0ang = q * (V - s);

    cplx K = b * ct - cstar - b * b_rs;

    c->r = r;
    c->x = x;
    c->delta = delta;
    c->R = R;
    c->sigma2 = sigma2;
    c->b = b;
    c->b_rs = b_rs;
    c->q = q;
    c->ct_re = creal(ct);
    c->ct_im = cimag(ct);
    c->cs_re = creal(cstar);
    c->cs_im = cimag(cstar);
    c->c0rad_re = creal(c0rad);
    c->c0rad_im = cimag(c0rad);
    c->c0ang = c0ang;
    c->K_re = creal(K);
    c->K_im = cimag(K);
    c->Fpref = 4.0 * OR_PI * (r * r + a * a * cs * cs) * delta / (sigma2 * r * r * r);
}

/* ------------------------------------------------------ angular part ---- */

/* Second-order centred differences (Sec. 2.2, end):
 *   L_th Phi_j = (Phi_{j+1} - 2 Phi_j + Phi_{j-1})/dth^2
 *              + cot th_j (Phi_{j+1} - Phi_{j-1})/(2 dth)
 * with parity ghosts Phi_{-1} = p Phi_0, Phi_{N} = p Phi_{N-1}. */
static cplx ltheta_at(const or_grid *g, const cplx *row, long j)
{
    long N = g->Nth;
    double p = ghost_parity(g);
    double dth = dth_of(g);
    double th = theta_of(g, j);
    cplx fm = (j > 0) ? row[j - 1] : p * row[0];
    cplx fp = (j < N - 1) ? row[j + 1] : p * row[N - 1];
    cplx f0 = row[j];
    return (fp - 2.0 * f0 + fm) / (dth * dth) + (cos(th) / sin(th)) * (fp - fm) / (2.0 * dth);
}

static double vtheta_minus_s(const or_grid *g, long j)
{
    double th = theta_of(g, j);
    double s = (double)g->s, m = (double)g->m;
    double sn = sin(th);
    return (m + s * cos(th)) * (m + s * cos(th)) / (sn * sn) - s;
}

/* The angular operator  A_th = -L_th + (m + s cos th)^2/sin^2 th - s  acting
 * on one theta row (complex).  Its continuum eigenvalues are (l-s)(l+s+1). */
void or_apply_atheta(const or_grid *g, const double *row_in, double *row_out)
{
    const cplx *in = (const cplx *)row_in;
    cplx *out = (cplx *)row_out;
    for (long j = 0; j < g->Nth; ++j)
        out[j] = -ltheta_at(g, in, j) + vtheta_minus_s(g, j) * in[j];
}

/* Row j of A_th as a tridiagonal matrix, ghosts folded into the diagonal. */
static void atheta_row(const or_grid *g, long j, double *lo, double *di, double *up)
{
    long N = g->Nth;
    double p = ghost_parity(g);
    double dth = dth_of(g);
    double th = theta_of(g, j);
    double cot = cos(th) / sin(th);
    double l = -(1.0 - 0.5 * cot * dth) / (dth * dth);
    double u = -(1.0 + 0.5 * cot * dth) / (dth * dth);
    double d = 2.0 / (dth * dth) + vtheta_minus_s(g, j);
    if (j == 0) { d += p * l; l = 0.0; }
    if (j == N - 1) { d += p * u; u = 0.0; }
    *lo = l;
    *di = d;
    *up = u;
}

/* ------------------------------------------------------------ source ---- */

/* F = 4 pi (r^2 + a^2 cos^2 th) Delta/(Sigma^2 r^3) T  (right side of Eq. 1
 * after the same division as the left side), with the circular-orbit
 * Gaussian  T = A exp(-(r*-r0*)^2/(2 sig_r^2) - (th-pi/2)^2/(2 sig_th^2))
 *               exp(-i m Omega t). */
static cplx source_F(const or_grid *g, const or_source *src, double rs0,
                     double rs, const or_coef *c, double th, double t)
{
    if (src == NULL || (src->amp_re == 0.0 && src->amp_im == 0.0)) return 0.0;
    double dr = rs - rs0, dth = th - 0.5 * OR_PI;
    double G = exp(-dr * dr / (2.0 * src->sig_r * src->sig_r)
                   - dth * dth / (2.0 * src->sig_th * src->sig_th));
    double phase = (double)g->m * src->Omega * t;
    cplx A = src->amp_re + I * src->amp_im;
    return c->Fpref * A * G * (cos(phase) - I * sin(phase));
}

/* ---------------------------------------------------------- checks ------ */

static int grid_ok(const or_grid *g)
{
    if (g->Nr < 3 || g->Nth < 1) return 0;
    if (!(g->rs_max > g->rs_min) || !(g->dt > 0.0) || !(g->M > 0.0)) return 0;
    if (!(fabs(g->a) < g->M)) return 0;
    return 1;
}

static void set_threads(const or_grid *g, int *nt)
{
#ifdef _OPENMP
    *nt = g->nthreads > 0 ? g->nthreads : omp_get_max_threads();
#else
    (void)g;
    *nt = 1;
#endif
}

/* -------------------------------------------------- Lax-Wendroff step ---- */

/* One two-step Lax-Wendroff update, Eqs. 13-14, of
 *     d_t u + D d_{r*} u = S,   u = {Phi_R, Phi_I, Pi_R, Pi_I},
 *     D = diag(b, b, -b, -b)                              (Eqs. 10-11)
 *     S = T - (M - D) d_{r*} u - L u - A u                 (Eq. 12)
 * Rows of S, from the first-order form above:
 *     full = 1 (every term of Eq. 12; the literal scheme):
 *         S_Phi = Pi
 *         S_Pi  = F + K Phi_{r*} - c_t Pi - c0rad Phi + q L_th Phi - c0ang Phi
 *     full = 0 (only T - (M - D) d_{r*} u; the split scheme, whose implicit
 *               half-steps carry -L u - A u):
 *         S_Phi = 0
 *         S_Pi  = F + K Phi_{r*}
 * Readings: S at a midpoint uses the averaged field of Eq. 13's first term
 * and the compact difference of Eq. 13's second term; S at a node in
 * Eq. 14 uses the average of the two adjacent midpoints and their
 * difference; the theta stencil acts on those same averaged fields.
 * Radial boundary rows are Phi = Pi = 0 (Sec. 2.2). */
static int lw_impl(const or_grid *g, const or_source *src, long n, int full,
                   const cplx *u, cplx *unew, cplx *mid)
{
    const long Nr = g->Nr, N = g->Nth;
    const double dt = g->dt, drs = drs_of(g);
    const cplx *Phi = u, *Pi = u + Nr * N;
    cplx *Phin = unew, *Pin = unew + Nr * N;
    cplx *mPhi = mid, *mPi = mid + (Nr - 1) * N;
    const double tn = (double)n * dt;
    double rs0 = 0.0;
    if (src != NULL) {
        double rp, rm;
        horizons(g->M, g->a, &rp, &rm);
        rs0 = or_rstar_of_x(g->M, g->a, src->r0 - rp);
    }
    int nt;
    set_threads(g, &nt);
    int bad = 0;

    /* Eq. 13: u^{n+1/2}_{i+1/2}, i = 0..Nr-2, source at t^n */
#pragma omp parallel for schedule(static) num_threads(nt) reduction(| : bad)
    for (long i = 0; i < Nr - 1; ++i) {
        double rs = g->rs_min + ((double)i + 0.5) * drs;
        double x;
        if (or_x_of_rstar(g->M, g->a, rs, &x) != 0) { bad |= 1; continue; }
        cplx *avg = (cplx *)malloc(sizeof(cplx) * (size_t)N);
        for (long j = 0; j < N; ++j) avg[j] = 0.5 * (Phi[(i + 1) * N + j] + Phi[i * N + j]);
        for (long j = 0; j < N; ++j) {
            double th = theta_of(g, j);
            or_coef c;
            or_point_coef(g, x, th, &c);
            cplx Phib = avg[j];
            cplx Pib = 0.5 * (Pi[(i + 1) * N + j] + Pi[i * N + j]);
            cplx dPhi = (Phi[(i + 1) * N + j] - Phi[i * N + j]) / drs;
            cplx dPi = (Pi[(i + 1) * N + j] - Pi[i * N + j]) / drs;
            cplx ct = c.ct_re + I * c.ct_im, K = c.K_re + I * c.K_im;
            cplx c0 = c.c0rad_re + I * c.c0rad_im;
            cplx SPhi = full ? Pib : 0.0;
            cplx SPi = source_F(g, src, rs0, rs, &c, th, tn) + K * dPhi;
            if (full) SPi += -ct * Pib - c0 * Phib + c.q * ltheta_at(g, avg, j) - c.c0ang * Phib;
            mPhi[i * N + j] = Phib - 0.5 * dt * (c.b * dPhi - SPhi);
            mPi[i * N + j] = Pib - 0.5 * dt * (-c.b * dPi - SPi);
        }
        free(avg);
    }
    if (bad) return -1;

    /* Eq. 14: u^{n+1}_i, i = 1..Nr-2, source at t^n + dt/2 */
#pragma omp parallel for schedule(static) num_threads(nt) reduction(| : bad)
    for (long i = 1; i < Nr - 1; ++i) {
        double rs = g->rs_min + (double)i * drs;
        double x;
        if (or_x_of_rstar(g->M, g->a, rs, &x) != 0) { bad |= 1; continue; }
        cplx *avg = (cplx *)malloc(sizeof(cplx) * (size_t)N);
        for (long j = 0; j < N; ++j) avg[j] = 0.5 * (mPhi[i * N + j] + mPhi[(i - 1) * N + j]);
        for (long j = 0; j < N; ++j) {
            double th = theta_of(g, j);
            or_coef c;
            or_point_coef(g, x, th, &c);
            cplx Phit = avg[j];
            cplx Pit = 0.5 * (mPi[i * N + j] + mPi[(i - 1) * N + j]);
            cplx dPhi = (mPhi[i * N + j] - mPhi[(i - 1) * N + j]) / drs;
            cplx dPi = (mPi[i * N + j] - mPi[(i - 1) * N + j]) / drs;
            cplx ct = c.ct_re + I * c.ct_im, K = c.K_re + I * c.K_im;
            cplx c0 = c.c0rad_re + I * c.c0rad_im;
            cplx SPhi = full ? Pit : 0.0;
            cplx SPi = source_F(g, src, rs0, rs, &c, th, tn + 0.5 * dt) + K * dPhi;
            if (full) SPi += -ct * Pit - c0 * Phit + c.q * ltheta_at(g, avg, j) - c.c0ang * Phit;
            Phin[i * N + j] = Phi[i * N + j] - dt * (c.b * dPhi - SPhi);
            Pin[i * N + j] = Pi[i * N + j] - dt * (-c.b * dPi - SPi);
        }
        free(avg);
    }
    if (bad) return -1;
    for (long j = 0; j < N; ++j) {
        Phin[j] = 0.0;
        Pin[j] = 0.0;
        Phin[(Nr - 1) * N + j] = 0.0;
        Pin[(Nr - 1) * N + j] = 0.0;
    }
    return 0;
}

/* ----------------------------------- implicit half-step (SDIRK2) ------- */

static void apply_B(long N, const double *lo, const double *di, const double *up,
                    const cplx *x, cplx *y)
{
    for (long j = 0; j < N; ++j) {
        cplx v = di[j] * x[j];
        if (j > 0) v += lo[j] * x[j - 1];
        if (j < N - 1) v += up[j] * x[j + 1];
        y[j] = v;
    }
}

/* Complex tridiagonal solve  (diag_j) x_j + c lo_j x_{j-1} + c up_j x_{j+1} = r_j
 * (Thomas algorithm, complex pivots). */
static void solve_tri_c(long N, double c, const double *lo, const cplx *dg, const double *up,
                        const cplx *r, cplx *x, cplx *cp)
{
    cplx denom = dg[0];
    cp[0] = (N > 1) ? c * up[0] / denom : 0.0;
    x[0] = r[0] / denom;
    for (long j = 1; j < N; ++j) {
        double sub = c * lo[j];
        denom = dg[j] - sub * cp[j - 1];
        cp[j] = (j < N - 1) ? c * up[j] / denom : 0.0;
        x[j] = (r[j] - sub * x[j - 1]) / denom;
    }
    for (long j = N - 2; j >= 0; --j) x[j] -= cp[j] * x[j + 1];
}

/* One step of length h for the algebraic part of the first-order
 * system, i.e. the terms -L u - A u of S (Eq. 12):
 *     Phi_t = Pi,   Pi_t = -(B + c0rad) Phi - c_t Pi,   B = q A_th
 * (B is the angular operator with the pole potential; c0rad and c_t are the
 * remaining non-derivative coefficients).  In the split scheme these terms
 * leave S and are integrated implicitly, because taken explicitly inside the
 * two Lax-Wendroff stages (which act on them as a midpoint rule) they are
 * unstable: the pole-cell angular modes and the near-horizon rotation
 * Im c_t ~ 2 m Omega_H have purely imaginary eigenvalues.
 * Integrator: the two-stage, L-stable, stiffly accurate SDIRK method of
 * order 2 (Alexander, SIAM J. Numer. Anal. 14, 1977), gamma = 1 - 1/sqrt(2):
 *     U1 = u + gamma h J U1
 *     U2 = u + (1-gamma) h J U1 + gamma h J U2,      u^new = U2.
 * Each stage (I - gamma h J) U = (rPhi, rPi) reduces to one complex
 * tridiagonal solve:
 *     [(1 + gh c_t) + gh^2 (B + c0rad)] U_Phi = (1 + gh c_t) rPhi + gh rPi
 *     U_Pi = (rPi - gh (B + c0rad) U_Phi) / (1 + gh c_t),      gh = gamma h. */
static int loc_impl(const or_grid *g, double h, const cplx *u, cplx *unew)
{
    const long Nr = g->Nr, N = g->Nth;
    const double drs = drs_of(g);
    const double gam = 1.0 - 1.0 / sqrt(2.0);
    const double gh = gam * h, c = gh * gh;
    const cplx *Phi = u, *Pi = u + Nr * N;
    cplx *Phin = unew, *Pin = unew + Nr * N;
    int nt;
    set_threads(g, &nt);
    int bad = 0;

#pragma omp parallel for schedule(static) num_threads(nt) reduction(| : bad)
    for (long i = 1; i < Nr - 1; ++i) {
        double rs = g->rs_min + (double)i * drs;
        double x;
        if (or_x_of_rstar(g->M, g->a, rs, &x) != 0) { bad |= 1; continue; }
        double *lo = (double *)malloc(sizeof(double) * (size_t)N * 3);
        double *di = lo + N, *up = lo + 2 * N;
        cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)N * 11);
        cplx *ct = w, *c0 = w + N, *dg = w + 2 * N, *cp = w + 3 * N, *rhs = w + 4 * N;
        cplx *F1 = w + 5 * N, *P1 = w + 6 * N, *BF = w + 7 * N, *rPhi = w + 8 * N, *rPi = w + 9 * N;
        cplx *F2 = w + 10 * N;
        const cplx *ph = Phi + i * N, *pi = Pi + i * N;
        for (long j = 0; j < N; ++j) {
            or_coef cf;
            or_point_coef(g, x, theta_of(g, j), &cf);
            double l, d, uu;
            atheta_row(g, j, &l, &d, &uu);
            lo[j] = cf.q * l;
            di[j] = cf.q * d;
            up[j] = cf.q * uu;
            ct[j] = cf.ct_re + I * cf.ct_im;
            c0[j] = cf.c0rad_re + I * cf.c0rad_im;
            dg[j] = 1.0 + gh * ct[j] + c * (di[j] + c0[j]);
        }
        /* stage 1 */
        for (long j = 0; j < N; ++j) rhs[j] = (1.0 + gh * ct[j]) * ph[j] + gh * pi[j];
        solve_tri_c(N, c, lo, dg, up, rhs, F1, cp);
        apply_B(N, lo, di, up, F1, BF);
        for (long j = 0; j < N; ++j) {
            BF[j] += c0[j] * F1[j];
            P1[j] = (pi[j] - gh * BF[j]) / (1.0 + gh * ct[j]);
        }
        /* stage 2: rhs = u + (1-gamma) h J U1 */
        for (long j = 0; j < N; ++j) {
            rPhi[j] = ph[j] + (1.0 - gam) * h * P1[j];
            rPi[j] = pi[j] - (1.0 - gam) * h * (BF[j] + ct[j] * P1[j]);
            rhs[j] = (1.0 + gh * ct[j]) * rPhi[j] + gh * rPi[j];
        }
        solve_tri_c(N, c, lo, dg, up, rhs, F2, cp);
        apply_B(N, lo, di, up, F2, BF);
        for (long j = 0; j < N; ++j) {
            BF[j] += c0[j] * F2[j];
            Phin[i * N + j] = F2[j];
            Pin[i * N + j] = (rPi[j] - gh * BF[j]) / (1.0 + gh * ct[j]);
        }
        free(w);
        free(lo);
    }
    if (bad) return -1;
    for (long j = 0; j < N; ++j) {
        Phin[j] = 0.0;
        Pin[j] = 0.0;
        Phin[(Nr - 1) * N + j] = 0.0;
        Pin[(Nr - 1) * N + j] = 0.0;
    }
    return 0;
}

/* ------------------------------------------------------------ public ---- */

int or_imp(const or_grid *g, double h, const double *u_in, double *u_out)
{
    if (!grid_ok(g) || !(h > 0.0)) return -10;
    return loc_impl(g, h, (const cplx *)u_in, (cplx *)u_out);
}

int or_lw(const or_grid *g, const or_source *src, long n, int full,
          const double *u_in, double *u_out)
{
    if (!grid_ok(g)) return -10;
    cplx *mid = (cplx *)malloc(sizeof(cplx) * (size_t)(g->Nr - 1) * (size_t)g->Nth * 2);
    if (!mid) return -11;
    int rc = lw_impl(g, src, n, full, (const cplx *)u_in, (cplx *)u_out, mid);
    free(mid);
    return rc;
}

/* Time stepping.
 *   literal: u^{n+1} = LW_n(u^n), Eqs. 13-14 with every term of Eq. 12 in S.
 *   split:   Strang splitting u^{n+1} = C_{dt/2} LW_n C_{dt/2} u^n, where
 *            C_h is the implicit step of the algebraic terms -L u - A u
 *            (loc_impl) and LW_n carries D and S = T - (M - D) d_{r*} u.
 *            Between consecutive steps the two half steps that meet,
 *            C_{dt/2} C_{dt/2}, are taken as one implicit step C_dt (both
 *            are second-order approximations of the same flow, so the
 *            composition stays second order).  The run therefore keeps the
 *            internal state s_n = LW_{n-1} C(s_{n-1}) and outputs the
 *            physical state u_n = C_{dt/2} s_n:
 *                s_{n0+1} = LW_{n0} C_{dt/2} u_{n0}         (first step)
 *                s_{n+1}  = LW_n C_dt s_n                    (later steps)
 *                u_{n}    = C_{dt/2} s_n. */
static int first_impl(const or_grid *g, const or_source *src, long n, const cplx *u, cplx *s_out,
                      cplx *t1, cplx *mid)
{
    int rc = loc_impl(g, 0.5 * g->dt, u, t1);
    if (rc) return rc;
    return lw_impl(g, src, n, 0, t1, s_out, mid);
}

static int next_impl(const or_grid *g, const or_source *src, long n, const cplx *s, cplx *s_out,
                     cplx *t1, cplx *mid)
{
    int rc = loc_impl(g, g->dt, s, t1);
    if (rc) return rc;
    return lw_impl(g, src, n, 0, t1, s_out, mid);
}

static cplx *scratch(const or_grid *g)
{
    size_t plane = (size_t)g->Nr * (size_t)g->Nth;
    return (cplx *)malloc(sizeof(cplx) * (plane * 2 + (size_t)(g->Nr - 1) * g->Nth * 2));
}

/* literal scheme: u^n -> u^{n+1};  split scheme: internal s_n -> s_{n+1}
 * (first = 1: from a physical state u_n, s_{n+1} = LW_n C_{dt/2} u_n). */
int or_step(const or_grid *g, const or_source *src, long n, int first,
            const double *u_in, double *u_out)
{
    if (!grid_ok(g)) return -10;
    size_t plane = (size_t)g->Nr * (size_t)g->Nth;
    cplx *buf = scratch(g);
    if (!buf) return -11;
    int rc;
    if (g->scheme == OR_SCHEME_LITERAL)
        rc = lw_impl(g, src, n, 1, (const cplx *)u_in, (cplx *)u_out, buf + 2 * plane);
    else if (first)
        rc = first_impl(g, src, n, (const cplx *)u_in, (cplx *)u_out, buf, buf + 2 * plane);
    else
        rc = next_impl(g, src, n, (const cplx *)u_in, (cplx *)u_out, buf, buf + 2 * plane);
    free(buf);
    return rc;
}

long or_extract_index(const or_grid *g)
{
    long i = lround((g->rs_ext - g->rs_min) / drs_of(g));
    if (i < 0) i = 0;
    if (i > g->Nr - 1) i = g->Nr - 1;
    return i;
}

/* Default extraction weights: projection on the lowest Schwarzschild
 * spin-weighted harmonic, Y = sin(th/2)^{|m+s|} cos(th/2)^{|m-s|}
 * (eigenvalue (l-s)(l+s+1) with l = max(|m|,|s|)), in the measure
 * sin th dth, normalised so that sum_j w_j Y_j = 1. */
void or_default_weights(const or_grid *g, double *w)
{
    long N = g->Nth;
    int e1 = abs(g->m + g->s), e2 = abs(g->m - g->s);
    double norm = 0.0;
    for (long j = 0; j < N; ++j) {
        double th = theta_of(g, j);
        double Y = pow(sin(0.5 * th), e1) * pow(cos(0.5 * th), e2);
        w[j] = sin(th) * Y;
        norm += sin(th) * Y * Y;
    }
    for (long j = 0; j < N; ++j) w[j] /= norm;
}

/* Waveform sample h = sum_j w_j Phi_{i_ext, j} in fixed j order. */
static void extract(const or_grid *g, const cplx *u, const double *w, double *h)
{
    long ie = or_extract_index(g), N = g->Nth;
    cplx acc = 0.0;
    for (long j = 0; j < N; ++j) acc += w[j] * u[ie * N + j];
    h[0] = creal(acc);
    h[1] = cimag(acc);
}

/* Advance the physical state u (in place) from step n0 by nsteps;
 * h_out[2k], h_out[2k+1] get the waveform sample of state n0+k,
 * k = 0..nsteps.  The split scheme starts a new Strang sequence at n0. */
int or_run(const or_grid *g, const or_source *src, long n0, long nsteps,
           double *u, const double *weights, double *h_out)
{
    if (!grid_ok(g) || nsteps < 0) return -10;
    size_t plane = (size_t)g->Nr * (size_t)g->Nth;
    double *w = (double *)malloc(sizeof(double) * (size_t)g->Nth);
    cplx *buf = (cplx *)malloc(sizeof(cplx) * (plane * 6 + (size_t)(g->Nr - 1) * g->Nth * 2));
    if (!w || !buf) { free(w); free(buf); return -11; }
    if (weights) memcpy(w, weights, sizeof(double) * (size_t)g->Nth);
    else or_default_weights(g, w);
    cplx *ph = (cplx *)u, *s = buf, *s2 = buf + 2 * plane, *t1 = buf + 4 * plane, *mid = buf + 6 * plane;
    if (h_out) extract(g, ph, w, h_out);
    int rc = 0;
    for (long k = 0; k < nsteps; ++k) {
        if (g->scheme == OR_SCHEME_LITERAL) {
            rc = lw_impl(g, src, n0 + k, 1, ph, s, mid);
            if (rc) break;
            memcpy(ph, s, sizeof(cplx) * 2 * plane);
        } else {
            if (k == 0) rc = first_impl(g, src, n0, ph, s, t1, mid);
            else rc = next_impl(g, src, n0 + k, s, s2, t1, mid);
            if (rc) break;
            if (k > 0) memcpy(s, s2, sizeof(cplx) * 2 * plane);
            rc = loc_impl(g, 0.5 * g->dt, s, ph);      /* physical u_{n0+k+1} */
            if (rc) break;
        }
        if (h_out) extract(g, ph, w, h_out + 2 * (k + 1));
    }
    free(w);
    free(buf);
    return rc;
}
