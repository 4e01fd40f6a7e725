/*
 * teuk_oracle.h -- plain FP64 CPU oracle for the time step of the
 * mode-decomposed (2+1)-D Teukolsky equation (Khanna & McKennon,
 * "An exploration of CUDA and CBEA for a gravitational wave
 * source-modelling application", Sec. 2, Eqs. 1-14).
 *
 * TEST INFRASTRUCTURE.  This library exists only to check the CUDA path.
 * Only tests/, __graft_entry__.smoke() and bench.py (its cpu_baseline leg
 * and its "--impl reference" arm) may load or call it.  It shares no code,
 * header, table or constant with the CUDA library under
 * paper_0909_4039_gb300/, and neither side includes the other.
 *
 * Everything is double precision.  Readings of the paper where it is
 * silent (all listed in the repository's design notes):
 *   - r*(r): Eq. 2 integrated with the usual integration constant
 *     (Sec. 2.2, Eq. 2);
 *   - M, L, A: not printed in the paper (Sec. 2.2 after Eq. 8 defers them
 *     to the literature); derived here from Eq. 1 with Eqs. 2-7;
 *   - theta grid cell centred, theta_j = (j+1/2) pi/Ntheta; the pole
 *     conditions of Sec. 2.2 enter as parity ghost cells;
 *   - two schemes.  "literal": Eqs. 13-14 with every term of Eq. 12 in S
 *     (unstable at dt = dr* / 2; kept for few-step checks).  "split": an
 *     implicit-explicit Strang splitting -- the algebraic terms -L u - A u
 *     of S are integrated by the L-stable two-stage SDIRK method of order
 *     2 (half steps at the ends of a run, one full step between two
 *     Lax-Wendroff steps), and the Lax-Wendroff step of Eqs. 13-14
 *     carries the transport D and S = T - (M - D) d_{r*} u;
 *   - the source T is a Gaussian on a circular equatorial orbit.
 *
 * State layout: u = [2][Nr][Ntheta] complex double, re/im interleaved,
 * theta fastest; plane 0 = Phi, plane 1 = Pi (Eqs. 4-5, 9).
 */
#ifndef TEUK_ORACLE_H
#define TEUK_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define OR_SCHEME_LITERAL 0
#define OR_SCHEME_SPLIT 1

typedef struct {
    int s;          /* spin weight (Eq. 1) */
    int m;          /* azimuthal mode number (Eq. 4) */
    double M;       /* black-hole mass */
    double a;       /* spin parameter, 0 <= |a| < M */
    long Nr;        /* radial nodes, r*_i = rs_min + i*drs, i = 0..Nr-1 */
    long Nth;       /* theta cells, theta_j = (j+1/2)*pi/Nth */
    double rs_min;  /* r* of node 0 */
    double rs_max;  /* r* of node Nr-1 */
    double dt;      /* time step */
    double rs_ext;  /* extraction radius (nearest node is used) */
    int scheme;     /* OR_SCHEME_LITERAL or OR_SCHEME_SPLIT */
    int nthreads;   /* OpenMP threads (<= 0: runtime default) */
} or_grid;

typedef struct {
    double amp_re, amp_im;   /* complex amplitude A of the source */
    double r0;               /* Boyer-Lindquist orbital radius */
    double sig_r;            /* Gaussian standard deviation in r* */
    double sig_th;           /* Gaussian standard deviation in theta */
    double Omega;            /* orbital angular frequency */
} or_source;

/* Coefficients of the first-order system at one point (Eqs. 9-12). */
typedef struct {
    double r, x, delta, R;        /* r, r - r_+, Delta, r^2 + a^2        */
    double sigma2;                /* Sigma^2 of Eq. 7                    */
    double b;                     /* Eq. 6                               */
    double b_rs;                  /* d b / d r* at fixed theta           */
    double q;                     /* Delta / Sigma^2                     */
    double ct_re, ct_im;          /* coefficient of Phi_t                */
    double cs_re, cs_im;          /* coefficient of Phi_{r*}             */
    double c0rad_re, c0rad_im;    /* radial part of the Phi coefficient  */
    double c0ang;                 /* q (V_theta - s), the angular part   */
    double K_re, K_im;            /* b c_t - c_* - b b_{,r*}             */
    double Fpref;                 /* 4 pi (r^2 + a^2 cos^2) Delta/(Sigma^2 r^3) */
} or_coef;

double or_rstar_of_x(double M, double a, double x);
int or_x_of_rstar(double M, double a, double rs, double *x_out);
void or_point_coef(const or_grid *g, double x, double theta, or_coef *c);
double or_kepler_omega(double M, double a, double r0);

void or_apply_atheta(const or_grid *g, const double *row_in, double *row_out);
void or_default_weights(const or_grid *g, double *w);
long or_extract_index(const or_grid *g);

int or_step(const or_grid *g, const or_source *src, long n, int first,
            const double *u_in, double *u_out);
int or_run(const or_grid *g, const or_source *src, long n0, long nsteps,
           double *u, const double *weights, double *h_out);
int or_imp(const or_grid *g, double h, const double *u_in, double *u_out);
int or_lw(const or_grid *g, const or_source *src, long n, int full,
          const double *u_in, double *u_out);

#ifdef __cplusplus
}
#endif
#endif
