// teuk_coef.cu -- FP64 generation of the coefficient tables on the device.
//
// Runs once per context (and once per source change).  Everything here is
// double precision, whatever the state precision: the radial tables, the
// theta tables, the Thomas pivots of the implicit stage matrix and the
// source patch are computed in FP64 and rounded to the state precision only
// when stored.
//
// Paper: Khanna & McKennon, arXiv:0909.4039, Sec. 2.
//   Eq. 2   dr* = (r^2 + a^2)/Delta dr, integrated with the usual constant
//   Eq. 4   Psi = e^{i m phi~} r^3 Phi
//   Eqs. 5-7, 9-12  first-order system; the coefficient forms are those of
//           the first-order form Phi_t + b Phi_{r*} = Pi,
//           Pi_t - b Pi_{r*} = F - c_t Pi + K Phi_{r*} - c_0 Phi + q L_th Phi,
//           which follows from Eq. 1 with Eqs. 2-4; they are regrouped here as
//           r-only polynomials divided by Sigma^2 (see RField).
#include <math.h>

#include "teuk_internal.cuh"

namespace teuk {
namespace {

struct Kerr {
    double M, a, rp, rm, kp, km;   // horizons and the two log weights of Eq. 2
};

__host__ __device__ inline Kerr make_kerr(double M, double a)
{
    Kerr k;
    double d = sqrt(M * M - a * a);
    k.M = M;
    k.a = a;
    k.rp = M + d;
    k.rm = M - d;
    k.kp = M * k.rp / d;   // 2 M r_+ / (r_+ - r_-)
    k.km = M * k.rm / d;   // 2 M r_- / (r_+ - r_-)
    return k;
}

// r*(x), x = r - r_+ > 0:
//   r* = r + 2M r_+/(r_+ - r_-) ln(x/2M) - 2M r_-/(r_+ - r_-) ln((x + r_+ - r_-)/2M)
__device__ inline double tortoise(const Kerr &k, double x)
{
    return k.rp + x + k.kp * log(x / (2.0 * k.M)) - k.km * log((x + (k.rp - k.rm)) / (2.0 * k.M));
}

// Inverse of tortoise() by Newton's method in u = ln x with a bisection
// safeguard.  d r*/d u = x (r^2 + a^2)/Delta = (r^2 + a^2)/(x + r_+ - r_-).
__device__ double x_of_rstar(const Kerr &k, double rs)
{
    double lo = -700.0, hi = 60.0;
    double u;
    if (rs > k.rp + 6.0 * k.M)
        u = log(rs);                       // far zone: r ~ r*
    else
        u = (rs - k.rp) / k.kp;            // near zone: r* ~ kp ln x
    u = fmin(fmax(u, lo + 1.0), hi - 1.0);
    for (int it = 0; it < 300; ++it) {
        double x = exp(u);
        double f = tortoise(k, x) - rs;
        if (f > 0.0) hi = u; else lo = u;
        double r = k.rp + x;
        double df = (r * r + k.a * k.a) / (x + (k.rp - k.rm));
        double un = u - f / df;
        if (!(un > lo && un < hi)) un = 0.5 * (lo + hi);
        double du = fabs(un - u);
        u = un;
        if (du <= 1e-16 * (1.0 + fabs(u)) || hi - lo <= 1e-15) break;
    }
    return exp(u);
}

// Forward-mode dual number v + d eps (eps^2 = 0): d carries the derivative
// with respect to the spin a through every operation.
struct Dual {
    double v, d;
};
__host__ __device__ inline Dual dual(double v, double d = 0.0) { return Dual{v, d}; }
__host__ __device__ inline Dual operator+(Dual a, Dual b) { return Dual{a.v + b.v, a.d + b.d}; }
__host__ __device__ inline Dual operator-(Dual a, Dual b) { return Dual{a.v - b.v, a.d - b.d}; }
__host__ __device__ inline Dual operator*(Dual a, Dual b) { return Dual{a.v * b.v, a.v * b.d + a.d * b.v}; }
__host__ __device__ inline Dual operator/(Dual a, Dual b)
{
    const double q = a.v / b.v;
    return Dual{q, (a.d - q * b.d) / b.v};
}
__host__ __device__ inline Dual operator*(double s, Dual a) { return Dual{s * a.v, s * a.d}; }

__host__ __device__ inline double dual_or(double M, double) { return M; }
__host__ __device__ inline Dual dual_or(double M, Dual) { return dual(M); }

// All r-only factors at one radial position (see RField), for N = double,
// or N = Dual with r, x, Delta and a carrying their spin derivatives.
template <typename N>
__device__ void rfields_t(double M, N a, int s, int m, N r, N x, N D, N *f)
{
    const double sd = (double)s, md = (double)m;
    const N R = r * r + a * a;
    f[RF_R] = R;
    f[RF_R2] = R * R;
    f[RF_AD] = a * a * D;
    f[RF_DELTA] = D;
    f[RF_CTR] = (2.0 * sd) * (r * D - M * (r * r - a * a));
    f[RF_CTI] = (4.0 * M * md) * (a * r);
    f[RF_CTC] = (2.0 * sd) * (a * D);
    f[RF_CSR] = 6.0 * (R * D / r) + 2.0 * (r * D) + (2.0 * sd) * (R * (r - dual_or(M, r)));
    f[RF_CSI] = (2.0 * md) * (a * R);
    f[RF_E1] = 2.0 * (r * D);
    f[RF_E2] = 2.0 * (r * D * R * R);
    f[RF_E3] = a * a * D * R * (r - dual_or(M, r));
    f[RF_C0R] = 6.0 * (D * D / (r * r)) + (6.0 * (1.0 + sd)) * (D * (r - dual_or(M, r)) / r);
    f[RF_C0I] = (6.0 * md) * (a * D / r) + (4.0 * sd * md) * (a * (r - dual_or(M, r)));
    f[RF_RR] = r;
    f[RF_X] = x;
}

__device__ void rfields(const Kerr &k, int s, int m, double x, double *f)
{
    const double r = k.rp + x;
    const double D = x * (x + (k.rp - k.rm));      // Delta without cancellation
    rfields_t<double>(k.M, k.a, s, m, r, x, D, f);
}

// d r*/d a at fixed r (Eq. 2 with its constant; x = r - r_+, d = r_+ - M):
//   (M^2 a / d^3) ln(x/(x + 2d)) + (M a / d^2) (r_+/x + r_-/(x + 2d)),
// so that at fixed r* the radius moves by dr/da = -(d r*/d a) Delta/(r^2 + a^2).
__host__ __device__ inline double drstar_da(const Kerr &k, double x)
{
    const double d = k.rp - k.M, a = k.a, M = k.M;
    if (a == 0.0) return 0.0;
    return (M * M * a / (d * d * d)) * log(x / (x + 2.0 * d)) + (M * a / (d * d)) * (k.rp / x + k.rm / (x + 2.0 * d));
}

// The r-table fields at fixed r* as duals in a: r(r*; a), x = r - r_+(a),
// Delta = x (x + r_+ - r_-) and a itself carry their derivatives.
__device__ void rfields_dual(const Kerr &k, int s, int m, double x, Dual *f)
{
    const double r = k.rp + x, d = k.rp - k.M, a = k.a;
    const double Dl = x * (x + 2.0 * d);
    const double dr = -drstar_da(k, x) * Dl / (r * r + a * a);
    const double drp = d > 0.0 ? -a / d : 0.0;   // d r_+ / d a
    const Dual rd = dual(r, dr), xd = dual(x, dr - drp), twod = dual(2.0 * d, d > 0.0 ? -2.0 * a / d : 0.0);
    rfields_t<Dual>(k.M, dual(a, 1.0), s, m, rd, xd, xd * (xd + twod), f);
}

// Step-table fields (SField) from the r-table fields f; the source block
// is zero (teuk_set_source fills it).
template <typename N>
__device__ void stab_fields(const N *f, double cp, N *g)
{
    g[SF_R2] = f[RF_R2];
    g[SF_AD] = f[RF_AD];
    g[SF_DELTA] = f[RF_DELTA];
    g[SF_CTR] = f[RF_CTR];
    g[SF_CTI] = f[RF_CTI];
    g[SF_CTC] = f[RF_CTC];
    g[SF_C0R] = f[RF_C0R];
    g[SF_C0I] = f[RF_C0I];
    g[SF_RB] = cp * f[RF_R];
    g[SF_E2] = cp * f[RF_E2];
    g[SF_E3] = cp * f[RF_E3];
    g[SF_RCTR] = cp * (f[RF_R] * f[RF_CTR]);
    g[SF_CSE] = cp * (f[RF_CSR] - f[RF_E1]);
    g[SF_RCTC] = cp * (f[RF_R] * f[RF_CTC]);
    g[SF_RCTI] = cp * (f[RF_R] * f[RF_CTI]);
    g[SF_CSI] = cp * f[RF_CSI];
    g[SF_SRE] = g[SF_SIM] = g[SF_SR2] = g[SF_SPAD] = 0.0 * f[RF_R];
}

struct CoefArgs {
    Kerr k;
    int s, m;
    int Nr, Nth;
    double rs_min, drs, dth;
    double gh, gh2;            // gamma h and its square for the pivot table being built
    double dt;                 // time step (scales the Lax-Wendroff block of the step table)
    int prec;                  // TEUK_FP64 / TEUK_FP32
    double *rtab64;
    void *rtabT;
    void *stab, *dstab;
    double *th64;
    void *thT;
    void *piv;
    double *w;
};

__global__ void k_rtab(CoefArgs A)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= 2 * A.Nr - 1) return;
    int i = p >> 1;
    double rs = (p & 1) ? A.rs_min + ((double)i + 0.5) * A.drs : A.rs_min + (double)i * A.drs;
    double x = x_of_rstar(A.k, rs);
    double f[NRF];
    rfields(A.k, A.s, A.m, x, f);
    for (int q = 0; q < NRF; ++q) A.rtab64[(size_t)p * NRF + q] = f[q];
    if (A.prec == TEUK_FP32) {
        float *o = (float *)A.rtabT;
        for (int q = 0; q < NRF; ++q) o[(size_t)p * NRF + q] = (float)f[q];
    }
    // step table (SField): the implicit block as is, the Lax-Wendroff block
    // times c_p = dt/dr* (node, Eq. 14) or dt/(2 dr*) (half node, Eq. 13)
    const double cp = ((p & 1) ? 0.5 : 1.0) * A.dt / A.drs;
    double g[NSF];
    stab_fields<double>(f, cp, g);
    // and its derivative with respect to a at fixed r* (the same formulas on
    // dual numbers; the source block is set by teuk_set_source)
    Dual fd[NRF], gd[NSF];
    rfields_dual(A.k, A.s, A.m, x, fd);
    stab_fields<Dual>(fd, cp, gd);
    if (A.prec == TEUK_FP32) {
        for (int q = 0; q < NSF; ++q) ((float *)A.stab)[(size_t)p * NSF + q] = (float)g[q];
        for (int q = 0; q < NSF; ++q) ((float *)A.dstab)[(size_t)p * NSF + q] = (float)gd[q].d;
    } else {
        for (int q = 0; q < NSF; ++q) ((double *)A.stab)[(size_t)p * NSF + q] = g[q];
        for (int q = 0; q < NSF; ++q) ((double *)A.dstab)[(size_t)p * NSF + q] = gd[q].d;
    }
}

// Theta tables and default extraction weights; one CTA, blockDim >= Nth.
__global__ void k_theta(CoefArgs A)
{
    __shared__ double red[32];
    int j = threadIdx.x;
    const int N = A.Nth;
    double num = 0.0;
    double Yw = 0.0;
    if (j < N) {
        double th = ((double)j + 0.5) * A.dth;
        double sn = sin(th), cs = cos(th);
        double cot = cs / sn;
        double id2 = 1.0 / (A.dth * A.dth);
        double am = -(1.0 - 0.5 * cot * A.dth) * id2;
        double ap = -(1.0 + 0.5 * cot * A.dth) * id2;
        double mc = (double)A.m + (double)A.s * cs;
        double a0 = 2.0 * id2 + mc * mc / (sn * sn) - (double)A.s;
        double par = (abs(A.m) % 2 == 0) ? 1.0 : -1.0;   // ghost parity (pole conditions)
        if (j == 0) { a0 += par * am; am = 0.0; }
        if (j == N - 1) { a0 += par * ap; ap = 0.0; }
        double v[NTF] = {sn * sn, cs, am, a0, ap, 0.0, 0.0, 0.0};   // source factors set later
        for (int q = 0; q < NTF; ++q) A.th64[q * N + j] = v[q];
        if (A.prec == TEUK_FP32)
            for (int q = 0; q < NTF; ++q) ((float *)A.thT)[q * N + j] = (float)v[q];
        // lowest harmonic sin(th/2)^{|m+s|} cos(th/2)^{|m-s|}
        double Y = pow(sin(0.5 * th), (double)abs(A.m + A.s)) * pow(cos(0.5 * th), (double)abs(A.m - A.s));
        Yw = sn * Y;
        num = sn * Y * Y;
    }
    // block sum of num
    for (int o = 16; o > 0; o >>= 1) num += __shfl_xor_sync(0xffffffffu, num, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = num;
    __syncthreads();
    if (threadIdx.x < 32) {
        int nw = (blockDim.x + 31) >> 5;
        double v = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    if (j < N) A.w[j] = Yw / red[0];
}

// Complex Thomas pivots of the implicit stage matrix (step h, gh = gamma h)
// of every node row i:
//   diag_j = 1 + gh c_t + gh^2 (c0rad + q A0_j),  sub_j = gh^2 q AM_j,
//   sup_j = gh^2 q AP_j;  d_0 = diag_0, d_j = diag_j - sub_j sup_{j-1}/d_{j-1};
// stored as e_j = 1/d_j at [i][j].
__global__ void k_pivots(CoefArgs A)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.Nr) return;
    const int N = A.Nth;
    const double *f = A.rtab64 + (size_t)(2 * i) * NRF;
    double dre = 1.0, dim = 0.0, prev_sup = 0.0;
    for (int j = 0; j < N; ++j) {
        double S2 = A.th64[TF_S2 * N + j], C = A.th64[TF_C * N + j];
        double am = A.th64[TF_AM * N + j], a0 = A.th64[TF_A0 * N + j], ap = A.th64[TF_AP * N + j];
        double sg = 1.0 / (f[RF_R2] - f[RF_AD] * S2);
        double q = f[RF_DELTA] * sg;
        double ctr = sg * f[RF_CTR], cti = sg * (f[RF_CTI] + f[RF_CTC] * C);
        double c0r = -sg * f[RF_C0R], c0i = -sg * f[RF_C0I];
        double gre = 1.0 + A.gh * ctr + A.gh2 * (c0r + q * a0);
        double gim = A.gh * cti + A.gh2 * c0i;
        if (j > 0) {
            // d_j = diag_j - sub_j sup_{j-1} / d_{j-1}
            double sub = A.gh2 * q * am;
            double ss = sub * prev_sup;
            double den = dre * dre + dim * dim;       // 1/d_{j-1} = conj(d)/|d|^2
            gre -= ss * dre / den;
            gim -= ss * (-dim) / den;
        }
        dre = gre;
        dim = gim;
        prev_sup = A.gh2 * q * ap;
        double den = dre * dre + dim * dim;
        double ere = dre / den, eim = -dim / den;
        size_t o = (size_t)i * N + j;
        if (A.prec == TEUK_FP32) ((float2 *)A.piv)[o] = make_float2((float)ere, (float)eim);
        else ((double2 *)A.piv)[o] = make_double2(ere, eim);
    }
}

struct PatchArgs {
    Kerr k;
    int Nr, Nth, p0, np, prec;
    double rs_min, drs, dth;
    double amp_re, amp_im, rs0, sig_r, sig_th;
    const double *rtab64;
    void *patch;    // A F_pref G (nullptr: not written)
    void *patchu;   // F_pref G, the unit-amplitude patch
};

// Spatial part of the source, A F_pref G(r*, theta), at the nodes and half
// nodes of patch rows; F_pref = 4 pi (r^2 + a^2 cos^2) Delta/(Sigma^2 r^3).
// The unit-amplitude part F_pref G is kept as well (source derivatives).
__global__ void k_patch(PatchArgs A)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int total = A.np * 2 * A.Nth;
    if (idx >= total) return;
    int j = idx % A.Nth;
    int pos = (idx / A.Nth) & 1;
    int pr = idx / (2 * A.Nth);
    int gi = A.p0 + pr;
    int p = 2 * gi + pos;
    double vre = 0.0, vim = 0.0;
    if (gi >= 0 && p <= 2 * A.Nr - 2) {
        const double *f = A.rtab64 + (size_t)p * NRF;
        double r = f[RF_RR], D = f[RF_DELTA];
        double th = ((double)j + 0.5) * A.dth;
        double cs = cos(th), sn = sin(th);
        double sig2 = f[RF_R2] - f[RF_AD] * sn * sn;
        double a = A.k.a;
        double pref = 4.0 * kPi * (r * r + a * a * cs * cs) * D / (sig2 * r * r * r);
        double rs = pos ? A.rs_min + ((double)gi + 0.5) * A.drs : A.rs_min + (double)gi * A.drs;
        double dr = rs - A.rs0, dq = th - 0.5 * kPi;
        double G = exp(-dr * dr / (2.0 * A.sig_r * A.sig_r) - dq * dq / (2.0 * A.sig_th * A.sig_th));
        vre = pref * G;
    }
    if (A.prec == TEUK_FP32) ((float2 *)A.patchu)[idx] = make_float2((float)vre, 0.0f);
    else ((double2 *)A.patchu)[idx] = make_double2(vre, 0.0);
    if (A.patch) {
        vim = A.amp_im * vre;
        vre = A.amp_re * vre;
        if (A.prec == TEUK_FP32) ((float2 *)A.patch)[idx] = make_float2((float)vre, (float)vim);
        else ((double2 *)A.patch)[idx] = make_double2(vre, vim);
    }
}

struct SrcArgs {
    Kerr k;
    int s, m;
    int Nr, Nth, p0, np, prec;
    double rs_min, drs, dth, a;
    double amp_re, amp_im, rs0, sig_r, sig_th, drs0_da;
    const double *rtab64;
    void *stab, *dstab;
    double *th64;
    void *thT;
};

// Source factors (SField, TField) at step-table position idx (and theta
// idx for the angular ones), from the FP64 r table; the same Gaussian and
// prefactor as k_patch, factored.
__global__ void k_src_fields(SrcArgs A)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < A.Nth) {
        const double th = ((double)idx + 0.5) * A.dth, cs = cos(th), dq = th - 0.5 * kPi;
        const double G = exp(-dq * dq / (2.0 * A.sig_th * A.sig_th));
        const double g2 = A.a * A.a * cs * cs * G;
        const double dg2 = 2.0 * A.a * cs * cs * G;   // d GA2 / d a
        A.th64[TF_GTH * A.Nth + idx] = G;
        A.th64[TF_GA2 * A.Nth + idx] = g2;
        A.th64[TF_DGA2 * A.Nth + idx] = dg2;
        if (A.prec == TEUK_FP32) {
            ((float *)A.thT)[TF_GTH * A.Nth + idx] = (float)G;
            ((float *)A.thT)[TF_GA2 * A.Nth + idx] = (float)g2;
            ((float *)A.thT)[TF_DGA2 * A.Nth + idx] = (float)dg2;
        }
    }
    if (idx >= 2 * A.Nr - 1) return;
    double sre = 0.0, sim = 0.0, r2 = 0.0, dsre = 0.0, dsim = 0.0, dr2 = 0.0;
    if (A.np > 0 && idx >= 2 * A.p0 && idx < 2 * (A.p0 + A.np)) {
        const double *f = A.rtab64 + (size_t)idx * NRF;
        const double r = f[RF_RR], D = f[RF_DELTA];
        const int gi = idx >> 1;
        const double rs = (idx & 1) ? A.rs_min + ((double)gi + 0.5) * A.drs : A.rs_min + (double)gi * A.drs;
        const double dr = rs - A.rs0;
        const double Gr = exp(-dr * dr / (2.0 * A.sig_r * A.sig_r));
        const double rad = 4.0 * kPi * D * Gr / (r * r * r);
        sre = A.amp_re * rad;
        sim = A.amp_im * rad;
        r2 = r * r;
        // spin derivatives at fixed r*: Delta and r through r(r*; a), the
        // Gaussian through its centre r0*(a)
        Dual fd[NRF];
        rfields_dual(A.k, A.s, A.m, f[RF_X], fd);
        const Dual rd = fd[RF_RR], Dd = fd[RF_DELTA];
        const Dual Gd = dual(Gr, Gr * dr * A.drs0_da / (A.sig_r * A.sig_r));
        const Dual radd = (4.0 * kPi) * (Dd * Gd / (rd * rd * rd));
        dsre = A.amp_re * radd.d;
        dsim = A.amp_im * radd.d;
        dr2 = (rd * rd).d;
    }
    const size_t o = (size_t)idx * NSF;
    if (A.prec == TEUK_FP32) {
        float *t = (float *)A.stab + o, *u = (float *)A.dstab + o;
        t[SF_SRE] = (float)sre;
        t[SF_SIM] = (float)sim;
        t[SF_SR2] = (float)r2;
        u[SF_SRE] = (float)dsre;
        u[SF_SIM] = (float)dsim;
        u[SF_SR2] = (float)dr2;
    } else {
        double *t = (double *)A.stab + o, *u = (double *)A.dstab + o;
        t[SF_SRE] = sre;
        t[SF_SIM] = sim;
        t[SF_SR2] = r2;
        u[SF_SRE] = dsre;
        u[SF_SIM] = dsim;
        u[SF_SR2] = dr2;
    }
}

__global__ void k_set_ctl(Ctl *c, long long step, int clear_flags)
{
    c->step = step;
    c->ticket = 0u;
    if (clear_flags) c->flags = 0u;
}

}  // namespace

cudaError_t launch_coef_tables(const teuk_grid_desc &d, double drs, double dt, void *coef,
                               const Layout &L, cudaStream_t st)
{
    CoefArgs A;
    A.k = make_kerr(d.M, d.a);
    A.s = d.s;
    A.m = d.m;
    A.Nr = (int)d.Nr;
    A.Nth = (int)d.Ntheta;
    A.rs_min = d.rstar_min;
    A.drs = drs;
    A.dth = kPi / (double)d.Ntheta;
    A.prec = d.precision;
    char *base = (char *)coef;
    A.rtab64 = (double *)(base + L.rtab64);
    A.rtabT = base + L.rtabT;
    A.stab = base + L.stab;
    A.dstab = base + L.dstab;
    A.dt = dt;
    A.th64 = (double *)(base + L.th64);
    A.thT = base + L.thT;
    A.w = (double *)(base + L.w);
    int np = 2 * A.Nr - 1;
    k_rtab<<<(np + 127) / 128, 128, 0, st>>>(A);
    int tb = ((A.Nth + 31) / 32) * 32;
    k_theta<<<1, tb, 0, st>>>(A);
    // pivots for implicit steps of length dt and dt/2
    A.gh = kGamma * dt;
    A.gh2 = A.gh * A.gh;
    A.piv = base + L.piv;
    k_pivots<<<(A.Nr + 127) / 128, 128, 0, st>>>(A);
    A.gh = kGamma * 0.5 * dt;
    A.gh2 = A.gh * A.gh;
    A.piv = base + L.pivh;
    k_pivots<<<(A.Nr + 127) / 128, 128, 0, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_patch(const teuk_grid_desc &d, double drs, void *coef, const Layout &L,
                         int p0, int np, double amp_re, double amp_im, double rs0,
                         double sig_r, double sig_th, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    PatchArgs A;
    A.k = make_kerr(d.M, d.a);
    A.Nr = (int)d.Nr;
    A.Nth = (int)d.Ntheta;
    A.p0 = p0;
    A.np = np;
    A.prec = d.precision;
    A.rs_min = d.rstar_min;
    A.drs = drs;
    A.dth = kPi / (double)d.Ntheta;
    A.amp_re = amp_re;
    A.amp_im = amp_im;
    A.rs0 = rs0;
    A.sig_r = sig_r;
    A.sig_th = sig_th;
    A.rtab64 = (const double *)((const char *)coef + L.rtab64);
    A.patch = (amp_re != 0.0 || amp_im != 0.0) ? (void *)((char *)coef + L.patch) : nullptr;
    A.patchu = (char *)coef + L.patchu;
    int total = np * 2 * A.Nth;
    k_patch<<<(total + 255) / 256, 256, 0, st>>>(A);
    return cudaGetLastError();
}

double host_drstar_da(double M, double a, double x) { return drstar_da(make_kerr(M, a), x); }

cudaError_t launch_src_fields(const teuk_grid_desc &d, double drs, void *coef, const Layout &L, int p0, int np,
                              double amp_re, double amp_im, double rs0, double sig_r, double sig_th,
                              double drs0_da, cudaStream_t st)
{
    SrcArgs A;
    A.k = make_kerr(d.M, d.a);
    A.s = d.s;
    A.m = d.m;
    A.drs0_da = drs0_da;
    A.Nr = (int)d.Nr;
    A.Nth = (int)d.Ntheta;
    A.p0 = p0;
    A.np = np;
    A.prec = d.precision;
    A.rs_min = d.rstar_min;
    A.drs = drs;
    A.dth = kPi / (double)d.Ntheta;
    A.a = d.a;
    A.amp_re = amp_re;
    A.amp_im = amp_im;
    A.rs0 = rs0;
    A.sig_r = sig_r;
    A.sig_th = sig_th;
    char *base = (char *)coef;
    A.rtab64 = (const double *)(base + L.rtab64);
    A.stab = base + L.stab;
    A.dstab = base + L.dstab;
    A.th64 = (double *)(base + L.th64);
    A.thT = base + L.thT;
    const int n = 2 * A.Nr - 1 > A.Nth ? 2 * A.Nr - 1 : A.Nth;
    k_src_fields<<<(n + 255) / 256, 256, 0, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_set_ctl(void *coef, const Layout &L, long long step, int clear_flags,
                           cudaStream_t st)
{
    k_set_ctl<<<1, 1, 0, st>>>((Ctl *)((char *)coef + L.ctl), step, clear_flags);
    return cudaGetLastError();
}

}  // namespace teuk
