// teuk_step.cu -- time-step kernels for sm_103a.
//
// Split scheme (default), one fused kernel per time step.  Each CTA owns a
// tile of TR consecutive r* rows with full theta rows and holds rows
// [i0-1, i0+TR] (one halo row each side) of both planes in shared memory:
//   A. load the tile; sigma2 = 1/Sigma^2 at its node rows
//   B. implicit half step (dt/2) of the algebraic terms -L u - A u on the
//      TR+2 rows: two SDIRK2 stages, each a complex tridiagonal solve in theta
//      done by one thread per row with the FP64-generated Thomas pivots
//   C. two-step Lax-Wendroff update (Eqs. 13-14) of the TR output rows with
//      S = T - (M - D) d_{r*} u, one thread per theta column marching down
//      the tile with a register window (this part has no theta coupling)
//   D. implicit half step on the TR output rows
//   E. store; the CTA holding the extraction node writes h_{n+1} (FP64 sum)
//      and the raw row into the ring buffer; the last CTA advances the
//      device step counter.
// The halo rows are recomputed by both neighbouring CTAs (B is row-local),
// so one step reads and writes the state exactly once.
//
// Literal scheme: two plain kernels (midpoints, nodes) with all of S inside
// the Lax-Wendroff stages, plus a one-CTA extraction kernel.
//
// Paper: Khanna & McKennon, arXiv:0909.4039, Sec. 2.2, Eqs. 9-14 and the
// boundary conditions stated after Eq. 14.
#include <math.h>

#include "teuk_internal.cuh"

namespace teuk {
namespace {

template <typename T> __device__ __forceinline__ T rcp_(T x);
template <> __device__ __forceinline__ float rcp_<float>(float x) { return __frcp_rn(x); }
template <> __device__ __forceinline__ double rcp_<double>(double x) { return __drcp_rn(x); }
template <typename T> __device__ __forceinline__ T sqrt_(T x);
template <> __device__ __forceinline__ float sqrt_<float>(float x) { return __fsqrt_rn(x); }
template <> __device__ __forceinline__ double sqrt_<double>(double x) { return __dsqrt_rn(x); }

template <typename C> __device__ __forceinline__ C cmk(decltype(C().x) a, decltype(C().x) b)
{
    C c;
    c.x = a;
    c.y = b;
    return c;
}
template <typename C> __device__ __forceinline__ C zero_c2()
{
    C c;
    c.x = 0;
    c.y = 0;
    return c;
}
template <typename C> __device__ __forceinline__ C cmul(C a, C b)
{
    return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C, typename T> __device__ __forceinline__ C cscale(T s, C a) { return cmk<C>(s * a.x, s * a.y); }
template <typename C, typename T> __device__ __forceinline__ C caxpy(T s, C a, C b)  // b + s a
{
    return cmk<C>(fma(s, a.x, b.x), fma(s, a.y, b.y));
}
template <typename C> __device__ __forceinline__ C cinv(C a)
{
    auto d = rcp_(a.x * a.x + a.y * a.y);
    return cmk<C>(a.x * d, -a.y * d);
}

// Local coefficients of the implicit part at node row (table f) and theta j.
template <typename T> struct Loc {
    typedef typename V2<T>::t c2;
    T q;      // Delta / Sigma^2
    c2 ct;    // c_t
    c2 c0;    // c0rad
    c2 a1;    // 1 + gh c_t
};

template <typename T>
__device__ __forceinline__ Loc<T> local_coef(T sg, const T *f, T C, T gh)
{
    typedef typename V2<T>::t c2;
    Loc<T> L;
    L.q = f[RF_DELTA] * sg;
    L.ct = cmk<c2>(sg * f[RF_CTR], sg * fma(f[RF_CTC], C, f[RF_CTI]));
    L.c0 = cmk<c2>(-sg * f[RF_C0R], -sg * f[RF_C0I]);
    L.a1 = cmk<c2>(fma(gh, L.ct.x, T(1)), gh * L.ct.y);
    return L;
}

// One implicit half step of length h = dt/2 on one r* row held in shared
// memory (phi, pi, sig: element j at [j]); f: the row's r table; th: theta
// tables; piv: pivots of this row (element j at piv[j * Nr]).
// SDIRK2: stage (I - gamma h J) U = (rPhi, rPi) is solved as
//   [(1 + gh c_t) + gh^2 (B + c0rad)] U_Phi = (1 + gh c_t) rPhi + gh rPi,
//   U_Pi = (rPi - gh (B + c0rad) U_Phi)/(1 + gh c_t),   B = q A_th,
// stage 1 with r = u, stage 2 with r = u + (1 - gamma) h J U1.  The stage-2
// right side uses u_Phi = U1_Phi - gh U1_Pi (stage-1 relation), so the
// original row need not be kept.
template <typename T>
__device__ void implicit_half_row(const StepParams<T> &p, typename V2<T>::t *phi,
                                  typename V2<T>::t *pi, const T *sig, const T *f,
                                  const T *th, const typename V2<T>::t *piv)
{
    typedef typename V2<T>::t c2;
    const int N = p.Nth;
    const size_t ps = (size_t)p.Nr;
    const T gh = p.gh, gh2 = p.gh2, h1g = p.h1g, h12g = p.h12g;
    const T *S2 = th + TF_S2 * N;
    (void)S2;
    const T *Cc = th + TF_C * N;
    const T *Am = th + TF_AM * N;
    const T *A0 = th + TF_A0 * N;
    const T *Ap = th + TF_AP * N;
    const c2 zero = cmk<c2>(T(0), T(0));

    // ---- stage 1, forward elimination: z_j = r_j - (sub_j e_{j-1}) z_{j-1}
    {
        c2 zprev = zero, eprev = zero;
        for (int j = 0; j < N; ++j) {
            Loc<T> L = local_coef<T>(sig[j], f, Cc[j], gh);
            c2 r = caxpy(gh, pi[j], cmul(L.a1, phi[j]));
            if (j > 0) {
                T sub = gh2 * L.q * Am[j];
                r = csub(r, cmul(cscale<c2>(sub, eprev), zprev));
            }
            phi[j] = r;
            zprev = r;
            eprev = piv[(size_t)j * ps];
        }
    }
    // ---- stage 1, back substitution; element jj = j + 1 is finished one
    // iteration late, once its three neighbours are known
    {
        c2 x2 = zero, x1 = zero, x0;   // x_{j+2}, x_{j+1}, x_j
        for (int j = N - 1; j >= -1; --j) {
            if (j >= 0) {
                Loc<T> L = local_coef<T>(sig[j], f, Cc[j], gh);
                c2 t = phi[j];
                if (j < N - 1) t = csub(t, cscale<c2>(gh2 * L.q * Ap[j], x1));
                x0 = cmul(t, piv[(size_t)j * ps]);
            } else {
                x0 = zero;
            }
            int jj = j + 1;
            if (jj <= N - 1) {
                Loc<T> L = local_coef<T>(sig[jj], f, Cc[jj], gh);
                // BF = (B + c0rad) U1_Phi at jj
                c2 bf = cscale<c2>(L.q, cadd(cadd(cscale<c2>(Am[jj], x0), cscale<c2>(A0[jj], x1)),
                                             cscale<c2>(Ap[jj], x2)));
                bf = cadd(bf, cmul(L.c0, x1));
                c2 P1 = cmul(csub(pi[jj], cscale<c2>(gh, bf)), cinv(L.a1));
                c2 rphi = caxpy(h12g, P1, x1);
                c2 rpi = csub(pi[jj], cscale<c2>(h1g, cadd(bf, cmul(L.ct, P1))));
                phi[jj] = caxpy(gh, rpi, cmul(L.a1, rphi));   // stage-2 right side
                pi[jj] = rpi;
            }
            x2 = x1;
            x1 = x0;
        }
    }
    // ---- stage 2, forward elimination
    {
        c2 zprev = zero, eprev = zero;
        for (int j = 0; j < N; ++j) {
            c2 r = phi[j];
            if (j > 0) {
                T q = f[RF_DELTA] * sig[j];
                r = csub(r, cmul(cscale<c2>(gh2 * q * Am[j], eprev), zprev));
            }
            phi[j] = r;
            zprev = r;
            eprev = piv[(size_t)j * ps];
        }
    }
    // ---- stage 2, back substitution and the Pi row
    {
        c2 x2 = zero, x1 = zero, x0;
        for (int j = N - 1; j >= -1; --j) {
            if (j >= 0) {
                T q = f[RF_DELTA] * sig[j];
                c2 t = phi[j];
                if (j < N - 1) t = csub(t, cscale<c2>(gh2 * q * Ap[j], x1));
                x0 = cmul(t, piv[(size_t)j * ps]);
            } else {
                x0 = zero;
            }
            int jj = j + 1;
            if (jj <= N - 1) {
                Loc<T> L = local_coef<T>(sig[jj], f, Cc[jj], gh);
                c2 bf = cscale<c2>(L.q, cadd(cadd(cscale<c2>(Am[jj], x0), cscale<c2>(A0[jj], x1)),
                                             cscale<c2>(Ap[jj], x2)));
                bf = cadd(bf, cmul(L.c0, x1));
                pi[jj] = cmul(csub(pi[jj], cscale<c2>(gh, bf)), cinv(L.a1));
                phi[jj] = x1;
            }
            x2 = x1;
            x1 = x0;
        }
    }
}

// b and K at one point from the r table f and theta tables (S2 = sin^2, C = cos).
template <typename T>
__device__ __forceinline__ void bK(const T *f, T sg, T S2, T C, T &b, typename V2<T>::t &K)
{
    b = f[RF_R] * sqrt_(sg);
    T kre = fma(b, f[RF_CTR], f[RF_CSR] - f[RF_E1]) + sg * fma(-f[RF_E3], S2, f[RF_E2]);
    T kim = fma(b, fma(f[RF_CTC], C, f[RF_CTI]), f[RF_CSI]);
    K.x = sg * kre;
    K.y = sg * kim;
}

template <typename T>
__device__ __forceinline__ typename V2<T>::t patch_val(const StepParams<T> &p, int gi, int pos, int j,
                                                        typename V2<T>::t phase)
{
    typedef typename V2<T>::t c2;
    int pr = gi - p.patch_p0;
    if (pr < 0 || pr >= p.patch_np) return cmk<c2>(T(0), T(0));
    c2 v = p.patch[((size_t)pr * 2 + pos) * p.Nth + j];
    return cmul(v, phase);
}

// Split-scheme Lax-Wendroff update of one theta column of the tile.
template <typename T>
__device__ void lw_column(const StepParams<T> &p, typename V2<T>::t *sPhi, typename V2<T>::t *sPi,
                          const T *sSig, const T *sRn, const T *sRh, const T *sTh, int j, int i0,
                          typename V2<T>::t ph1, typename V2<T>::t ph2, bool src)
{
    typedef typename V2<T>::t c2;
    const int N = p.Nth, P = p.pitch, TR = p.tile_rows, Nr = p.Nr;
    const T S2 = sTh[TF_S2 * N + j], C = sTh[TF_C * N + j];
    const T hdt = p.half_dt, dt = p.dt, ri = p.drs_inv;
    const c2 zero = cmk<c2>(T(0), T(0));

    // midpoint u*_{k+1/2} between tile rows k and k+1 (Eq. 13, S = F + K Phi_{r*})
    auto midpoint = [&](int k, c2 fa, c2 ga, c2 fb, c2 gb, c2 &mf, c2 &mg) {
        int gh_ = i0 - 1 + k;   // global i of the lower node
        if (gh_ < 0 || gh_ > Nr - 2) {
            mf = zero;
            mg = zero;
            return;
        }
        const T *f = sRh + k * NRF;
        T sg = rcp_(fma(-f[RF_AD], S2, f[RF_R2]));
        T b;
        c2 K;
        bK<T>(f, sg, S2, C, b, K);
        c2 fbar = cscale<c2>(T(0.5), cadd(fa, fb));
        c2 gbar = cscale<c2>(T(0.5), cadd(ga, gb));
        c2 df = cscale<c2>(ri, csub(fb, fa));
        c2 dg = cscale<c2>(ri, csub(gb, ga));
        c2 S = cmul(K, df);
        if (src) S = cadd(S, patch_val(p, gh_, 1, j, ph1));
        mf = csub(fbar, cscale<c2>(hdt * b, df));
        mg = cadd(gbar, cscale<c2>(hdt, cadd(cscale<c2>(b, dg), S)));
    };

    c2 fa = sPhi[j], ga = sPi[j];
    c2 fb = sPhi[P + j], gb = sPi[P + j];
    c2 mfp, mgp;
    midpoint(0, fa, ga, fb, gb, mfp, mgp);
    for (int lr = 1; lr <= TR; ++lr) {
        int gi = i0 + lr - 1;
        if (gi >= Nr) break;
        c2 fc = sPhi[(lr + 1) * P + j], gc = sPi[(lr + 1) * P + j];
        c2 mf, mg;
        midpoint(lr, fb, gb, fc, gc, mf, mg);
        c2 nf = zero, ng = zero;
        if (gi >= 1 && gi <= Nr - 2) {
            // Eq. 14 at node gi, S = F(t + dt/2) + K (u*_{i+1/2} - u*_{i-1/2})/dr*
            const T *f = sRn + lr * NRF;
            T sg = sSig[lr * P + j];
            T b;
            c2 K;
            bK<T>(f, sg, S2, C, b, K);
            c2 df = cscale<c2>(ri, csub(mf, mfp));
            c2 dg = cscale<c2>(ri, csub(mg, mgp));
            c2 S = cmul(K, df);
            if (src) S = cadd(S, patch_val(p, gi, 0, j, ph2));
            nf = csub(fb, cscale<c2>(dt * b, df));
            ng = cadd(gb, cscale<c2>(dt, cadd(cscale<c2>(b, dg), S)));
        }
        sPhi[lr * P + j] = nf;
        sPi[lr * P + j] = ng;
        fb = fc;
        gb = gc;
        mfp = mf;
        mgp = mg;
    }
}

__device__ __forceinline__ double2 phase_at(double mOmega, double t)
{
    double ph = mOmega * t;
    const double twopi = 2.0 * kPi;
    ph -= twopi * floor(ph / twopi);
    double s, c;
    sincos(ph, &s, &c);
    return make_double2(c, -s);   // e^{-i m Omega t}
}

template <typename T> __device__ __forceinline__ typename V2<T>::t from_d2(double2 v)
{
    typedef typename V2<T>::t c2;
    return cmk<c2>((T)v.x, (T)v.y);
}

// FP64 extraction of one row held anywhere (shared or global); one warp.
template <typename T>
__device__ void extract_warp(const StepParams<T> &p, const typename V2<T>::t *row, long long step)
{
    const int lane = threadIdx.x & 31;
    const int N = p.Nth;
    double sre = 0.0, sim = 0.0;
    for (int j = lane; j < N; j += 32) {
        double w = p.w[j];
        sre = fma(w, (double)row[j].x, sre);
        sim = fma(w, (double)row[j].y, sim);
    }
    for (int o = 16; o > 0; o >>= 1) {
        sre += __shfl_xor_sync(0xffffffffu, sre, o);
        sim += __shfl_xor_sync(0xffffffffu, sim, o);
    }
    long long slot = step % (long long)p.wave_cap;
    double2 *dst = p.wave + (size_t)slot * (size_t)(N + 1);
    if (lane == 0) {
        dst[0] = make_double2(sre, sim);
        if (!isfinite(sre) || !isfinite(sim)) atomicOr(&p.ctl->flags, FLAG_NONFINITE);
    }
    for (int j = lane; j < N; j += 32) dst[1 + j] = make_double2((double)row[j].x, (double)row[j].y);
}

template <typename T>
__global__ void __launch_bounds__(256) k_split_step(const StepParams<T> p)
{
    typedef typename V2<T>::t c2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double2 sph[2];
    __shared__ long long s_n;
    const int Nr = p.Nr, N = p.Nth, TR = p.tile_rows, R = TR + 2, P = p.pitch;
    const int tid = threadIdx.x, NT = blockDim.x;
    const int i0 = blockIdx.x * TR;

    c2 *sPhi = (c2 *)smem_raw;
    c2 *sPi = sPhi + R * P;
    T *sSig = (T *)(sPi + R * P);
    T *sRn = sSig + R * P;
    T *sRh = sRn + R * NRF;
    T *sTh = sRh + (R - 1) * NRF;

    const bool src = p.patch_np > 0 && i0 + TR >= p.patch_p0 && i0 - 1 <= p.patch_p0 + p.patch_np;
    if (tid == 0) {
        long long n = *((volatile long long *)&p.ctl->step);
        s_n = n;
        if (src) {
            double t = (double)n * p.dt64;
            sph[0] = phase_at(p.mOmega, t);
            sph[1] = phase_at(p.mOmega, t + 0.5 * p.dt64);
        }
    }
    // ---- A: tile load (rows i0-1 .. i0+TR), tables
    const c2 zero = cmk<c2>(T(0), T(0));
    for (int idx = tid; idx < R * N; idx += NT) {
        int lr = idx / N, j = idx - lr * N;
        int gi = i0 - 1 + lr;
        c2 f = zero, g = zero;
        if (gi >= 0 && gi < Nr) {
            f = p.uin[(size_t)gi * N + j];
            g = p.uin[((size_t)Nr + gi) * N + j];
        }
        sPhi[lr * P + j] = f;
        sPi[lr * P + j] = g;
    }
    for (int idx = tid; idx < R * NRF; idx += NT) {
        int lr = idx / NRF, q = idx - lr * NRF;
        int gi = i0 - 1 + lr;
        sRn[idx] = (gi >= 0 && gi < Nr) ? p.rtab[(size_t)(2 * gi) * NRF + q] : T(0);
    }
    for (int idx = tid; idx < (R - 1) * NRF; idx += NT) {
        int k = idx / NRF, q = idx - k * NRF;
        int gi = i0 - 1 + k;
        sRh[idx] = (gi >= 0 && gi <= Nr - 2) ? p.rtab[(size_t)(2 * gi + 1) * NRF + q] : T(0);
    }
    for (int idx = tid; idx < NTF * N; idx += NT) sTh[idx] = p.thtab[idx];
    __syncthreads();
    for (int idx = tid; idx < R * N; idx += NT) {
        int lr = idx / N, j = idx - lr * N;
        int gi = i0 - 1 + lr;
        T v = T(0);
        if (gi >= 0 && gi < Nr) v = rcp_(fma(-sRn[lr * NRF + RF_AD], sTh[TF_S2 * N + j], sRn[lr * NRF + RF_R2]));
        sSig[lr * P + j] = v;
    }
    __syncthreads();
    // ---- B: implicit half step on all tile rows (boundary rows become zero)
    if (tid < R) {
        int gi = i0 - 1 + tid;
        if (gi >= 1 && gi <= Nr - 2) {
            implicit_half_row<T>(p, sPhi + tid * P, sPi + tid * P, sSig + tid * P, sRn + tid * NRF, sTh,
                                 p.piv + gi);
        } else {
            for (int j = 0; j < N; ++j) {
                sPhi[tid * P + j] = zero;
                sPi[tid * P + j] = zero;
            }
        }
    }
    __syncthreads();
    // ---- C: Lax-Wendroff, one thread per theta column
    {
        c2 ph1 = zero, ph2 = zero;
        if (src) {
            ph1 = from_d2<T>(sph[0]);
            ph2 = from_d2<T>(sph[1]);
        }
        for (int j = tid; j < N; j += NT) lw_column<T>(p, sPhi, sPi, sSig, sRn, sRh, sTh, j, i0, ph1, ph2, src);
    }
    __syncthreads();
    // ---- D: implicit half step on the output rows
    if (tid < TR) {
        int lr = tid + 1;
        int gi = i0 + tid;
        if (gi >= 1 && gi <= Nr - 2)
            implicit_half_row<T>(p, sPhi + lr * P, sPi + lr * P, sSig + lr * P, sRn + lr * NRF, sTh,
                                 p.piv + gi);
    }
    __syncthreads();
    // ---- E: store, extraction, step counter
    for (int idx = tid; idx < TR * N; idx += NT) {
        int k = idx / N, j = idx - k * N;
        int gi = i0 + k;
        if (gi >= Nr) continue;
        p.uout[(size_t)gi * N + j] = sPhi[(k + 1) * P + j];
        p.uout[((size_t)Nr + gi) * N + j] = sPi[(k + 1) * P + j];
    }
    if (p.i_ext >= i0 && p.i_ext < i0 + TR && tid < 32)
        extract_warp<T>(p, sPhi + (p.i_ext - i0 + 1) * P, s_n + 1);
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        unsigned t = atomicAdd(&p.ctl->ticket, 1u);
        if (t == gridDim.x - 1) {
            p.ctl->step = s_n + 1;
            p.ctl->ticket = 0u;
            __threadfence();
        }
    }
}

// ------------------------------------------------------------ literal scheme

// S_Pi of the literal scheme at one point: all of Eq. 12,
//   F + K dPhi - c_t Pi - c0rad Phi - q (A_th Phi)_j.
template <typename T>
__device__ __forceinline__ typename V2<T>::t literal_SPi(const StepParams<T> &p, const T *f, const T *th,
                                                          int j, typename V2<T>::t phm,
                                                          typename V2<T>::t ph0, typename V2<T>::t php,
                                                          typename V2<T>::t pi0, typename V2<T>::t dphi, T &b)
{
    typedef typename V2<T>::t c2;
    const int N = p.Nth;
    T S2 = th[TF_S2 * N + j], C = th[TF_C * N + j];
    T sg = rcp_(fma(-f[RF_AD], S2, f[RF_R2]));
    c2 K;
    bK<T>(f, sg, S2, C, b, K);
    Loc<T> L = local_coef<T>(sg, f, C, p.gh);
    c2 aphi = cadd(cadd(cscale<c2>(th[TF_AM * N + j], phm), cscale<c2>(th[TF_A0 * N + j], ph0)),
                   cscale<c2>(th[TF_AP * N + j], php));
    c2 S = cmul(K, dphi);
    S = csub(S, cmul(L.ct, pi0));
    S = csub(S, cmul(L.c0, ph0));
    S = csub(S, cscale<c2>(L.q, aphi));
    return S;
}

template <typename T>
__global__ void k_literal_mid(const StepParams<T> p)
{
    typedef typename V2<T>::t c2;
    const int N = p.Nth, Nr = p.Nr;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (Nr - 1) * N) return;
    int i = idx / N, j = idx - i * N;
    long long n = *((volatile long long *)&p.ctl->step);
    const c2 *Phi = p.uin, *Pi = p.uin + (size_t)Nr * N;
    auto avg = [&](int jj) {
        return cscale<c2>(T(0.5), cadd(Phi[(size_t)i * N + jj], Phi[(size_t)(i + 1) * N + jj]));
    };
    c2 f0 = avg(j);
    c2 fm = (j > 0) ? avg(j - 1) : zero_c2<c2>();
    c2 fp = (j < N - 1) ? avg(j + 1) : zero_c2<c2>();
    c2 gbar = cscale<c2>(T(0.5), cadd(Pi[(size_t)i * N + j], Pi[(size_t)(i + 1) * N + j]));
    c2 df = cscale<c2>(p.drs_inv, csub(Phi[(size_t)(i + 1) * N + j], Phi[(size_t)i * N + j]));
    c2 dg = cscale<c2>(p.drs_inv, csub(Pi[(size_t)(i + 1) * N + j], Pi[(size_t)i * N + j]));
    const T *f = p.rtab + (size_t)(2 * i + 1) * NRF;
    T b;
    c2 S = literal_SPi<T>(p, f, p.thtab, j, fm, f0, fp, gbar, df, b);
    if (p.patch_np > 0) S = cadd(S, patch_val(p, i, 1, j, from_d2<T>(phase_at(p.mOmega, (double)n * p.dt64))));
    c2 *mPhi = p.mid, *mPi = p.mid + (size_t)(Nr - 1) * N;
    mPhi[idx] = cadd(f0, cscale<c2>(p.half_dt, csub(gbar, cscale<c2>(b, df))));
    mPi[idx] = cadd(gbar, cscale<c2>(p.half_dt, cadd(cscale<c2>(b, dg), S)));
}

template <typename T>
__global__ void k_literal_node(const StepParams<T> p)
{
    typedef typename V2<T>::t c2;
    const int N = p.Nth, Nr = p.Nr;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= Nr * N) return;
    int i = idx / N, j = idx - i * N;
    c2 *oPhi = p.uout, *oPi = p.uout + (size_t)Nr * N;
    if (i == 0 || i == Nr - 1) {
        oPhi[idx] = zero_c2<c2>();
        oPi[idx] = zero_c2<c2>();
        return;
    }
    long long n = *((volatile long long *)&p.ctl->step);
    const c2 *Phi = p.uin, *Pi = p.uin + (size_t)Nr * N;
    const c2 *mPhi = p.mid, *mPi = p.mid + (size_t)(Nr - 1) * N;
    auto avg = [&](int jj) {
        return cscale<c2>(T(0.5), cadd(mPhi[(size_t)i * N + jj], mPhi[(size_t)(i - 1) * N + jj]));
    };
    c2 f0 = avg(j);
    c2 fm = (j > 0) ? avg(j - 1) : zero_c2<c2>();
    c2 fp = (j < N - 1) ? avg(j + 1) : zero_c2<c2>();
    c2 gt = cscale<c2>(T(0.5), cadd(mPi[(size_t)i * N + j], mPi[(size_t)(i - 1) * N + j]));
    c2 df = cscale<c2>(p.drs_inv, csub(mPhi[(size_t)i * N + j], mPhi[(size_t)(i - 1) * N + j]));
    c2 dg = cscale<c2>(p.drs_inv, csub(mPi[(size_t)i * N + j], mPi[(size_t)(i - 1) * N + j]));
    const T *f = p.rtab + (size_t)(2 * i) * NRF;
    T b;
    c2 S = literal_SPi<T>(p, f, p.thtab, j, fm, f0, fp, gt, df, b);
    if (p.patch_np > 0)
        S = cadd(S, patch_val(p, i, 0, j, from_d2<T>(phase_at(p.mOmega, (double)n * p.dt64 + 0.5 * p.dt64))));
    oPhi[idx] = cadd(Phi[idx], cscale<c2>(p.dt, csub(gt, cscale<c2>(b, df))));
    oPi[idx] = cadd(Pi[idx], cscale<c2>(p.dt, cadd(cscale<c2>(b, dg), S)));
}

// Extraction of a state's row into the ring buffer; optionally advances the
// device step counter (literal scheme, after its node kernel).
template <typename T>
__global__ void k_extract(const StepParams<T> p, const typename V2<T>::t *u, long long step, int advance)
{
    long long n = step;
    if (step < 0) n = *((volatile long long *)&p.ctl->step) + 1;
    extract_warp<T>(p, u + (size_t)p.i_ext * p.Nth, n);
    if (advance && threadIdx.x == 0) p.ctl->step = n;
}

__global__ void k_to_f32(const double2 *src, float2 *dst, size_t n)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}
__global__ void k_from_f32(const float2 *src, double2 *dst, size_t n)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = make_double2((double)src[i].x, (double)src[i].y);
}

}  // namespace

template <typename T>
size_t split_smem_bytes(int tile_rows, int Nth)
{
    size_t R = (size_t)tile_rows + 2, P = (size_t)Nth + 1;
    return R * P * (2 * sizeof(typename V2<T>::t) + sizeof(T)) + (R + (R - 1)) * NRF * sizeof(T) +
           (size_t)NTF * Nth * sizeof(T);
}

template <typename T>
cudaError_t launch_split_step(const StepParams<T> &p, int threads, size_t smem, cudaStream_t st)
{
    // opt in to the dynamic shared memory this launch needs (once per size)
    static size_t configured[2] = {0, 0};
    int key = sizeof(T) == 4 ? 0 : 1;
    if (smem > configured[key]) {
        cudaError_t e = cudaFuncSetAttribute(k_split_step<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured[key] = smem;
    }
    int grid = (p.Nr + p.tile_rows - 1) / p.tile_rows;
    k_split_step<T><<<grid, threads, smem, st>>>(p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_literal_step(const StepParams<T> &p, cudaStream_t st)
{
    int nm = (p.Nr - 1) * p.Nth, nn = p.Nr * p.Nth;
    k_literal_mid<T><<<(nm + 255) / 256, 256, 0, st>>>(p);
    k_literal_node<T><<<(nn + 255) / 256, 256, 0, st>>>(p);
    k_extract<T><<<1, 32, 0, st>>>(p, p.uout, -1, 1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_extract(const StepParams<T> &p, const typename V2<T>::t *u, long long step, cudaStream_t st)
{
    k_extract<T><<<1, 32, 0, st>>>(p, u, step, 0);
    return cudaGetLastError();
}

cudaError_t launch_convert_to(int prec, const double2 *src, void *dst, size_t n, cudaStream_t st)
{
    if (prec == TEUK_FP64) return cudaMemcpyAsync(dst, src, n * sizeof(double2), cudaMemcpyDeviceToDevice, st);
    k_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, (float2 *)dst, n);
    return cudaGetLastError();
}

cudaError_t launch_convert_from(int prec, const void *src, double2 *dst, size_t n, cudaStream_t st)
{
    if (prec == TEUK_FP64) return cudaMemcpyAsync(dst, src, n * sizeof(double2), cudaMemcpyDeviceToDevice, st);
    k_from_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const float2 *)src, dst, n);
    return cudaGetLastError();
}

template size_t split_smem_bytes<float>(int, int);
template size_t split_smem_bytes<double>(int, int);
template cudaError_t launch_split_step<float>(const StepParams<float> &, int, size_t, cudaStream_t);
template cudaError_t launch_split_step<double>(const StepParams<double> &, int, size_t, cudaStream_t);
template cudaError_t launch_literal_step<float>(const StepParams<float> &, cudaStream_t);
template cudaError_t launch_literal_step<double>(const StepParams<double> &, cudaStream_t);
template cudaError_t launch_extract<float>(const StepParams<float> &, const float2 *, long long, cudaStream_t);
template cudaError_t launch_extract<double>(const StepParams<double> &, const double2 *, long long, cudaStream_t);

}  // namespace teuk
