// teuk_dev.cuh -- device code shared by the step kernels of libteuk:
// complex and packed FP32 arithmetic, vector moves, the implicit (SDIRK2)
// row solves, the Lax-Wendroff stages, bulk copies with bounded mbarrier
// waits, extraction, and the per-tile body of the split-scheme kernels.
// Every translation unit that includes it gets its own copy (internal
// linkage); the kernels themselves are defined in the .cu files.
//
// Paper: Khanna & McKennon, arXiv:0909.4039, Sec. 2.2, Eqs. 9-14 and the
// boundary conditions stated after Eq. 14.
#pragma once

#include <math.h>
#include <stdio.h>

#include <mutex>
#include <utility>
#include <vector>

#include "teuk_internal.cuh"

namespace teuk {
namespace {

// 1/x and 1/sqrt(x) for coefficients: the hardware approximations in FP32
// (relative error a few units in the last place, far below the FP32 state's
// own rounding over a step), correctly rounded operations in FP64.
template <typename T> __device__ __forceinline__ T rcp_fast(T x);
template <> __device__ __forceinline__ float rcp_fast<float>(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <> __device__ __forceinline__ double rcp_fast<double>(double x) { return __drcp_rn(x); }
template <typename T> __device__ __forceinline__ T rsq_(T x);
template <> __device__ __forceinline__ float rsq_<float>(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <> __device__ __forceinline__ double rsq_<double>(double x) { return __drcp_rn(__dsqrt_rn(x)); }

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
// Every sum of two products below is written with one explicit fma.  Left
// to the compiler, a*b + c*d may fuse either product, and which one it fuses
// depends on the code around the inlined call; kernels that share these
// helpers (one to three steps per launch, batched, persistent) then round the
// same expression differently.  With the fusion fixed they agree bit for bit.
template <typename C> __device__ __forceinline__ C cmul(C a, C b)
{
    return cmk<C>(fma(a.x, b.x, -(a.y * b.y)), fma(a.x, b.y, a.y * b.x));
}
// c + a b
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C c)
{
    return cmk<C>(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// c - a b
template <typename C> __device__ __forceinline__ C cfnma(C a, C b, C c)
{
    return cmk<C>(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C, typename T> __device__ __forceinline__ C cscale(T s, C a) { return cmk<C>(s * a.x, s * a.y); }
template <typename C, typename T> __device__ __forceinline__ C caxpy(T s, C a, C b)  // b + s a
{
    return cmk<C>(fma(s, a.x, b.x), fma(s, a.y, b.y));
}
// FP32 specialisations on packed pairs (add/sub/mul/fma .f32x2 of the
// sm_100 family): one instruction for both components, each lane rounded
// exactly as the scalar operation, so results do not change.  The complex
// multiply keeps scalar fmas: its packed form needs swapped and negated
// operand pairs, which cost more moves than the packing saves.
__device__ __forceinline__ unsigned long long pk2(float x, float y)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r)
{
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a.x, a.y)), "l"(pk2(b.x, b.y)));
    return upk2(d);
}
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a.x, a.y)), "l"(pk2(b.x, b.y)));
    return upk2(d);
}
template <> __device__ __forceinline__ float2 cscale<float2, float>(float s, float2 a)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(s, s)), "l"(pk2(a.x, a.y)));
    return upk2(d);
}
template <> __device__ __forceinline__ float2 caxpy<float2, float>(float s, float2 a, float2 b)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk2(s, s)), "l"(pk2(a.x, a.y)), "l"(pk2(b.x, b.y)));
    return upk2(d);
}
template <typename C> __device__ __forceinline__ C cinv(C a)
{
    auto d = rcp_fast(fma(a.x, a.x, a.y * a.y));
    return cmk<C>(a.x * d, -a.y * d);
}

// ---- 16-byte vector moves between registers and memory.  The address
// must be 16-byte aligned; S * sizeof(V) must be a multiple of 16.
template <typename V> struct Q16;
template <> struct Q16<float> { typedef float4 t; };
template <> struct Q16<float2> { typedef float4 t; };
template <> struct Q16<double> { typedef double2 t; };
template <> struct Q16<double2> { typedef double2 t; };
__device__ __forceinline__ void unpack16(const float4 &v, float *r) { r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w; }
__device__ __forceinline__ void unpack16(const float4 &v, float2 *r)
{
    r[0] = make_float2(v.x, v.y);
    r[1] = make_float2(v.z, v.w);
}
__device__ __forceinline__ void unpack16(const double2 &v, double *r) { r[0] = v.x; r[1] = v.y; }
__device__ __forceinline__ void unpack16(const double2 &v, double2 *r) { r[0] = v; }
__device__ __forceinline__ float4 pack16(const float2 *r) { return make_float4(r[0].x, r[0].y, r[1].x, r[1].y); }
__device__ __forceinline__ double2 pack16(const double2 *r) { return r[0]; }

template <int S, typename V> __device__ __forceinline__ void vload(V *r, const V *src)
{
    typedef typename Q16<V>::t Q;
    constexpr int per = (int)(16 / sizeof(V));
    static_assert(S % per == 0, "vector load of a partial 16-byte chunk");
    const Q *q = reinterpret_cast<const Q *>(src);
#pragma unroll
    for (int i = 0; i < S / per; ++i) unpack16(q[i], r + i * per);
}
template <int S, typename V> __device__ __forceinline__ void vstore(V *dst, const V *r)
{
    typedef typename Q16<V>::t Q;
    constexpr int per = (int)(16 / sizeof(V));
    static_assert(S % per == 0, "vector store of a partial 16-byte chunk");
    Q *q = reinterpret_cast<Q *>(dst);
#pragma unroll
    for (int i = 0; i < S / per; ++i) q[i] = pack16(r + i * per);
}

// a / b for a >= 0, b > 0: a shift when b is a power of two (theta counts
// and lane groups usually are), else an unsigned division, which is
// shorter than the signed one.
__device__ __forceinline__ int udiv(int a, int b)
{
    if ((b & (b - 1)) == 0) return a >> (__ffs(b) - 1);
    return (int)((unsigned)a / (unsigned)b);
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

template <typename C> __device__ __forceinline__ C shfl_up_c(C v, int d, int w)
{
    v.x = __shfl_up_sync(0xffffffffu, v.x, d, w);
    v.y = __shfl_up_sync(0xffffffffu, v.y, d, w);
    return v;
}
template <typename C> __device__ __forceinline__ C shfl_down_c(C v, int d, int w)
{
    v.x = __shfl_down_sync(0xffffffffu, v.x, d, w);
    v.y = __shfl_down_sync(0xffffffffu, v.y, d, w);
    return v;
}

// Magnitude below which a scan multiplier is dropped: far below the unit
// roundoff of the state precision (2^-24 in FP32, 2^-53 in FP64).
template <typename T> struct ScanTol;
template <> struct ScanTol<float> { static constexpr float v = 1e-10f; };
template <> struct ScanTol<double> { static constexpr double v = 1e-19; };

// One implicit SDIRK2 step of length h (constants K) on one r* row held in
// shared memory (phi, pi: element j at [j]; prow: the row's Thomas pivots,
// shared or global; f: the row's r-table entry, 16-byte aligned; th: theta
// tables), by a group of G consecutive lanes.
// Lane g holds the contiguous theta segment [g S, g S + S) in registers;
// with vec every segment is whole and 16-byte aligned and moves by vector
// loads and stores.
//
// Stage (I - gamma h J) U = (rPhi, rPi), J u = (Pi, -(B + c0rad) Phi - c_t Pi),
// B = q A_th, is solved as
//   [(1 + gh c_t) + gh^2 (B + c0rad)] U_Phi = (1 + gh c_t) rPhi + gh rPi,
//   U_Pi = (rPi - gh (B + c0rad) U_Phi) / (1 + gh c_t);
// stage 1 with r = u, stage 2 with r = u + (1 - gamma) h J U1, u^new = U2.
// The tridiagonal solve uses the FP64-generated LU pivots e_j = 1/d_j:
//   forward   z_j = r_j - m_j z_{j-1},  m_j = sub_j e_{j-1}
//   backward  x_j = e_j z_j - f_j x_{j+1},  f_j = e_j sup_j.
// Both are first-order affine recurrences.  Each lane composes the affine
// map of its segment; the maps are scanned across the G lanes with
// shuffles (Kogge-Stone, log2 G levels) and each lane then runs its segment
// from the incoming value.  The multiplicative part of every map depends
// only on the matrix, so it is scanned once per call and both stages scan
// only the additive part.  Rows with active == false (boundary or outside
// the grid) take part in the shuffles with neutral data and write zeros.
// Per-element coefficients of one row's implicit stage (lane segment of S
// elements): LU pivots e, forward multipliers m_j = sub_j e_{j-1}, backward
// multipliers fk_j = e_j sup_j, c_t, row j of B + c0rad as (qam, dg, qap),
// and 1/(1 + gh c_t).  Loaded together with the lane's (Phi, Pi) segment.
template <typename T, int S> struct RowCoef {
    typedef typename V2<T>::t c2;
    c2 e[S], m[S], fk[S], ct[S], dg[S], ia1[S];
    T qam[S], qap[S];
};

// Elements past the end of the row (and every element of an inactive row)
// are neutral: sigma = 0 (so q = c_t = c0rad = 0), zero data, e = 1, zero
// angular row.  Padded elements only follow the real ones of a segment and
// only feed lanes that hold no real element, so the recurrences need no
// bounds tests, and a neutral row maps to zero.
template <typename T, int S>
__device__ __forceinline__ void row_load(const ImpConst<T> &K, const typename V2<T>::t *phi,
                                         const typename V2<T>::t *pi, const typename V2<T>::t *prow, const T *f,
                                         const T *th, int N, int len, int j0, int G, bool vec, RowCoef<T, S> &C,
                                         typename V2<T>::t (&w)[S], typename V2<T>::t (&y)[S])
{
    typedef typename V2<T>::t c2;
    const c2 zero = cmk<c2>(T(0), T(0));
    const c2 one = cmk<c2>(T(1), T(0));
    const T gh = K.gh, gh2 = K.gh2;
    T fr[NRF];
    vload<NRF>(fr, f);
    const T D = fr[RF_DELTA], ctr = fr[RF_CTR], cti = fr[RF_CTI], ctc = fr[RF_CTC], c0r = fr[RF_C0R],
            c0i = fr[RF_C0I], R2 = fr[RF_R2], AD = fr[RF_AD];
    const T *S2t = th + TF_S2 * N;
    const T *Cc = th + TF_C * N;
    const T *Am = th + TF_AM * N;
    const T *A0 = th + TF_A0 * N;
    const T *Ap = th + TF_AP * N;

    // rsv = 1/Sigma (zero for neutral elements)
    T rsv[S], ccv[S], am[S], a0[S], ap[S];
    if (vec && len == S) {
        T s2v[S];
        vload<S>(s2v, S2t + j0);
        vload<S>(ccv, Cc + j0);
        vload<S>(am, Am + j0);
        vload<S>(a0, A0 + j0);
        vload<S>(ap, Ap + j0);
        vload<S>(C.e, prow + j0);
        vload<S>(w, phi + j0);
        vload<S>(y, pi + j0);
#pragma unroll
        for (int k = 0; k < S; ++k) rsv[k] = rsq_(fma(-AD, s2v[k], R2));
    } else {
#pragma unroll
        for (int k = 0; k < S; ++k) {
            const bool real = k < len;
            const int j = real ? j0 + k : 0;
            rsv[k] = real ? rsq_(fma(-AD, S2t[j], R2)) : T(0);
            ccv[k] = real ? Cc[j] : T(0);
            am[k] = real ? Am[j] : T(0);
            a0[k] = real ? A0[j] : T(0);
            ap[k] = real ? Ap[j] : T(0);
            C.e[k] = real ? prow[j] : one;
            w[k] = real ? phi[j] : zero;
            y[k] = real ? pi[j] : zero;
        }
    }
    // Row j of B + c0rad is (qam_j, dg_j, qap_j) = (q AM_j, q A0_j + c0rad_j, q AP_j).
#pragma unroll
    for (int k = 0; k < S; ++k) {
        const T sg = rsv[k] * rsv[k];
        const T q = D * sg;
        C.ct[k] = cmk<c2>(sg * ctr, sg * fma(ctc, ccv[k], cti));
        C.dg[k] = cmk<c2>(fma(q, a0[k], -sg * c0r), -sg * c0i);
        C.qam[k] = q * am[k];
        C.qap[k] = q * ap[k];
        C.ia1[k] = cinv(cmk<c2>(fma(gh, C.ct[k].x, T(1)), gh * C.ct[k].y));
    }
    const c2 e_prev = shfl_up_c(C.e[S - 1], 1, G);   // e_{j0-1} (lane g-1 holds a full segment)
#pragma unroll
    for (int k = 0; k < S; ++k) {
        C.m[k] = cscale<c2>(gh2 * C.qam[k], k ? C.e[k - 1] : e_prev);
        C.fk[k] = cscale<c2>(gh2 * C.qap[k], C.e[k]);
    }
}

// Scan plan of a pair of first-order affine recurrences over one row
//   forward  t_j = r_j - fm_j t_{j-1},   backward  x_j = y_j - bm_j x_{j+1}:
// Af0, Ab0 are the multiplicative parts of the lane's segment maps.  Level l
// of a scan adds, to each lane's value, a neighbour's value times that
// level's multiplier (the product of the segment multipliers it spans).
// Once every multiplier of a level is below ScanTol in magnitude the level
// adds nothing the state precision can hold, and neither do the levels
// above it (their multipliers are products of these), so the scans stop
// there: nf levels forward, nb backward.  The test is taken over this row's
// group of G lanes only, so a row's result does not depend on the rows that
// share its warp; the shuffles run for the levels any group of the warp
// needs (nfw, nbw).  The data scans recompute the multipliers of the levels
// they use instead of keeping one per level in registers.
template <typename T> struct ScanPlan {
    typename V2<T>::t Af0, Ab0;
    int nf, nb, nfw, nbw;
};

template <typename T, int S>
__device__ __forceinline__ ScanPlan<T> scan_plan(const typename V2<T>::t (&fm)[S], const typename V2<T>::t (&bm)[S],
                                                 int g, int G)
{
    typedef typename V2<T>::t c2;
    constexpr int LOGMAX = 5;
    const c2 one = cmk<c2>(T(1), T(0));
    ScanPlan<T> P;
    P.Af0 = one;
    P.Ab0 = one;
    P.nf = P.nb = P.nfw = P.nbw = 0;
#pragma unroll
    for (int k = 0; k < S; ++k) P.Af0 = cmul(cmk<c2>(-fm[k].x, -fm[k].y), P.Af0);
#pragma unroll
    for (int k = S - 1; k >= 0; --k) P.Ab0 = cmul(cmk<c2>(-bm[k].x, -bm[k].y), P.Ab0);
    const T tol2 = ScanTol<T>::v * ScanTol<T>::v;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned gbase = lane - (unsigned)g;
    const unsigned gmask = G >= 32 ? 0xffffffffu : ((1u << G) - 1u);
    c2 Af = P.Af0, Ab = P.Ab0;
    bool gf = true, gb = true;
#pragma unroll
    for (int l = 0; l < LOGMAX; ++l) {
        const int d = 1 << l;
        if (d >= G) break;
        const unsigned bf = __ballot_sync(0xffffffffu, g >= d && fma(Af.x, Af.x, Af.y * Af.y) > tol2);
        const unsigned bb = __ballot_sync(0xffffffffu, g + d < G && fma(Ab.x, Ab.x, Ab.y * Ab.y) > tol2);
        gf = gf && ((bf >> gbase) & gmask) != 0u;
        gb = gb && ((bb >> gbase) & gmask) != 0u;
        const bool wf = __any_sync(0xffffffffu, gf), wb = __any_sync(0xffffffffu, gb);
        if (!wf && !wb) break;
        if (gf) P.nf = l + 1;
        if (gb) P.nb = l + 1;
        if (wf) P.nfw = l + 1;
        if (wb) P.nbw = l + 1;
        if (2 * d >= G) break;
        const c2 Ao = shfl_up_c(Af, d, G), Bo = shfl_down_c(Ab, d, G);
        if (gf && g >= d) Af = cmul(Af, Ao);
        if (gb && g + d < G) Ab = cmul(Ab, Bo);
    }
    return P;
}

// The same plan from the stored levels of the row (forward | backward << 8,
// computed once by scan_plan in k_scan_plans); the levels are a function
// of the row's coefficients alone, so the stored and the recomputed plans
// agree.  Every lane of the warp calls this (warp-wide level counts).
template <typename T, int S>
__device__ __forceinline__ ScanPlan<T> scan_plan_stored(const typename V2<T>::t (&fm)[S],
                                                        const typename V2<T>::t (&bm)[S], int plan)
{
    typedef typename V2<T>::t c2;
    ScanPlan<T> P;
    P.Af0 = cmk<c2>(T(1), T(0));
    P.Ab0 = P.Af0;
#pragma unroll
    for (int k = 0; k < S; ++k) P.Af0 = cmul(cmk<c2>(-fm[k].x, -fm[k].y), P.Af0);
#pragma unroll
    for (int k = S - 1; k >= 0; --k) P.Ab0 = cmul(cmk<c2>(-bm[k].x, -bm[k].y), P.Ab0);
    P.nf = plan & 0xff;
    P.nb = (plan >> 8) & 0xff;
    P.nfw = (int)__reduce_max_sync(0xffffffffu, (unsigned)P.nf);
    P.nbw = (int)__reduce_max_sync(0xffffffffu, (unsigned)P.nb);
    return P;
}

// w <- x with forward t_j = w_j - fm_j t_{j-1} (t_{-1} = 0), y_j = pm_j t_j,
// backward x_j = y_j - bm_j x_{j+1} (x_N = 0), each affine recurrence as a
// segmented scan over the G lanes of the row.  The scan levels run in a
// rolled loop over the planned count (usually one): five unrolled levels
// behind runtime guards cost about 8 % of a step.
template <typename T, int S>
__device__ __forceinline__ void seg_solve(typename V2<T>::t (&w)[S], const typename V2<T>::t (&fm)[S],
                                          const typename V2<T>::t (&pm)[S], const typename V2<T>::t (&bm)[S],
                                          const ScanPlan<T> &P, int g, int G)
{
    typedef typename V2<T>::t c2;
    const c2 zero = cmk<c2>(T(0), T(0));
    const c2 one = cmk<c2>(T(1), T(0));
    c2 B = zero;
#pragma unroll
    for (int k = 0; k < S; ++k) B = cfnma(fm[k], B, w[k]);
    {
        c2 A = P.Af0;
#pragma unroll 1
        for (int l = 0; l < P.nfw; ++l) {
            const int d = 1 << l;
            c2 Bo = shfl_up_c(B, d, G), Ao = one;
            if (l + 1 < P.nfw) Ao = shfl_up_c(A, d, G);
            if (l < P.nf && g >= d) {
                B = cfma(A, Bo, B);
                if (l + 1 < P.nf) A = cmul(A, Ao);
            }
        }
    }
    c2 z = shfl_up_c(B, 1, G);
    if (g == 0) z = zero;
#pragma unroll
    for (int k = 0; k < S; ++k) {
        z = cfnma(fm[k], z, w[k]);
        w[k] = cmul(pm[k], z);
    }
    B = zero;
#pragma unroll
    for (int k = S - 1; k >= 0; --k) B = cfnma(bm[k], B, w[k]);
    {
        c2 A = P.Ab0;
#pragma unroll 1
        for (int l = 0; l < P.nbw; ++l) {
            const int d = 1 << l;
            c2 Bo = shfl_down_c(B, d, G), Ao = one;
            if (l + 1 < P.nbw) Ao = shfl_down_c(A, d, G);
            if (l < P.nb && g + d < G) {
                B = cfma(A, Bo, B);
                if (l + 1 < P.nb) A = cmul(A, Ao);
            }
        }
    }
    c2 x = shfl_down_c(B, 1, G);
    if (g == G - 1) x = zero;
#pragma unroll
    for (int k = S - 1; k >= 0; --k) {
        x = cfnma(bm[k], x, w[k]);
        w[k] = x;
    }
}

// Writes a lane's segment back (real elements only).
template <typename T, int S>
__device__ __forceinline__ void row_store(typename V2<T>::t *phi, typename V2<T>::t *pi,
                                          const typename V2<T>::t (&w)[S], const typename V2<T>::t (&y)[S], int j0,
                                          int lenw, bool vec)
{
    if (lenw <= 0) return;
    if (vec) {
        vstore<S>(phi + j0, w);
        vstore<S>(pi + j0, y);
    } else {
#pragma unroll
        for (int k = 0; k < S; ++k) {
            if (k < lenw) {
                phi[j0 + k] = w[k];
                pi[j0 + k] = y[k];
            }
        }
    }
}

// plan: the row's stored scan levels (K.plan), 0 for a row that is not active.
template <typename T, int S>
__device__ void implicit_row_group(const ImpConst<T> &K, typename V2<T>::t *phi, typename V2<T>::t *pi,
                                   const typename V2<T>::t *prow, const T *f, const T *th, int N, bool active,
                                   bool in_tile, int g, int G, bool vec, int plan)
{
    typedef typename V2<T>::t c2;
    const c2 zero = cmk<c2>(T(0), T(0));
    const int j0 = g * S;
    int len = N - j0;
    len = len < 0 ? 0 : (len > S ? S : len);
    const int lenw = len;          // real elements of the segment (written back)
    if (!active) len = 0;
    const T gh = K.gh;
    RowCoef<T, S> C;
    c2 w[S], y[S];
    row_load<T, S>(K, phi, pi, prow, f, th, N, len, j0, G, vec, C, w, y);
    const ScanPlan<T> P = scan_plan_stored<T, S>(C.m, C.fk, active ? plan : 0);

    // (B + c0rad) U_Phi for the whole segment
    auto apply_B = [&](c2 *bf) {
        c2 xl = shfl_up_c(w[S - 1], 1, G), xr = shfl_down_c(w[0], 1, G);
        if (g == 0) xl = zero;
        if (g == G - 1) xr = zero;
#pragma unroll
        for (int k = 0; k < S; ++k) {
            c2 xm = k ? w[k - 1] : xl;
            c2 xp = (k + 1 < S) ? w[(k + 1) < S ? k + 1 : S - 1] : xr;
            bf[k] = cfma(C.dg[k], w[k], caxpy(C.qap[k], xp, cscale<c2>(C.qam[k], xm)));
        }
    };

    // ---- stage 1: r = (1 + gh c_t) Phi + gh Pi
#pragma unroll
    for (int k = 0; k < S; ++k) {
        c2 a1 = cmk<c2>(fma(gh, C.ct[k].x, T(1)), gh * C.ct[k].y);
        w[k] = caxpy(gh, y[k], cmul(a1, w[k]));
    }
    seg_solve<T, S>(w, C.m, C.e, C.fk, P, g, G);
    {
        c2 bf[S];
        apply_B(bf);
#pragma unroll
        for (int k = 0; k < S; ++k) {
            c2 a1 = cmk<c2>(fma(gh, C.ct[k].x, T(1)), gh * C.ct[k].y);
            c2 P1 = cmul(caxpy(-gh, bf[k], y[k]), C.ia1[k]);
            c2 rphi = caxpy(K.h12g, P1, w[k]);                     // U1_Phi + (1 - 2 gamma) h U1_Pi
            c2 rpi = caxpy(-K.h1g, cfma(C.ct[k], P1, bf[k]), y[k]);
            w[k] = caxpy(gh, rpi, cmul(a1, rphi));
            y[k] = rpi;
        }
    }
    // ---- stage 2
    seg_solve<T, S>(w, C.m, C.e, C.fk, P, g, G);
    {
        c2 bf[S];
        apply_B(bf);
#pragma unroll
        for (int k = 0; k < S; ++k) y[k] = cmul(caxpy(-gh, bf[k], y[k]), C.ia1[k]);
    }
    if (in_tile) row_store<T, S>(phi, pi, w, y, j0, lenw, vec);
}

// ---- Forward implicit step, as the step kernels apply it.
//
// The SDIRK2 step of implicit_row_group, evaluated with less arithmetic.
// With W = B + c0rad (tridiagonal in theta: q AM, q A0 + c0rad, q AP) the
// stage equations (I - gamma h J) U = r, J u = (Pi, -W Phi - c_t Pi), are
// solved for the Pi component first:
//   M U_Pi = r_Pi - gh W r_Phi,   U_Phi = r_Phi + gh U_Pi,
//   M = (1 + gh c_t) + gh^2 W
// (substitute U_Phi into the Pi row).  Stage 1 has r = u; stage 2 has
// r = u + (1 - gamma) h J U1, and with Wu = W u_Phi, Y = W U1_Pi (so that
// W U1_Phi = Wu + gh Y and W r2_Phi = Wu + (1 - gamma) h Y) its right side
// and result are
//   M U2_Pi = u_Pi - h Wu - 2 gamma (1 - gamma) h^2 Y - (1 - gamma) h c_t U1_Pi,
//   U2_Phi  = u_Phi + (1 - gamma) h U1_Pi + gh U2_Pi.
// Two products with W per step, no division by 1 + gh c_t.  M = L U with
// the FP64-generated pivots e_j = 1/d_j is solved as
//   forward   z_j = e_j (r_j - sub_j z_{j-1}),   sub_j = gh^2 q AM_j,
//   backward  x_j = z_j - fk_j x_{j+1},          fk_j  = e_j gh^2 q AP_j,
// each a segmented scan over the G lanes of the row (as seg_solve).

// Per-element coefficients of one row's implicit step (lane segment of S).
template <typename T, int S> struct ImpCoef {
    typedef typename V2<T>::t c2;
    c2 e[S];            // LU pivots of M
    c2 fk[S];           // backward multipliers
    c2 dg[S];           // diagonal of W
    c2 ct[S];           // (1 - gamma) h c_t
    T sub[S];           // subdiagonal of M
    T qam[S], qap[S];   // off-diagonals of W
};

// Row constants of the implicit step from the row's step-table entry f
// (SField, implicit block); c_t's factors carry (1 - gamma) h.
template <typename T> struct ImpRow {
    T R2, AD, D, ctr, cti, ctc, c0r, c0i;
};
template <typename T>
__device__ __forceinline__ ImpRow<T> imp_row(const ImpConst<T> &K, const T *f)
{
    T fr[8];
    vload<8>(fr, f);
    ImpRow<T> r;
    r.R2 = fr[SF_R2];
    r.AD = fr[SF_AD];
    r.D = fr[SF_DELTA];
    r.ctr = K.h1g * fr[SF_CTR];
    r.cti = K.h1g * fr[SF_CTI];
    r.ctc = K.h1g * fr[SF_CTC];
    r.c0r = fr[SF_C0R];
    r.c0i = fr[SF_C0I];
    return r;
}
// 1/Sigma^2 at one element (sin^2 theta = s2)
template <typename T>
__device__ __forceinline__ T imp_sg(const ImpRow<T> &r, T s2) { return rcp_fast(fma(-r.AD, s2, r.R2)); }
// The coefficients of one element from sg = 1/Sigma^2, cos theta, the
// angular row (am, a0, ap) and the pivot e.  The materialised planes of the
// FP64 path (k_mat_coef) are made by this same function.
template <typename T>
__device__ __forceinline__ void imp_elem(const ImpConst<T> &K, const ImpRow<T> &r, T sg, T cc, T am, T a0, T ap,
                                         typename V2<T>::t e, typename V2<T>::t &ct, typename V2<T>::t &dg, T &qam,
                                         T &qap, T &sub, typename V2<T>::t &fk)
{
    typedef typename V2<T>::t c2;
    const T q = r.D * sg;
    ct = cmk<c2>(sg * r.ctr, sg * fma(r.ctc, cc, r.cti));
    dg = cmk<c2>(fma(q, a0, -(sg * r.c0r)), -(sg * r.c0i));
    qam = q * am;
    qap = q * ap;
    sub = K.gh2 * qam;
    fk = cscale<c2>(K.gh2 * qap, e);
}

// Loads the lane's segment (state, pivots, theta tables) and forms the
// coefficients; f is the row's step-table entry (SField, implicit block).
// Elements past the end of the row and every element of an inactive row
// are neutral (zero data, e = 1, zero W and c_t), as in row_load.
template <typename T, int S>
__device__ __forceinline__ void imp_load(const ImpConst<T> &K, const typename V2<T>::t *phi,
                                         const typename V2<T>::t *pi, const typename V2<T>::t *prow, const T *f,
                                         const T *th, int N, int len, int j0, bool vec, ImpCoef<T, S> &C,
                                         typename V2<T>::t (&w)[S], typename V2<T>::t (&y)[S])
{
    typedef typename V2<T>::t c2;
    const c2 zero = cmk<c2>(T(0), T(0));
    const c2 one = cmk<c2>(T(1), T(0));
    const ImpRow<T> r = imp_row(K, f);
    const T *S2t = th + TF_S2 * N;
    const T *Cc = th + TF_C * N;
    const T *Am = th + TF_AM * N;
    const T *A0 = th + TF_A0 * N;
    const T *Ap = th + TF_AP * N;
    T sgv[S], ccv[S], am[S], a0[S], ap[S];
    if (vec && len == S) {
        T s2v[S];
        vload<S>(s2v, S2t + j0);
        vload<S>(ccv, Cc + j0);
        vload<S>(am, Am + j0);
        vload<S>(a0, A0 + j0);
        vload<S>(ap, Ap + j0);
        vload<S>(C.e, prow + j0);
        vload<S>(w, phi + j0);
        vload<S>(y, pi + j0);
#pragma unroll
        for (int k = 0; k < S; ++k) sgv[k] = imp_sg(r, s2v[k]);
    } else {
#pragma unroll
        for (int k = 0; k < S; ++k) {
            const bool real = k < len;
            const int j = real ? j0 + k : 0;
            sgv[k] = real ? imp_sg(r, S2t[j]) : T(0);
            ccv[k] = real ? Cc[j] : T(0);
            am[k] = real ? Am[j] : T(0);
            a0[k] = real ? A0[j] : T(0);
            ap[k] = real ? Ap[j] : T(0);
            C.e[k] = real ? prow[j] : one;
            w[k] = real ? phi[j] : zero;
            y[k] = real ? pi[j] : zero;
        }
    }
#pragma unroll
    for (int k = 0; k < S; ++k)
        imp_elem(K, r, sgv[k], ccv[k], am[k], a0[k], ap[k], C.e[k], C.ct[k], C.dg[k], C.qam[k], C.qap[k], C.sub[k],
                 C.fk[k]);
}

// The same segment with the coefficients read from the materialised planes
// (row gi of the full step's tables; FP64 state), bit for bit what imp_load
// forms.
template <typename T, int S>
__device__ __forceinline__ void imp_load_mat(const MatPlanes<T> &M, const typename V2<T>::t *phi,
                                             const typename V2<T>::t *pi, const typename V2<T>::t *prow, int gi,
                                             int N, int len, int j0, bool vec, ImpCoef<T, S> &C,
                                             typename V2<T>::t (&w)[S], typename V2<T>::t (&y)[S])
{
    typedef typename V2<T>::t c2;
    const c2 zero = cmk<c2>(T(0), T(0));
    const c2 one = cmk<c2>(T(1), T(0));
    const size_t o = (size_t)gi * N + j0;
    if (vec && len == S) {
        vload<S>(C.e, prow + j0);
        vload<S>(w, phi + j0);
        vload<S>(y, pi + j0);
        vload<S>(C.fk, M.fk + o);
        vload<S>(C.dg, M.dg + o);
        vload<S>(C.ct, M.ct + o);
        vload<S>(C.sub, M.sub + o);
        vload<S>(C.qam, M.qam + o);
        vload<S>(C.qap, M.qap + o);
    } else {
#pragma unroll
        for (int k = 0; k < S; ++k) {
            const bool real = k < len;
            const size_t q = real ? o + k : 0;
            C.e[k] = real ? prow[j0 + k] : one;
            w[k] = real ? phi[j0 + k] : zero;
            y[k] = real ? pi[j0 + k] : zero;
            C.fk[k] = real ? M.fk[q] : zero;
            C.dg[k] = real ? M.dg[q] : zero;
            C.ct[k] = real ? M.ct[q] : zero;
            C.sub[k] = real ? M.sub[q] : T(0);
            C.qam[k] = real ? M.qam[q] : T(0);
            C.qap[k] = real ? M.qap[q] : T(0);
        }
    }
}

// Scan plan of the LU solve from the row's stored levels: the segment maps'
// multiplicative parts are prod(-e_j sub_j) forward and prod(-fk_j)
// backward (formed only when a level uses them).
// The lane segment's products prod(-e_j sub_j) (Af0) and prod(-fk_j) (Ab0),
// factor by factor: separate products of the sub-diagonals and of the
// pivots can overflow and underflow on stiff rows.  k_scan_plans stores
// them per row and lane with this same function.
template <typename T, int S>
__device__ __forceinline__ ScanPlan<T> scan_plan_products(const ImpCoef<T, S> &C)
{
    typedef typename V2<T>::t c2;
    ScanPlan<T> P;
    P.Af0 = cmk<c2>(T(1), T(0));
    P.Ab0 = P.Af0;
#pragma unroll
    for (int k = 0; k < S; ++k) P.Af0 = cmul(cscale<c2>(-C.sub[k], C.e[k]), P.Af0);
#pragma unroll
    for (int k = S - 1; k >= 0; --k) P.Ab0 = cmul(cmk<c2>(-C.fk[k].x, -C.fk[k].y), P.Ab0);
    return P;
}

// seg: the row's stored segment products ([G][2] per row, see ImpConst) or
// NULL (formed here).
template <typename T, int S>
__device__ __forceinline__ ScanPlan<T> scan_plan_lu(const ImpCoef<T, S> &C, int plan,
                                                    const typename V2<T>::t *seg = nullptr)
{
    typedef typename V2<T>::t c2;
    ScanPlan<T> P;
    P.Af0 = cmk<c2>(T(1), T(0));
    P.Ab0 = P.Af0;
    P.nf = plan & 0xff;
    P.nb = (plan >> 8) & 0xff;
    P.nfw = (int)__reduce_max_sync(0xffffffffu, (unsigned)P.nf);
    P.nbw = (int)__reduce_max_sync(0xffffffffu, (unsigned)P.nb);
    if (seg) {
        if (P.nfw > 0) P.Af0 = seg[0];
        if (P.nbw > 0) P.Ab0 = seg[1];
        return P;
    }
    if (P.nfw > 0) {
#pragma unroll
        for (int k = 0; k < S; ++k) P.Af0 = cmul(cscale<c2>(-C.sub[k], C.e[k]), P.Af0);
    }
    if (P.nbw > 0) {
#pragma unroll
        for (int k = S - 1; k >= 0; --k) P.Ab0 = cmul(cmk<c2>(-C.fk[k].x, -C.fk[k].y), P.Ab0);
    }
    return P;
}

// w <- M^{-1} w for the lane's segment (see above); the scan levels run as
// in seg_solve.
template <typename T, int S>
__device__ __forceinline__ void seg_solve_lu(typename V2<T>::t (&w)[S], const ImpCoef<T, S> &C, const ScanPlan<T> &P,
                                             int g, int G)
{
    typedef typename V2<T>::t c2;
    const c2 zero = cmk<c2>(T(0), T(0));
    const c2 one = cmk<c2>(T(1), T(0));
    c2 B = zero;
#pragma unroll
    for (int k = 0; k < S; ++k) B = cmul(C.e[k], caxpy(-C.sub[k], B, w[k]));
    if (P.nfw == 1) {
        // the common case: one level (the loop below, without its overhead)
        const c2 Bo = shfl_up_c(B, 1, G);
        if (P.nf >= 1 && g >= 1) B = cfma(P.Af0, Bo, B);
    } else {
        c2 A = P.Af0;
#pragma unroll 1
        for (int l = 0; l < P.nfw; ++l) {
            const int d = 1 << l;
            c2 Bo = shfl_up_c(B, d, G), Ao = one;
            if (l + 1 < P.nfw) Ao = shfl_up_c(A, d, G);
            if (l < P.nf && g >= d) {
                B = cfma(A, Bo, B);
                if (l + 1 < P.nf) A = cmul(A, Ao);
            }
        }
    }
    // lane 0's incoming value meets sub = 0 (first row of the operator)
    c2 z = shfl_up_c(B, 1, G);
#pragma unroll
    for (int k = 0; k < S; ++k) {
        z = cmul(C.e[k], caxpy(-C.sub[k], z, w[k]));
        w[k] = z;
    }
    B = zero;
#pragma unroll
    for (int k = S - 1; k >= 0; --k) B = cfnma(C.fk[k], B, w[k]);
    if (P.nbw == 1) {
        const c2 Bo = shfl_down_c(B, 1, G);
        if (P.nb >= 1 && g + 1 < G) B = cfma(P.Ab0, Bo, B);
    } else {
        c2 A = P.Ab0;
#pragma unroll 1
        for (int l = 0; l < P.nbw; ++l) {
            const int d = 1 << l;
            c2 Bo = shfl_down_c(B, d, G), Ao = one;
            if (l + 1 < P.nbw) Ao = shfl_down_c(A, d, G);
            if (l < P.nb && g + d < G) {
                B = cfma(A, Bo, B);
                if (l + 1 < P.nb) A = cmul(A, Ao);
            }
        }
    }
    // the last lane's incoming value meets fk = 0 (last row, or padding)
    c2 x = shfl_down_c(B, 1, G);
#pragma unroll
    for (int k = S - 1; k >= 0; --k) {
        x = cfnma(C.fk[k], x, w[k]);
        w[k] = x;
    }
}

// out = W x for the lane's segment; x_{j0-1} and x_{j0+S} come from the
// neighbouring lanes.  Past the row's ends the shuffles return the lane's
// own (finite) values, which meet zero off-diagonals: the angular operator's
// first row has no sub-diagonal and its last no super-diagonal (the pole
// ghosts are folded into the diagonal), and padding elements are zero.
template <typename T, int S>
__device__ __forceinline__ void apply_W(const ImpCoef<T, S> &C, const typename V2<T>::t (&x)[S],
                                        typename V2<T>::t (&out)[S], int g, int G)
{
    typedef typename V2<T>::t c2;
    const c2 xl = shfl_up_c(x[S - 1], 1, G), xr = shfl_down_c(x[0], 1, G);
#pragma unroll
    for (int k = 0; k < S; ++k) {
        const c2 xm = k ? x[k - 1] : xl;
        const c2 xp = (k + 1 < S) ? x[(k + 1) < S ? k + 1 : S - 1] : xr;
        out[k] = cfma(C.dg[k], x[k], caxpy(C.qap[k], xp, cscale<c2>(C.qam[k], xm)));
    }
}

// One implicit SDIRK2 step of length h (constants K) on one r* row held in
// shared memory, by a group of G consecutive lanes (lane g holds theta
// elements [g S, g S + S)); f is the row's step-table entry; plan the row's
// stored scan levels (0 for a row that is not active).  Same map as
// implicit_row_group.
template <typename T, int S, bool MAT = false>
__device__ void implicit_row_fwd(const ImpConst<T> &K0, typename V2<T>::t *phi, typename V2<T>::t *pi,
                                 const typename V2<T>::t *prow, const T *f, const T *th, int N, bool active,
                                 bool in_tile, int g, int G, bool vec, int plan, const MatPlanes<T> *mat = nullptr,
                                 int gi = 0, typename V2<T>::t *u1phi = nullptr, typename V2<T>::t *u1pi = nullptr,
                                 const typename V2<T>::t *seg = nullptr)
{
    typedef typename V2<T>::t c2;
    const ImpConst<T> K = K0;   // the step's constants, read once from the parameters
    const int j0 = g * S;
    int len = N - j0;
    len = len < 0 ? 0 : (len > S ? S : len);
    const int lenw = len;
    if (!active) len = 0;
    ImpCoef<T, S> C;
    c2 w[S], y[S], v[S];
    if constexpr (MAT)
        imp_load_mat<T, S>(*mat, phi, pi, prow, gi, N, len, j0, vec, C, w, y);
    else
        imp_load<T, S>(K, phi, pi, prow, f, th, N, len, j0, vec, C, w, y);
    const ScanPlan<T> P = scan_plan_lu<T, S>(C, active ? plan : 0, seg);
    {
        c2 Wu[S];
        apply_W<T, S>(C, w, Wu, g, G);
#pragma unroll
        for (int k = 0; k < S; ++k) {
            v[k] = caxpy(-K.h, Wu[k], y[k]);     // u_Pi - h Wu
            y[k] = caxpy(-K.gh, Wu[k], y[k]);    // stage 1 right side
        }
    }
    seg_solve_lu<T, S>(y, C, P, g, G);             // U1_Pi
    if (u1phi && in_tile) {
        // the first stage value U1 (U1_Phi = u_Phi + gh U1_Pi), for the adjoint's spin term
        c2 t[S];
#pragma unroll
        for (int k = 0; k < S; ++k) t[k] = caxpy(K.gh, y[k], w[k]);
        row_store<T, S>(u1phi, u1pi, t, y, j0, lenw, vec);
    }
    {
        c2 Y[S];
        apply_W<T, S>(C, y, Y, g, G);
#pragma unroll
        for (int k = 0; k < S; ++k) {
            w[k] = caxpy(K.h1g, y[k], w[k]);                            // u_Phi + (1 - gamma) h U1_Pi
            v[k] = cfnma(C.ct[k], y[k], caxpy(-K.g2h1, Y[k], v[k]));   // stage 2 right side
        }
    }
    seg_solve_lu<T, S>(v, C, P, g, G);             // U2_Pi
#pragma unroll
    for (int k = 0; k < S; ++k) w[k] = caxpy(K.gh, v[k], w[k]);
    if (in_tile) row_store<T, S>(phi, pi, w, v, j0, lenw, vec);
}

template <typename C> __device__ __forceinline__ C conj_c(C a) { return cmk<C>(a.x, -a.y); }

// Hermitian adjoint (for <x, y> = Re sum conj(x) y) of implicit_row_group's
// map on one row: the SDIRK2 stages in reverse order with conjugated
// coefficients.  The stage matrix M = (1 + gh c_t) + gh^2 (B + c0rad) = L U
// gives M^H = U^H L^H, solved as t_j = r_j - conj(fk_{j-1}) t_{j-1},
// y_j = conj(e_j) t_j, x_j = y_j - conj(m_{j+1}) x_{j+1}; (B + c0rad)^H has
// rows (qap_{j-1}, conj(dg_j), qam_{j+1}).  (phi, pi) hold the adjoint of
// the output on entry and the adjoint of the input on exit.
template <typename T, int S>
__device__ void implicit_row_adjoint(const ImpConst<T> &K, typename V2<T>::t *phi, typename V2<T>::t *pi,
                                     const typename V2<T>::t *prow, const T *f, const T *th, int N, bool active,
                                     bool in_tile, int g, int G, bool vec)
{
    typedef typename V2<T>::t c2;
    const c2 zero = cmk<c2>(T(0), T(0));
    const int j0 = g * S;
    int len = N - j0;
    len = len < 0 ? 0 : (len > S ? S : len);
    const int lenw = len;
    if (!active) len = 0;
    const T gh = K.gh;
    RowCoef<T, S> C;
    c2 w[S], y[S];
    row_load<T, S>(K, phi, pi, prow, f, th, N, len, j0, G, vec, C, w, y);
    // multipliers of M^H and the shifted angular rows of (B + c0rad)^H
    c2 fm[S], pm[S], bm[S];
    T qapp[S], qamn[S];
    {
        const c2 fk_prev = shfl_up_c(C.fk[S - 1], 1, G);
        const c2 m_next = shfl_down_c(C.m[0], 1, G);
        T qap_prev = __shfl_up_sync(0xffffffffu, C.qap[S - 1], 1, G);
        T qam_next = __shfl_down_sync(0xffffffffu, C.qam[0], 1, G);
        if (g == 0) qap_prev = T(0);
        if (g == G - 1) qam_next = T(0);
#pragma unroll
        for (int k = 0; k < S; ++k) {
            const c2 fkp = k ? C.fk[k - 1] : fk_prev;
            const c2 mn = (k + 1 < S) ? C.m[(k + 1) < S ? k + 1 : S - 1] : m_next;
            fm[k] = (g == 0 && k == 0) ? zero : conj_c(fkp);
            pm[k] = conj_c(C.e[k]);
            bm[k] = (g == G - 1 && k == S - 1) ? zero : conj_c(mn);   // m_N = 0
            qapp[k] = k ? C.qap[k - 1] : qap_prev;
            qamn[k] = (k + 1 < S) ? C.qam[(k + 1) < S ? k + 1 : S - 1] : qam_next;
        }
    }
    const ScanPlan<T> P = scan_plan<T, S>(fm, bm, g, G);
    // (B + c0rad)^H v for the whole segment, v held in v[]
    auto apply_BH = [&](const c2 *v, c2 *out) {
        c2 vl = shfl_up_c(v[S - 1], 1, G), vr = shfl_down_c(v[0], 1, G);
        if (g == 0) vl = zero;
        if (g == G - 1) vr = zero;
#pragma unroll
        for (int k = 0; k < S; ++k) {
            c2 vm = k ? v[k - 1] : vl;
            c2 vp = (k + 1 < S) ? v[(k + 1) < S ? k + 1 : S - 1] : vr;
            out[k] = cadd(cmul(conj_c(C.dg[k]), v[k]), caxpy(qamn[k], vp, cscale<c2>(qapp[k], vm)));
        }
    };
    // w = adjoint of U2_Phi, y = adjoint of U2_Pi
    c2 r2p[S], ub[S];
    {
        c2 bf[S];
#pragma unroll
        for (int k = 0; k < S; ++k) {
            const c2 iac = conj_c(C.ia1[k]);
            r2p[k] = cmul(iac, y[k]);                   // adjoint of r2_Pi
            bf[k] = cscale<c2>(-gh, r2p[k]);            // adjoint of bf2
        }
        apply_BH(bf, ub);
#pragma unroll
        for (int k = 0; k < S; ++k) w[k] = cadd(w[k], ub[k]);
    }
    seg_solve<T, S>(w, fm, pm, bm, P, g, G);       // adjoint of w2
#pragma unroll
    for (int k = 0; k < S; ++k) {
        const c2 a1c = cmk<c2>(fma(gh, C.ct[k].x, T(1)), -gh * C.ct[k].y);
        const c2 w2b = w[k];
        r2p[k] = caxpy(gh, w2b, r2p[k]);                     // adjoint of r2_Pi
        const c2 r2f = cmul(a1c, w2b);                       // adjoint of r2_Phi
        y[k] = r2p[k];                                       // adjoint of u_Pi (so far)
        // U1_Pi adjoint: from r2_Pi (-h1g conj(c_t)) and r2_Phi (h12g)
        c2 u1p = caxpy(K.h12g, r2f, cscale<c2>(-K.h1g, cmul(conj_c(C.ct[k]), r2p[k])));
        const c2 iac = conj_c(C.ia1[k]);
        const c2 t = cmul(iac, u1p);
        y[k] = cadd(y[k], t);                                // adjoint of u_Pi through U1_Pi
        ub[k] = cadd(cscale<c2>(-K.h1g, r2p[k]), cscale<c2>(-gh, t));   // adjoint of bf1
        w[k] = r2f;                                          // adjoint of U1_Phi (so far)
    }
    {
        c2 bh[S];
        apply_BH(ub, bh);
#pragma unroll
        for (int k = 0; k < S; ++k) w[k] = cadd(w[k], bh[k]);
    }
    seg_solve<T, S>(w, fm, pm, bm, P, g, G);       // adjoint of w0
#pragma unroll
    for (int k = 0; k < S; ++k) {
        const c2 a1c = cmk<c2>(fma(gh, C.ct[k].x, T(1)), -gh * C.ct[k].y);
        const c2 w0b = w[k];
        y[k] = caxpy(gh, w0b, y[k]);
        w[k] = cmul(a1c, w0b);
    }
    if (in_tile) row_store<T, S>(phi, pi, w, y, j0, lenw, vec);
}

// b and K at one point from the r table f, rs = 1/Sigma and the theta
// tables (S2 = sin^2, C = cos).
template <typename T>
__device__ __forceinline__ void bK(const T *f, T rs, T S2, T C, T &b, typename V2<T>::t &K)
{
    const T sg = rs * rs;
    b = f[RF_R] * rs;
    T kre = fma(sg, fma(-f[RF_E3], S2, f[RF_E2]), fma(b, f[RF_CTR], f[RF_CSR] - f[RF_E1]));
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

// The Lax-Wendroff phase reads the first 12 fields of an r-table entry.
static_assert(RF_R < 12 && RF_R2 < 12 && RF_AD < 12 && RF_CTR < 12 && RF_CTI < 12 && RF_CTC < 12 &&
                  RF_CSR < 12 && RF_CSI < 12 && RF_E1 < 12 && RF_E2 < 12 && RF_E3 < 12,
              "r-table fields used by the Lax-Wendroff phase must lie in its first 12 entries");

// Split-scheme Lax-Wendroff update (Eqs. 13-14 with S = F + K Phi_{r*}) of
// tile rows [ra, rb) in theta column j, in place.  (pf, pg) is the old value
// of row ra-1 and (nf, ng) the old value of row rb: both may belong to other
// threads' segments, so the caller reads them before a barrier.  sSt holds
// the step-table entries of the tile (SField): node row lr at 2 lr, the half
// node between rows k and k+1 at 2 k + 1, with the stage factors c_p folded
// in, so that with beta = c_p b and kap = c_p K
//   Eq. 13:  Phi* = (Phi_a + Phi_b)/2 - beta (Phi_b - Phi_a)
//            Pi*  = (Pi_a + Pi_b)/2 + beta (Pi_b - Pi_a) + kap (Phi_b - Phi_a) + (dt/2) F
//   Eq. 14:  Phi' = Phi - beta (Phi*_+ - Phi*_-)
//            Pi'  = Pi + beta (Pi*_+ - Pi*_-) + kap (Phi*_+ - Phi*_-) + dt F.
// ph1 and ph2 are the source phases e^{-i m Omega t} at t_n and t_n + dt/2
// times dt/2 and dt; the spatial part of F comes from its factors in the
// step and theta tables (SField), so the stages read no global memory.
// Tile row lr is global row g0 + lr.
// INTERIOR: every node and midpoint of the segment lies strictly inside
// the grid (1 <= row <= Nr - 2), so the boundary tests are left out; they
// cost about 8 % of a step when taken in every tile.
// beta = c_p b and kap = c_p K of the Lax-Wendroff stages at the position
// of step-table entry f and theta (sin^2 = S2, cos = C).  The materialised
// planes of the FP64 path (k_mat_coef) are made by this same function.
template <typename T>
__device__ __forceinline__ void lw_coef(const T *f, T S2, T C, T &beta, typename V2<T>::t &kap, T *sg_out = nullptr)
{
    typedef typename V2<T>::t c2;
    constexpr int NA = 16 / (int)sizeof(T);   // one 16-byte load holds R2 and AD
    T a[NA], l[8];
    vload<NA>(a, f);
    vload<8>(l, f + SF_RB);
    const T rs = rsq_(fma(-a[SF_AD], S2, a[SF_R2]));
    const T sg = rs * rs;
    beta = rs * l[SF_RB - SF_RB];
    const T kx = fma(sg, fma(-l[SF_E3 - SF_RB], S2, l[SF_E2 - SF_RB]), fma(rs, l[SF_RCTR - SF_RB], l[SF_CSE - SF_RB]));
    const T ky = fma(rs, fma(l[SF_RCTC - SF_RB], C, l[SF_RCTI - SF_RB]), l[SF_CSI - SF_RB]);
    kap = cmk<c2>(sg * kx, sg * ky);
    if (sg_out) *sg_out = sg;
}

// beta = c_p b, kap = c_p K and 1/Sigma^2 at step-table entry f, with their
// derivatives with respect to a (df: the entry's spin derivative).  The
// values are those lw_coef forms.
template <typename T> struct LwDa {
    typedef typename V2<T>::t c2;
    T beta, dbeta, sg, dsg;
    c2 kap, dkap;
};
template <typename T>
__device__ __forceinline__ LwDa<T> lw_coef_da(const T *f, const T *df, T S2, T C)
{
    typedef typename V2<T>::t c2;
    LwDa<T> o;
    const T sig = fma(-f[SF_AD], S2, f[SF_R2]);
    const T dsig = fma(-df[SF_AD], S2, df[SF_R2]);
    const T rs = rsq_(sig);
    o.sg = rs * rs;
    const T drs = T(-0.5) * rs * o.sg * dsig;
    o.dsg = -o.sg * o.sg * dsig;
    o.beta = rs * f[SF_RB];
    o.dbeta = fma(drs, f[SF_RB], rs * df[SF_RB]);
    const T t = fma(-f[SF_E3], S2, f[SF_E2]), dt_ = fma(-df[SF_E3], S2, df[SF_E2]);
    const T X = fma(o.sg, t, fma(rs, f[SF_RCTR], f[SF_CSE]));
    const T dX = o.dsg * t + o.sg * dt_ + drs * f[SF_RCTR] + rs * df[SF_RCTR] + df[SF_CSE];
    const T u = fma(f[SF_RCTC], C, f[SF_RCTI]), du = fma(df[SF_RCTC], C, df[SF_RCTI]);
    const T Y = fma(rs, u, f[SF_CSI]);
    const T dY = drs * u + rs * du + df[SF_CSI];
    o.kap = cmk<c2>(o.sg * X, o.sg * Y);
    o.dkap = cmk<c2>(o.dsg * X + o.sg * dX, o.dsg * Y + o.sg * dY);
    return o;
}

// Spin derivatives of one element's implicit-operator coefficients: dW's
// diagonal ddg and off-diagonals (dqam, dqap) and dc_t (unscaled), from the
// row constants r, the table entry fr and its derivative dfr (SField,
// implicit block), and the element's theta values.
template <typename T>
__device__ __forceinline__ void imp_da(const ImpRow<T> &r, const T (&fr)[8], const T (&dfr)[8], T s2, T cc, T am,
                                       T a0, T ap, typename V2<T>::t &ddg, typename V2<T>::t &dct, T &dqam,
                                       T &dqap)
{
    typedef typename V2<T>::t c2;
    const T sg = imp_sg(r, s2);
    const T dsg = -sg * sg * fma(-dfr[SF_AD], s2, dfr[SF_R2]);
    const T dq = fma(dfr[SF_DELTA], sg, r.D * dsg);
    dqam = dq * am;
    dqap = dq * ap;
    ddg = cmk<c2>(fma(dq, a0, -fma(dsg, r.c0r, sg * dfr[SF_C0R])), -fma(dsg, r.c0i, sg * dfr[SF_C0I]));
    const T ctr = dfr[SF_CTR], cti = fma(dfr[SF_CTC], cc, dfr[SF_CTI]);
    dct = cmk<c2>(fma(dsg, fr[SF_CTR], sg * ctr), fma(dsg, fma(fr[SF_CTC], cc, fr[SF_CTI]), sg * cti));
}

template <typename T, bool INTERIOR, bool MAT = false, bool SRC = true>
__device__ void lw_segment(const StepParams<T> &p, typename V2<T>::t *sPhi, typename V2<T>::t *sPi,
                           const T *sSt, const T *sTh, int j, int ra, int rb,
                           typename V2<T>::t pf, typename V2<T>::t pg, typename V2<T>::t nf,
                           typename V2<T>::t ng, int g0, typename V2<T>::t ph1, typename V2<T>::t ph2,
                           bool src)
{
    typedef typename V2<T>::t c2;
    const int N = p.Nth, P = p.pitch, Nr = p.Nr;
    const T S2 = sTh[TF_S2 * N + j], C = sTh[TF_C * N + j];
    const c2 zero = cmk<c2>(T(0), T(0));
    const T half = T(0.5);
    T gth = T(0), ga2 = T(0);
    if (SRC && src) {
        gth = sTh[TF_GTH * N + j];
        ga2 = sTh[TF_GA2 * N + j];
    }

    // beta and kap at tile position e (2 lr: node, 2 k + 1: half node), and
    // 1/Sigma^2 there when the source needs it
    auto coef = [&](int e, T &beta, c2 &kap, T &sg, bool need_sg) {
        if constexpr (MAT) {
            T v[4];
            vload<4>(v, p.mat.lw + ((size_t)(2 * g0 + e) * N + j) * 4);
            beta = v[0];
            kap = cmk<c2>(v[1], v[2]);
            if (need_sg) {
                const T *f = sSt + e * NSF;
                const T rs = rsq_(fma(-f[SF_AD], S2, f[SF_R2]));
                sg = rs * rs;
            }
        } else {
            lw_coef<T>(sSt + e * NSF, S2, C, beta, kap, &sg);
        }
    };
    // source at tile position e times the scaled phase ph (zero outside the
    // patch rows): F = SRC sg (SR2 GTH + GA2)
    auto source = [&](int e, T sg, c2 ph) {
        const T *f = sSt + e * NSF;
        T sv[4];
        vload<4>(sv, f + SF_SRE);
        const c2 F = cscale<c2>(sg * fma(sv[SF_SR2 - SF_SRE], gth, ga2), cmk<c2>(sv[0], sv[1]));
        return cmul(F, ph);
    };

    // u*_{k+1/2} between tile rows k and k+1 (Eq. 13)
    auto midpoint = [&](int k, c2 fa, c2 ga, c2 fb, c2 gb, c2 &mf, c2 &mg) {
        int gl = g0 + k;   // global index of the lower node
        if (!INTERIOR && (gl < 0 || gl > Nr - 2)) {
            mf = zero;
            mg = zero;
            return;
        }
        T beta, sg;
        c2 kap;
        const bool s_row = SRC && src && gl >= p.patch_p0 && gl < p.patch_p0 + p.patch_np;
        coef(2 * k + 1, beta, kap, sg, s_row);
        const c2 df = csub(fb, fa);
        mf = caxpy(-beta, df, cscale<c2>(half, cadd(fa, fb)));
        c2 t = caxpy(beta, csub(gb, ga), cscale<c2>(half, cadd(ga, gb)));
        if (s_row) t = cadd(t, source(2 * k + 1, sg, ph1));
        mg = cfma(kap, df, t);
    };

    c2 fb = sPhi[ra * P + j], gb = sPi[ra * P + j];
    c2 mfp, mgp;
    midpoint(ra - 1, pf, pg, fb, gb, mfp, mgp);
    // two rows per trip: the window's values change registers instead of
    // being copied at the end of every row
#pragma unroll 2
    for (int lr = ra; lr < rb; ++lr) {
        int gi = g0 + lr;
        if (!INTERIOR && gi >= Nr) break;
        c2 fc, gc;
        if (lr + 1 < rb) {
            fc = sPhi[(lr + 1) * P + j];
            gc = sPi[(lr + 1) * P + j];
        } else {
            fc = nf;
            gc = ng;
        }
        c2 mf, mg;
        midpoint(lr, fb, gb, fc, gc, mf, mg);
        c2 nfv = zero, ngv = zero;
        if (INTERIOR || (gi >= 1 && gi <= Nr - 2)) {
            // Eq. 14 at node gi
            T beta, sg;
            c2 kap;
            const bool s_row = SRC && src && gi >= p.patch_p0 && gi < p.patch_p0 + p.patch_np;
            coef(2 * lr, beta, kap, sg, s_row);
            const c2 dmf = csub(mf, mfp);
            nfv = caxpy(-beta, dmf, fb);
            c2 t = caxpy(beta, csub(mg, mgp), gb);
            if (s_row) t = cadd(t, source(2 * lr, sg, ph2));
            ngv = cfma(kap, dmf, t);
        }
        sPhi[lr * P + j] = nfv;
        sPi[lr * P + j] = ngv;
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

// Lax-Wendroff phase of tile rows r0 .. r0+nr-1 (tile row lr is global row
// g0 + lr; rows r0-1 and r0+nr are read as neighbours) by NC threads with
// index ctid.  With N <= NC every column is cut into
// NC / N row segments; the rows on either side of a segment are read before
// bar() (a barrier over the NC threads), as the neighbouring segments
// overwrite them.
template <typename T, bool INTERIOR, bool MAT = false, typename Bar, bool SRC = true>
__device__ __forceinline__ void lw_phase(const StepParams<T> &p, typename V2<T>::t *sPhi, typename V2<T>::t *sPi,
                                         const T *sSt, const T *sTh, int r0, int nr, int g0, int ctid, int NC,
                                         bool src, typename V2<T>::t ph1, typename V2<T>::t ph2, Bar bar)
{
    typedef typename V2<T>::t c2;
    const int N = p.Nth, P = p.pitch;
    const c2 zero = cmk<c2>(T(0), T(0));
    if (N <= NC) {
        const int nseg = udiv(NC, N);
        const int sl = udiv(nr + nseg - 1, nseg);
        const int sgm = udiv(ctid, N), j = ctid - sgm * N;
        int ra = r0 + sgm * sl, rb = r0 + (sgm + 1) * sl;
        if (rb > r0 + nr) rb = r0 + nr;
        const bool work = sgm < nseg && ra < rb;
        c2 pf = zero, pg = zero, nf = zero, ng = zero;
        if (work) {
            pf = sPhi[(ra - 1) * P + j];
            pg = sPi[(ra - 1) * P + j];
            nf = sPhi[rb * P + j];
            ng = sPi[rb * P + j];
        }
        bar();
        if (work) lw_segment<T, INTERIOR, MAT, SRC>(p, sPhi, sPi, sSt, sTh, j, ra, rb, pf, pg, nf, ng, g0, ph1, ph2, src);
    } else {
        // each thread owns whole columns: rows r0-1 and r0+nr are read before any write
        for (int j = ctid; j < N; j += NC) {
            c2 pf = sPhi[(r0 - 1) * P + j], pg = sPi[(r0 - 1) * P + j];
            c2 nf = sPhi[(r0 + nr) * P + j], ng = sPi[(r0 + nr) * P + j];
            lw_segment<T, INTERIOR, MAT, SRC>(p, sPhi, sPi, sSt, sTh, j, r0, r0 + nr, pf, pg, nf, ng, g0, ph1, ph2, src);
        }
    }
}

// Barrier over the first n threads of the CTA (named barrier id).
__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
// The same barrier; returns whether pred holds in all n threads.
__device__ __forceinline__ int named_sync_and(int id, int n, int pred)
{
    int r;
    asm volatile("{ .reg .pred p, q; setp.ne.s32 p, %1, 0; bar.red.and.pred q, %2, %3, p; selp.s32 %0, 1, 0, q; }"
                 : "=r"(r) : "r"(pred), "r"(id), "r"(n) : "memory");
    return r;
}

// ---- TMA bulk copies (1-D, global <-> shared) and the mbarrier that
// completes them.  Every wait is bounded.
__device__ __forceinline__ unsigned smem_u32(const void *ptr) { return (unsigned)__cvta_generic_to_shared(ptr); }
__device__ __forceinline__ void mbar_init(unsigned long long *m, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *m, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *m)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(m)) : "memory");
}
// Brings global bytes [src, src + bytes) into L2 without waiting (16-byte
// aligned, a multiple of 16 bytes).
__device__ __forceinline__ void prefetch_l2(const void *src, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_wait(unsigned long long *m, unsigned parity, int limit)
{
    unsigned ok = 0;
    for (int it = 0; it < limit && !ok; ++it)
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(ok) : "r"(smem_u32(m)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, unsigned bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
constexpr int kWaitLimit = 1 << 22;   // try_wait rounds before a copy is declared lost

// FP64 weighted sum h = sum_j w_j row_j in the order extract_warp uses; lane 0
// of the calling warp returns it.
template <typename T>
__device__ double2 sample_warp(const StepParams<T> &p, const typename V2<T>::t *row)
{
    const int lane = threadIdx.x & 31;
    double sre = 0.0, sim = 0.0;
    for (int j = lane; j < p.Nth; j += 32) {
        double w = p.w[j];
        sre = fma(w, (double)row[j].x, sre);
        sim = fma(w, (double)row[j].y, sim);
    }
    for (int o = 16; o > 0; o >>= 1) {
        sre += __shfl_xor_sync(0xffffffffu, sre, o);
        sim += __shfl_xor_sync(0xffffffffu, sim, o);
    }
    return make_double2(sre, sim);
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

// Fused step of the split scheme (merged Strang composition): the tile's
// input is s_n (or the physical state u_n when p.first), the output is
//   s_{n+1} = LW_n C_h s_n,   h = dt (h = dt/2 when p.first),
// and the physical sample u_{n+1} = C_{dt/2} s_{n+1} is taken on the
// extraction row.  With p.imp_only the kernel only applies C_{dt/2} to the
// tile rows (used to output the physical state).
// The work of one CTA: tile number `tile` of the grid described by p, whose
// step takes `ntiles` CTAs (the last of them to start advances the step
// index), for KS = 1, 2 or 3 time steps per launch.  The tile holds its TR
// output rows plus KS halo rows on either side (R = TR + 2 KS; tile row lr is
// global row g0 + lr, g0 = i0 - KS).  Step k (from 0) updates rows
// k + 1 .. R - 2 - k, so the last one updates the TR output rows; the state
// read and written per step falls to 1/KS at the cost of recomputing the
// extra halo rows.  The result is bitwise that of KS single steps.
template <typename T, int S, int KS>
__device__ __forceinline__ void split_tile(const StepParams<T> &p, int tile, int ntiles)
{
    typedef typename V2<T>::t c2;
    constexpr int kMaxChunks = 8;
    static_assert(KS >= 1 && KS <= 3, "one to three steps per launch");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double2 sph[2 * KS];
    __shared__ long long s_n;
    __shared__ __align__(8) unsigned long long s_mbar[kMaxChunks];
    __shared__ int s_plan[kMaxTileRows + 6];   // stored scan levels of the tile rows
    const int Nr = p.Nr, N = p.Nth, TR = p.tile_rows, R = TR + 2 * KS, P = p.pitch;
    const int tid = threadIdx.x, NT = blockDim.x;
    const int i0 = tile * TR, g0 = i0 - KS;
    const int G = p.group;

    const SplitSmem plan = split_smem_plan(R, N, (int)sizeof(T));
    c2 *sPhi = (c2 *)(smem_raw + plan.phi);
    c2 *sPi = (c2 *)(smem_raw + plan.pi);
    T *sSt = (T *)(smem_raw + plan.rt);   // step-table entries (SField) of the tile's positions
    T *sTh = (T *)(smem_raw + plan.th);
    c2 *xPhi = (c2 *)(smem_raw + plan.total);   // KS > 1: copy of the extraction row
    c2 *xPi = xPhi + N;
    // implicit step of this launch: dt/2 for the first step and for the state
    // output (one step per launch only; with more steps per launch it is the
    // full step, chosen at compile time so that its constants are read at
    // fixed parameter offsets)
    const ImpConst<T> &K = (KS == 1 && (p.first || p.imp_only)) ? p.half : p.full;

    const bool src = !p.imp_only && p.patch_np > 0 && i0 + TR + KS - 1 >= p.patch_p0 &&
                     g0 <= p.patch_p0 + p.patch_np;
    if constexpr (KS == 1) {
        // forward tape: the input's extraction row, from the input buffer
        if (p.tape && p.i_ext >= i0 && p.i_ext < i0 + TR && p.i_ext < Nr) {
            c2 *x = p.tape + tape_x_off(Nr, N);
            for (int j = tid; j < N; j += NT) {
                x[j] = p.uin[(size_t)p.i_ext * N + j];
                x[N + j] = p.uin[((size_t)Nr + p.i_ext) * N + j];
            }
        }
    }
    if (tid == 0) {
        long long n = p.nfix >= 0 ? p.nfix : *((volatile long long *)&p.ctl->step);
        s_n = n;
        if (!p.imp_only && p.nfix < 0) {
            // The last CTA to read the step index advances it.  Later kernels
            // on the stream see the new value; no CTA of this launch reads it
            // again, so no CTA has to wait for its own stores first.
            __threadfence();
            unsigned t = atomicAdd(&p.ctl->ticket, 1u);
            if (t == (unsigned)ntiles - 1u) {
                p.ctl->ticket = 0u;
                p.ctl->step = n + KS;
            }
        }
        if (src)
            for (int k = 0; k < KS; ++k) {
                double t = (double)(n + k) * p.dt64;
                // phases of Eqs. 13 and 14 times their stage lengths dt/2 and dt
                const double2 e1 = phase_at(p.mOmega, t), e2 = phase_at(p.mOmega, t + 0.5 * p.dt64);
                sph[2 * k] = make_double2(0.5 * p.dt64 * e1.x, 0.5 * p.dt64 * e1.y);
                sph[2 * k + 1] = make_double2(p.dt64 * e2.x, p.dt64 * e2.y);
            }
    }
    // ---- A: tile rows g0 .. g0+R-1 (state), r and theta tables; the row
    // solves read their pivots from global memory (L2), which leaves room for
    // taller tiles
    const c2 zero = cmk<c2>(T(0), T(0));
    // (row, column) walk of the tile without integer division in the loop
    const int t_lr = udiv(tid, N), t_j = tid - t_lr * N;
    const int d_lr = udiv(NT, N), d_j = NT - d_lr * N;
    // rows of the tile that exist on the grid: [ga, gb] globally, from tile row la
    const int ga = g0 < 0 ? 0 : g0;
    const int gb = g0 + R - 1 > Nr - 1 ? Nr - 1 : g0 + R - 1;
    const int la = ga - g0, nrows = gb - ga + 1;
    // The state tile arrives in chunks of whole implicit passes, one mbarrier
    // each, so that the first pass can start while later rows are in flight.
    const int lgG = __ffs(G) - 1;   // G is a power of two
    const int rpp = NT >> lgG;      // theta rows per implicit pass
    int cr = rpp;                   // rows per chunk
    while (udiv(R + cr - 1, cr) > kMaxChunks) cr += rpp;
    const int nch = udiv(R + cr - 1, cr);
    if (p.bulk) {
        if (tid == 0) {
            for (int c = 0; c < nch; ++c) mbar_init(&s_mbar[c], 1);
            for (int c = 0; c < nch; ++c) {
                int r0 = c * cr, r1 = r0 + cr;
                if (r1 > R) r1 = R;
                if (r0 < la) r0 = la;
                if (r1 > la + nrows) r1 = la + nrows;
                unsigned bytes = r1 > r0 ? (unsigned)(r1 - r0) * (unsigned)N * (unsigned)sizeof(c2) : 0u;
                mbar_expect_tx(&s_mbar[c], 2 * bytes);   // with no bytes this is a plain arrival
                if (bytes) {
                    const size_t gr = (size_t)(ga + r0 - la);
                    bulk_g2s(sPhi + r0 * P, p.uin + gr * N, bytes, &s_mbar[c]);
                    bulk_g2s(sPi + r0 * P, p.uin + ((size_t)Nr + gr) * N, bytes, &s_mbar[c]);
                    // the chunk's pivot rows, which the row solves read from global memory
                    prefetch_l2(K.piv + gr * N, bytes);
                }
            }
        }
        // rows off the grid (first and last tiles only) are zero
        for (int lr = t_lr, j = t_j; lr < R;) {
            if (lr < la || lr >= la + nrows) {
                sPhi[lr * P + j] = zero;
                sPi[lr * P + j] = zero;
            }
            lr += d_lr;
            j += d_j;
            if (j >= N) { j -= N; ++lr; }
        }
    } else {
        for (int lr = t_lr, j = t_j; lr < R;) {
            int gi = g0 + lr;
            c2 fv = zero, gv = zero;
            if (gi >= 0 && gi < Nr) {
                fv = p.uin[(size_t)gi * N + j];
                gv = p.uin[((size_t)Nr + gi) * N + j];
            }
            sPhi[lr * P + j] = fv;
            sPi[lr * P + j] = gv;
            lr += d_lr;
            j += d_j;
            if (j >= N) { j -= N; ++lr; }
        }
    }
    {
        // step-table positions 2 g0 .. 2(g0+R-1); those off the grid are zero
        const long long pbase = 2LL * g0;
        const long long pmax = 2LL * Nr - 2;
        for (int idx = tid; idx < (2 * R - 1) * NSF; idx += NT) {
            int e = idx / NSF, q = idx - e * NSF;
            long long pos = pbase + e;
            sSt[idx] = (pos >= 0 && pos <= pmax) ? p.stab[(size_t)pos * NSF + q] : T(0);
        }
    }
    for (int idx = tid; idx < NTF * N; idx += NT) sTh[idx] = p.thtab[idx];
    // Every implicit step of the launch uses K: with more steps per launch K
    // is the full step (the launcher refuses first steps and state outputs).
    for (int lr = tid; lr < R; lr += NT) {
        const int gi = g0 + lr;
        s_plan[lr] = (gi >= 0 && gi < Nr) ? K.plan[gi] : 0;
    }
    __syncthreads();
    const int g = tid & (G - 1), tq = tid >> lgG;   // lane in the row group, row of the pass
    const bool vec = p.vec != 0;
    // bound of the waits on this tile's state copy (the drain after a failed
    // wait always uses kWaitLimit, so no copy is in flight when the CTA exits)
    const int wait_lim = p.wait0 >= 0 ? p.wait0 : kWaitLimit;
    // implicit step on tile rows [lo, hi)
    // use_mat: the step is a full one and the FP64 planes are on
    auto implicit_rows = [&](const ImpConst<T> &Ki, int lo, int hi, bool wait_chunks, int &ok, bool use_mat) {
        for (int base = lo; base < hi; base += rpp) {
            if (wait_chunks && p.bulk && ok) {
                // the chunks that hold this pass's rows
                int last = base + rpp - 1;
                if (last > hi - 1) last = hi - 1;
                for (int c = udiv(base, cr); c <= udiv(last, cr); ++c) ok &= (int)mbar_wait(&s_mbar[c], 0, wait_lim);
            }
            int lr = base + tq;
            bool in_tile = lr < hi;
            int gi = g0 + lr;
            bool active = in_tile && gi >= 1 && gi <= Nr - 2;
            int lrc = in_tile ? lr : lo;
            // forward tape: the first stage value of each output row
            c2 *t1f = nullptr, *t1g = nullptr;
            if constexpr (KS == 1) {
                if (p.tape && in_tile && lr >= 1 && lr <= TR && gi < Nr) {
                    t1f = p.tape + (size_t)gi * N;
                    t1g = p.tape + ((size_t)Nr + gi) * N;
                }
            }
            // FP64: the stored segment products spare FP64 arithmetic, the
            // bound of that path; FP32 forms them (cheaper than the loads)
            const c2 *segr = sizeof(T) == 8 ? Ki.seg + ((size_t)(active ? gi : 1) * G + g) * 2 : nullptr;
            if constexpr (sizeof(T) == 8) {
                if (use_mat) {
                    implicit_row_fwd<T, S, true>(Ki, sPhi + lrc * P, sPi + lrc * P, Ki.piv + (size_t)(active ? gi : 1) * N, nullptr, nullptr,
                                                 N, active, in_tile, g, G, vec, s_plan[lrc], &p.mat, gi, t1f, t1g, segr);
                    continue;
                }
            }
            implicit_row_fwd<T, S>(Ki, sPhi + lrc * P, sPi + lrc * P, Ki.piv + (size_t)(active ? gi : 1) * N, sSt + 2 * lrc * NSF, sTh, N,
                                   active, in_tile, g, G, vec, s_plan[lrc], nullptr, 0, t1f, t1g, segr);
        }
    };
    // physical sample u = C_{dt/2} s of the extraction row (tile row lx) in
    // place, or of its copy in (xPhi, xPi); warp 0
    auto extract_row = [&](int lx, long long slot, bool copy) {
        if (tid < 32) {
            c2 *rf = copy ? xPhi : sPhi + lx * P, *rg = copy ? xPi : sPi + lx * P;
            bool mine = tid < G;
            bool active = mine && p.i_ext >= 1 && p.i_ext <= Nr - 2;
            implicit_row_fwd<T, S>(p.half, rf, rg, p.half.piv + (size_t)p.i_ext * N, sSt + 2 * lx * NSF, sTh, N,
                                     active, mine, tid & (G - 1), G, vec, p.half.plan[p.i_ext]);
            __syncwarp();
            if (p.nfix >= 0) {
                // a step applied to caller buffers: the sample alone, to h_out
                const double2 h = sample_warp<T>(p, rf);
                if (tid == 0) *p.h_out = h;
            } else {
                extract_warp<T>(p, rf, slot);
            }
        }
    };
    const bool ext = !p.imp_only && (p.nfix < 0 || p.h_out != nullptr) && p.i_ext >= i0 && p.i_ext < i0 + TR &&
                     p.i_ext < Nr;
    // ---- B and C, once per time step of the launch.  Step k (from 0) runs
    // the implicit stage on tile rows k .. R-1-k and the Lax-Wendroff stages
    // on rows k+1 .. R-2-k, so the output rows KS .. KS+TR-1 are exact after
    // the last step.  One loop body serves every step: a multi-step kernel's
    // code is no larger than the one-step kernel's.
    int ok = 1;   // every bounded wait of this thread succeeded
    const auto sync_all = [] { __syncthreads(); };
#pragma unroll 1
    for (int k = 0; k < KS; ++k) {
        // implicit step: dt/2 for a first step and for the state output, else dt
        const ImpConst<T> &Ki = (KS == 1 && k == 0) ? K : p.full;
        const int lo = p.imp_only ? KS : k, hi = p.imp_only ? TR + KS : R - k;
        implicit_rows(Ki, lo, hi, k == 0, ok, p.mat_on && !(k == 0 && (p.first || p.imp_only)));
        if (k == 0) {
            // the remaining phases read every row of the tile
            if (p.bulk && ok)
                for (int c = 0; c < nch; ++c) ok &= (int)mbar_wait(&s_mbar[c], 0, wait_lim);
            // all threads agree on the outcome of the bounded waits before acting on it
            if (!__syncthreads_and(ok)) {
                // a copy did not complete: report, wait once more, leave the tile alone
                if (tid == 0) {
                    atomicOr(&p.ctl->flags, FLAG_TIMEOUT);
                    for (int c = 0; c < nch; ++c) mbar_wait(&s_mbar[c], 0, kWaitLimit);
                }
                return;
            }
            if (p.imp_only) break;
            if constexpr (KS == 1) {
                if (p.tape) {
                    // forward tape: the implicit stage's output U2 of the output
                    // rows, before the Lax-Wendroff stages overwrite them
                    c2 *u2 = p.tape + tape_u2_off(Nr, N);
                    for (int idx = tid; idx < TR * N; idx += NT) {
                        const int lr = 1 + idx / N, j = idx - (lr - 1) * N;
                        const int gi = g0 + lr;
                        if (gi < Nr) {
                            u2[(size_t)gi * N + j] = sPhi[lr * P + j];
                            u2[((size_t)Nr + gi) * N + j] = sPi[lr * P + j];
                        }
                    }
                    __syncthreads();
                }
            }
        } else {
            __syncthreads();
        }
        c2 ph1 = zero, ph2 = zero;
        if (src) {
            ph1 = from_d2<T>(sph[2 * k]);
            ph2 = from_d2<T>(sph[2 * k + 1]);
        }
        // rows g0 .. g0+R-1 all inside [1, Nr-2] except in the first and last tiles
        const bool interior = g0 >= 1 && g0 + R <= Nr - 1;
        bool lw_done = false;
        if constexpr (sizeof(T) == 8) {
            if (p.mat_on) {
                if (interior)
                    lw_phase<T, true, true>(p, sPhi, sPi, sSt, sTh, k + 1, R - 2 - 2 * k, g0, tid, NT, src, ph1, ph2,
                                            sync_all);
                else
                    lw_phase<T, false, true>(p, sPhi, sPi, sSt, sTh, k + 1, R - 2 - 2 * k, g0, tid, NT, src, ph1, ph2,
                                             sync_all);
                lw_done = true;
            }
        }
        if (!lw_done) {
            // most tiles hold no source row: they take a form without the source tests
            if (interior && !src)
                lw_phase<T, true, false, decltype(sync_all), false>(p, sPhi, sPi, sSt, sTh, k + 1, R - 2 - 2 * k, g0,
                                                                    tid, NT, false, ph1, ph2, sync_all);
            else if (interior)
                lw_phase<T, true>(p, sPhi, sPi, sSt, sTh, k + 1, R - 2 - 2 * k, g0, tid, NT, src, ph1, ph2, sync_all);
            else
                lw_phase<T, false>(p, sPhi, sPi, sSt, sTh, k + 1, R - 2 - 2 * k, g0, tid, NT, src, ph1, ph2, sync_all);
        }
        __syncthreads();
        if (k + 1 < KS && ext) {
            // sample of step n+k+1 from a copy of the extraction row; the row
            // itself goes on into the next step
            if (tid < 32) {
                const int lx = p.i_ext - g0;
                for (int j = tid; j < N; j += 32) {
                    xPhi[j] = sPhi[lx * P + j];
                    xPi[j] = sPi[lx * P + j];
                }
            }
            __syncthreads();
            extract_row(p.i_ext - g0, s_n + k + 1, true);
        }
    }
    // ---- D: store the output rows (tile rows KS .. KS+TR-1)
    const int nout = (Nr - i0) < TR ? (Nr - i0) : TR;
    if (p.bulk) {
        fence_proxy_async();      // shared-memory writes become visible to the bulk copy
        __syncthreads();
        if (tid == 0) {
            unsigned bytes = (unsigned)nout * (unsigned)N * (unsigned)sizeof(c2);
            bulk_s2g(p.uout + (size_t)i0 * N, sPhi + KS * P, bytes);
            bulk_s2g(p.uout + ((size_t)Nr + i0) * N, sPi + KS * P, bytes);
            bulk_commit();
            bulk_wait_read();     // the tile may be reused (extraction) and the CTA may exit
        }
    } else {
        for (int k = t_lr, j = t_j; k < TR;) {
            int gi = i0 + k;
            if (gi < Nr) {
                p.uout[(size_t)gi * N + j] = sPhi[(k + KS) * P + j];
                p.uout[((size_t)Nr + gi) * N + j] = sPi[(k + KS) * P + j];
            }
            k += d_lr;
            j += d_j;
            if (j >= N) { j -= N; ++k; }
        }
    }
    if (p.imp_only) return;
    // ---- E: physical sample u_{n+KS} = C_{dt/2} s_{n+KS} on the extraction row
    if (ext) {
        __syncthreads();
        extract_row(p.i_ext - g0, s_n + KS, false);
    }
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *m)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(m)) : "memory");
}

}  // namespace

// Raise a kernel's dynamic shared-memory limit to the device maximum, once
// per kernel and device.  Occupancy queries and launches never lower it, so
// a launch within the maximum is valid whatever was queried before it.
static inline cudaError_t smem_limit_max(const void *fn)
{
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (const auto &d : done)
        if (d.first == fn && d.second == dev) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes a;
    e = cudaFuncGetAttributes(&a, fn);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)a.sharedSizeBytes);
    if (e != cudaSuccess) return e;
    done.emplace_back(fn, dev);
    return cudaSuccess;
}

}  // namespace teuk
