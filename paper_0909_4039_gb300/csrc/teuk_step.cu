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
// helpers (one or two steps per launch, batched, persistent) then round the
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
// threads' segments, so the caller reads them before a barrier.  sRt holds
// the r-table entries of the tile: node row lr at 2 lr, the half node
// between rows k and k+1 at 2 k + 1.  Tile row lr is global row g0 + lr.
// INTERIOR: every node and midpoint of the segment lies strictly inside
// the grid (1 <= row <= Nr - 2), so the boundary tests are left out; they
// cost about 8 % of a step when taken in every tile.
template <typename T, bool INTERIOR>
__device__ void lw_segment(const StepParams<T> &p, typename V2<T>::t *sPhi, typename V2<T>::t *sPi,
                           const T *sRt, const T *sTh, int j, int ra, int rb,
                           typename V2<T>::t pf, typename V2<T>::t pg, typename V2<T>::t nf,
                           typename V2<T>::t ng, int g0, typename V2<T>::t ph1, typename V2<T>::t ph2,
                           bool src)
{
    typedef typename V2<T>::t c2;
    const int N = p.Nth, P = p.pitch, Nr = p.Nr;
    const T S2 = sTh[TF_S2 * N + j], C = sTh[TF_C * N + j];
    const T hdt = p.half_dt, dt = p.dt, ri = p.drs_inv;
    const c2 zero = cmk<c2>(T(0), T(0));

    // u*_{k+1/2} between tile rows k and k+1 (Eq. 13)
    auto midpoint = [&](int k, c2 fa, c2 ga, c2 fb, c2 gb, c2 &mf, c2 &mg) {
        int gl = g0 + k;   // global index of the lower node
        if (!INTERIOR && (gl < 0 || gl > Nr - 2)) {
            mf = zero;
            mg = zero;
            return;
        }
        T f[12];   // fields R .. E3 of the half-node entry
        vload<12>(f, sRt + (2 * k + 1) * NRF);
        T rs = rsq_(fma(-f[RF_AD], S2, f[RF_R2]));
        T b;
        c2 K;
        bK<T>(f, rs, S2, C, b, K);
        c2 fbar = cscale<c2>(T(0.5), cadd(fa, fb));
        c2 gbar = cscale<c2>(T(0.5), cadd(ga, gb));
        c2 df = cscale<c2>(ri, csub(fb, fa));
        c2 dg = cscale<c2>(ri, csub(gb, ga));
        c2 Sv = cmul(K, df);
        if (src) Sv = cadd(Sv, patch_val(p, gl, 1, j, ph1));
        mf = caxpy(-(hdt * b), df, fbar);
        mg = caxpy(hdt, caxpy(b, dg, Sv), gbar);
    };

    c2 fb = sPhi[ra * P + j], gb = sPi[ra * P + j];
    c2 mfp, mgp;
    midpoint(ra - 1, pf, pg, fb, gb, mfp, mgp);
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
            T f[12];   // fields R .. E3 of the node entry
            vload<12>(f, sRt + 2 * lr * NRF);
            T rs = rsq_(fma(-f[RF_AD], S2, f[RF_R2]));
            T b;
            c2 K;
            bK<T>(f, rs, S2, C, b, K);
            c2 df = cscale<c2>(ri, csub(mf, mfp));
            c2 dg = cscale<c2>(ri, csub(mg, mgp));
            c2 Sv = cmul(K, df);
            if (src) Sv = cadd(Sv, patch_val(p, gi, 0, j, ph2));
            nfv = caxpy(-(dt * b), df, fb);
            ngv = caxpy(dt, caxpy(b, dg, Sv), gb);
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
template <typename T, bool INTERIOR, typename Bar>
__device__ __forceinline__ void lw_phase(const StepParams<T> &p, typename V2<T>::t *sPhi, typename V2<T>::t *sPi,
                                         const T *sRt, const T *sTh, int r0, int nr, int g0, int ctid, int NC,
                                         bool src, typename V2<T>::t ph1, typename V2<T>::t ph2, Bar bar)
{
    typedef typename V2<T>::t c2;
    const int N = p.Nth, P = p.pitch;
    const c2 zero = cmk<c2>(T(0), T(0));
    if (N <= NC) {
        const int nseg = NC / N;
        const int sl = (nr + nseg - 1) / nseg;
        const int j = ctid % N, sgm = ctid / N;
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
        if (work) lw_segment<T, INTERIOR>(p, sPhi, sPi, sRt, sTh, j, ra, rb, pf, pg, nf, ng, g0, ph1, ph2, src);
    } else {
        // each thread owns whole columns: rows r0-1 and r0+nr are read before any write
        for (int j = ctid; j < N; j += NC) {
            c2 pf = sPhi[(r0 - 1) * P + j], pg = sPi[(r0 - 1) * P + j];
            c2 nf = sPhi[(r0 + nr) * P + j], ng = sPi[(r0 + nr) * P + j];
            lw_segment<T, INTERIOR>(p, sPhi, sPi, sRt, sTh, j, r0, r0 + nr, pf, pg, nf, ng, g0, ph1, ph2, src);
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
// index), for KS = 1 or 2 time steps per launch.  The tile holds its TR output
// rows plus KS halo rows on either side (R = TR + 2 KS; tile row lr is global
// row g0 + lr, g0 = i0 - KS).  With KS = 2 the first step updates rows
// 1 .. R-2 and the second the TR output rows; the state read and written per
// step halves at the cost of recomputing the extra halo rows.  The result is
// bitwise that of KS single steps.
template <typename T, int S, int KS>
__device__ __forceinline__ void split_tile(const StepParams<T> &p, int tile, int ntiles)
{
    typedef typename V2<T>::t c2;
    constexpr int kMaxChunks = 8;
    static_assert(KS == 1 || KS == 2, "one or two steps per launch");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double2 sph[2 * KS];
    __shared__ long long s_n;
    __shared__ __align__(8) unsigned long long s_mbar[kMaxChunks];
    __shared__ int s_plan[kMaxTileRows + 4];   // stored scan levels of the tile rows
    const int Nr = p.Nr, N = p.Nth, TR = p.tile_rows, R = TR + 2 * KS, P = p.pitch;
    const int tid = threadIdx.x, NT = blockDim.x;
    const int i0 = tile * TR, g0 = i0 - KS;
    const int G = p.group;

    const SplitSmem plan = split_smem_plan(R, N, (int)sizeof(T));
    c2 *sPhi = (c2 *)(smem_raw + plan.phi);
    c2 *sPi = (c2 *)(smem_raw + plan.pi);
    c2 *sPiv = (c2 *)(smem_raw + plan.piv);
    T *sRt = (T *)(smem_raw + plan.rt);
    T *sTh = (T *)(smem_raw + plan.th);
    c2 *xPhi = (c2 *)(smem_raw + plan.total);   // KS = 2: copy of the extraction row
    c2 *xPi = xPhi + N;
    // implicit step of this launch: dt/2 for the first step and for the state output
    const ImpConst<T> &K = (p.first || p.imp_only) ? p.half : p.full;

    const bool src = !p.imp_only && p.patch_np > 0 && i0 + TR + KS - 1 >= p.patch_p0 &&
                     g0 <= p.patch_p0 + p.patch_np;
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
                sph[2 * k] = phase_at(p.mOmega, t);
                sph[2 * k + 1] = phase_at(p.mOmega, t + 0.5 * p.dt64);
            }
    }
    // ---- A: tile rows g0 .. g0+R-1 (state and pivots), r and theta tables
    const c2 zero = cmk<c2>(T(0), T(0));
    // (row, column) walk of the tile without integer division in the loop
    const int t_lr = tid / N, t_j = tid - t_lr * N;
    const int d_lr = NT / N, d_j = NT - d_lr * N;
    // rows of the tile that exist on the grid: [ga, gb] globally, from tile row la
    const int ga = g0 < 0 ? 0 : g0;
    const int gb = g0 + R - 1 > Nr - 1 ? Nr - 1 : g0 + R - 1;
    const int la = ga - g0, nrows = gb - ga + 1;
    // The state tile arrives in chunks of whole implicit passes, one mbarrier
    // each, so that the first pass can start while later rows are in flight.
    const int rpp = NT / G;   // theta rows per implicit pass
    int cr = rpp;             // rows per chunk
    while ((R + cr - 1) / cr > kMaxChunks) cr += rpp;
    const int nch = (R + cr - 1) / cr;
    if (p.bulk) {
        if (tid == 0) {
            for (int c = 0; c < nch; ++c) mbar_init(&s_mbar[c], 1);
            for (int c = 0; c < nch; ++c) {
                int r0 = c * cr, r1 = r0 + cr;
                if (r1 > R) r1 = R;
                if (r0 < la) r0 = la;
                if (r1 > la + nrows) r1 = la + nrows;
                unsigned bytes = r1 > r0 ? (unsigned)(r1 - r0) * (unsigned)N * (unsigned)sizeof(c2) : 0u;
                mbar_expect_tx(&s_mbar[c], 3 * bytes);   // with no bytes this is a plain arrival
                if (bytes) {
                    const size_t gr = (size_t)(ga + r0 - la);
                    bulk_g2s(sPhi + r0 * P, p.uin + gr * N, bytes, &s_mbar[c]);
                    bulk_g2s(sPi + r0 * P, p.uin + ((size_t)Nr + gr) * N, bytes, &s_mbar[c]);
                    bulk_g2s(sPiv + r0 * P, K.piv + gr * N, bytes, &s_mbar[c]);
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
            c2 fv = zero, gv = zero, ev = zero;
            if (gi >= 0 && gi < Nr) {
                fv = p.uin[(size_t)gi * N + j];
                gv = p.uin[((size_t)Nr + gi) * N + j];
                ev = K.piv[(size_t)gi * N + j];
            }
            sPhi[lr * P + j] = fv;
            sPi[lr * P + j] = gv;
            sPiv[lr * P + j] = ev;
            lr += d_lr;
            j += d_j;
            if (j >= N) { j -= N; ++lr; }
        }
    }
    {
        // r-table positions 2 g0 .. 2(g0+R-1); those off the grid are zero
        const long long pbase = 2LL * g0;
        const long long pmax = 2LL * Nr - 2;
        for (int idx = tid; idx < (2 * R - 1) * NRF; idx += NT) {
            int e = idx / NRF, q = idx - e * NRF;
            long long pos = pbase + e;
            sRt[idx] = (pos >= 0 && pos <= pmax) ? p.rtab[(size_t)pos * NRF + q] : T(0);
        }
    }
    for (int idx = tid; idx < NTF * N; idx += NT) sTh[idx] = p.thtab[idx];
    // Every implicit step of the launch uses K: with two steps per launch K
    // is the full step (the launcher refuses first steps and state outputs).
    for (int lr = tid; lr < R; lr += NT) {
        const int gi = g0 + lr;
        s_plan[lr] = (gi >= 0 && gi < Nr) ? K.plan[gi] : 0;
    }
    __syncthreads();
    const int g = tid % G;
    const bool vec = p.vec != 0;
    // implicit step on tile rows [lo, hi)
    auto implicit_rows = [&](const ImpConst<T> &Ki, int lo, int hi, bool wait_chunks, int &ok) {
        for (int base = lo; base < hi; base += rpp) {
            if (wait_chunks && p.bulk && ok) {
                // the chunks that hold this pass's rows
                int last = base + rpp - 1;
                if (last > hi - 1) last = hi - 1;
                for (int c = base / cr; c <= last / cr; ++c) ok &= (int)mbar_wait(&s_mbar[c], 0, kWaitLimit);
            }
            int lr = base + tid / G;
            bool in_tile = lr < hi;
            int gi = g0 + lr;
            bool active = in_tile && gi >= 1 && gi <= Nr - 2;
            int lrc = in_tile ? lr : lo;
            implicit_row_group<T, S>(Ki, sPhi + lrc * P, sPi + lrc * P, sPiv + lrc * P, sRt + 2 * lrc * NRF, sTh, N,
                                     active, in_tile, g, G, vec, s_plan[lrc]);
        }
    };
    // physical sample u = C_{dt/2} s of the extraction row (tile row lx) in
    // place, or of its copy in (xPhi, xPi); warp 0
    auto extract_row = [&](int lx, long long slot, bool copy) {
        if (tid < 32) {
            c2 *rf = copy ? xPhi : sPhi + lx * P, *rg = copy ? xPi : sPi + lx * P;
            bool mine = tid < G;
            bool active = mine && p.i_ext >= 1 && p.i_ext <= Nr - 2;
            implicit_row_group<T, S>(p.half, rf, rg, p.half.piv + (size_t)p.i_ext * N, sRt + 2 * lx * NRF, sTh, N,
                                     active, mine, tid % G, G, vec, p.half.plan[p.i_ext]);
            __syncwarp();
            extract_warp<T>(p, rf, slot);
        }
    };
    const bool ext = !p.imp_only && p.nfix < 0 && p.i_ext >= i0 && p.i_ext < i0 + TR && p.i_ext < Nr;
    // ---- B and C, once per time step of the launch.  Step k (from 0) runs
    // the implicit stage on tile rows k .. R-1-k and the Lax-Wendroff stages
    // on rows k+1 .. R-2-k, so the output rows KS .. KS+TR-1 are exact after
    // the last step.  One loop body serves every step: the two-step kernel's
    // code is no larger than the one-step kernel's.
    int ok = 1;   // every bounded wait of this thread succeeded
    const auto sync_all = [] { __syncthreads(); };
#pragma unroll 1
    for (int k = 0; k < KS; ++k) {
        // implicit step: dt/2 for a first step and for the state output, else dt
        const ImpConst<T> &Ki = k == 0 ? K : p.full;
        const int lo = p.imp_only ? KS : k, hi = p.imp_only ? TR + KS : R - k;
        implicit_rows(Ki, lo, hi, k == 0, ok);
        if (k == 0) {
            // the remaining phases read every row of the tile
            if (p.bulk && ok)
                for (int c = 0; c < nch; ++c) ok &= (int)mbar_wait(&s_mbar[c], 0, kWaitLimit);
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
        } else {
            __syncthreads();
        }
        c2 ph1 = zero, ph2 = zero;
        if (src) {
            ph1 = from_d2<T>(sph[2 * k]);
            ph2 = from_d2<T>(sph[2 * k + 1]);
        }
        // rows g0 .. g0+R-1 all inside [1, Nr-2] except in the first and last tiles
        if (g0 >= 1 && g0 + R <= Nr - 1)
            lw_phase<T, true>(p, sPhi, sPi, sRt, sTh, k + 1, R - 2 - 2 * k, g0, tid, NT, src, ph1, ph2, sync_all);
        else
            lw_phase<T, false>(p, sPhi, sPi, sRt, sTh, k + 1, R - 2 - 2 * k, g0, tid, NT, src, ph1, ph2, sync_all);
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

template <typename T, int S>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && S <= 4) ? 2 : 1) k_split_step(const StepParams<T> p)
{
    split_tile<T, S, 1>(p, (int)blockIdx.x, (int)gridDim.x);
}

// Two time steps per launch (temporal blocking): see split_tile.
template <typename T, int S>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && S <= 4) ? 2 : 1) k_split_step2(const StepParams<T> p)
{
    split_tile<T, S, 2>(p, (int)blockIdx.x, (int)gridDim.x);
}

// Batched split step: every CTA takes entry blockIdx.x of the tile list,
// (instance, tile), stages that instance's parameters in shared memory and
// computes the tile.  One launch advances every instance of the batch by one
// step; the instances may differ in every parameter (grid, spin, mode,
// source, tile height) as long as they share the state precision and the
// theta segment S.  KS = 2: two time steps per launch, as k_split_step2.
template <typename T, int S, int KS>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && S <= 4) ? 2 : 1)
    k_split_batch(const StepParams<T> *params, const int2 *tiles)
{
    __shared__ __align__(16) StepParams<T> sp;
    static_assert(sizeof(StepParams<T>) % 4 == 0 && sizeof(StepParams<T>) <= 4 * 256, "parameter copy");
    const int2 e = tiles[blockIdx.x];
    if (threadIdx.x < sizeof(StepParams<T>) / 4)
        reinterpret_cast<int *>(&sp)[threadIdx.x] = reinterpret_cast<const int *>(params + e.x)[threadIdx.x];
    __syncthreads();
    split_tile<T, S, KS>(sp, e.y, (sp.Nr + sp.tile_rows - 1) / sp.tile_rows);
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *m)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(m)) : "memory");
}

// Persistent form of k_split_step (same arithmetic, same output).  The CTA
// keeps the theta tables and walks the tiles blockIdx.x, blockIdx.x +
// gridDim.x, ...  Warp NC/32 is the producer: its lane 0 loads tile k+2 into
// the buffer that tile k used as soon as tile k is stored, so tiles arrive
// while the NC consumer threads compute the previous one.  Per buffer b:
//   full[b]   completes when the tile's state rows and r-table entries are
//             resident (transaction count);
//   empty[b]  completes when every consumer warp has finished the tile and
//             fenced its shared-memory writes for the bulk store.
// Every wait is bounded; a lost copy sets FLAG_TIMEOUT and ends the CTA.
// Registers per thread so that one CTA of NC + 32 threads fits an SM: its
// warps are spread over the SM's four sub-partitions of 16K registers each.
template <int NC> struct PersistRegs {
    static constexpr int warps_per_quarter = (NC / 32 + 1 + 3) / 4;
    static constexpr int raw = 16384 / (warps_per_quarter * 32);
    static constexpr int v = (raw > 255 ? 255 : raw) / 8 * 8;
};

template <typename T, int S, int NC>
__global__ void __maxnreg__(PersistRegs<NC>::v) k_split_persist(const StepParams<T> p)
{
    typedef typename V2<T>::t c2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double2 sph[2];
    __shared__ long long s_n;
    __shared__ __align__(8) unsigned long long s_full[2], s_empty[2];
    const int Nr = p.Nr, N = p.Nth, TR = p.tile_rows, R = TR + 2, P = p.pitch;
    const int tid = threadIdx.x;
    const int G = p.group;
    const PersistSmem plan = persist_smem_plan(R, N, (int)sizeof(T));
    T *sTh = (T *)(smem_raw + plan.th);
    c2 *xPhi = (c2 *)(smem_raw + plan.xphi);
    c2 *xPi = (c2 *)(smem_raw + plan.xpi);
    T *xF = (T *)(smem_raw + plan.xf);
    auto bphi = [&](int b) { return (c2 *)(smem_raw + plan.buf + b * plan.bsize); };
    auto bpi = [&](int b) { return (c2 *)(smem_raw + plan.buf + b * plan.bsize + plan.bpi); };
    auto bpiv = [&](int b) { return (c2 *)(smem_raw + plan.buf + b * plan.bsize + plan.bpiv); };
    auto brt = [&](int b) { return (T *)(smem_raw + plan.buf + b * plan.bsize + plan.brt); };
    const ImpConst<T> &K = p.first ? p.half : p.full;
    const int ntiles = (Nr + TR - 1) / TR;
    const int nmine = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    // Geometry of tile number it of this CTA: on-grid rows [ga, gb] from tile
    // row la (nrows of them), on-grid r-table positions from entry lp (npos).
    struct Geo {
        int i0, ga, la, nrows, pos0, lp, npos;
    };
    auto geo = [&](int it) {
        Geo q;
        q.i0 = ((int)blockIdx.x + it * (int)gridDim.x) * TR;
        q.ga = q.i0 - 1 < 0 ? 0 : q.i0 - 1;
        const int gb = q.i0 + TR > Nr - 1 ? Nr - 1 : q.i0 + TR;
        q.la = q.ga - (q.i0 - 1);
        q.nrows = gb - q.ga + 1;
        const int pb = 2 * (q.i0 - 1), pe0 = 2 * (q.i0 + TR);
        q.pos0 = pb < 0 ? 0 : pb;
        const int pe = pe0 > 2 * Nr - 2 ? 2 * Nr - 2 : pe0;
        q.lp = q.pos0 - pb;
        q.npos = pe - q.pos0 + 1;
        return q;
    };

    if (tid == 0) {
        long long n = *((volatile long long *)&p.ctl->step);
        s_n = n;
        // the last CTA to read the step index advances it
        __threadfence();
        unsigned t = atomicAdd(&p.ctl->ticket, 1u);
        if (t == gridDim.x - 1) {
            p.ctl->ticket = 0u;
            p.ctl->step = n + 1;
        }
        if (p.patch_np > 0) {
            double tt = (double)n * p.dt64;
            sph[0] = phase_at(p.mOmega, tt);
            sph[1] = phase_at(p.mOmega, tt + 0.5 * p.dt64);
        }
        mbar_init(&s_full[0], 1);
        mbar_init(&s_full[1], 1);
        mbar_init(&s_empty[0], NC / 32);
        mbar_init(&s_empty[1], NC / 32);
    }
    for (int idx = tid; idx < NTF * N; idx += blockDim.x) sTh[idx] = p.thtab[idx];
    __syncthreads();

    if (tid >= NC) {
        // ---------------- producer
        if (tid != NC) return;
        auto load = [&](int it) {
            const int b = it & 1;
            const Geo q = geo(it);
            const unsigned bs = (unsigned)q.nrows * (unsigned)N * (unsigned)sizeof(c2);
            const unsigned br = (unsigned)q.npos * NRF * (unsigned)sizeof(T);
            mbar_expect_tx(&s_full[b], 3 * bs + br);
            bulk_g2s(bphi(b) + q.la * P, p.uin + (size_t)q.ga * N, bs, &s_full[b]);
            bulk_g2s(bpi(b) + q.la * P, p.uin + ((size_t)Nr + q.ga) * N, bs, &s_full[b]);
            bulk_g2s(bpiv(b) + q.la * P, K.piv + (size_t)q.ga * N, bs, &s_full[b]);
            bulk_g2s(brt(b) + q.lp * NRF, p.rtab + (size_t)q.pos0 * NRF, br, &s_full[b]);
        };
        if (nmine > 0) load(0);
        if (nmine > 1) load(1);
        for (int it = 0; it < nmine; ++it) {
            const int b = it & 1;
            if (!mbar_wait(&s_empty[b], (unsigned)((it >> 1) & 1), kWaitLimit)) {
                atomicOr(&p.ctl->flags, FLAG_TIMEOUT);
                break;
            }
            const Geo q = geo(it);
            const int nout = (Nr - q.i0) < TR ? (Nr - q.i0) : TR;
            const unsigned bytes = (unsigned)nout * (unsigned)N * (unsigned)sizeof(c2);
            bulk_s2g(p.uout + (size_t)q.i0 * N, bphi(b) + P, bytes);
            bulk_s2g(p.uout + ((size_t)Nr + q.i0) * N, bpi(b) + P, bytes);
            bulk_commit();
            if (it + 2 < nmine) {
                bulk_wait_read();   // buffer b is read out: refill it
                load(it + 2);
            }
        }
        bulk_wait_read();
        return;
    }

    // ---------------- consumers (threads 0 .. NC-1)
    const c2 zero = cmk<c2>(T(0), T(0));
    const int rpp = NC / G;
    const int g = tid % G;
    const bool vec = p.vec != 0;
    const int t_lr = tid / N, t_j = tid - t_lr * N;
    const int d_lr = NC / N, d_j = NC - d_lr * N;
    c2 ph1 = zero, ph2 = zero;
    if (p.patch_np > 0) {
        ph1 = from_d2<T>(sph[0]);
        ph2 = from_d2<T>(sph[1]);
    }
    auto bar = [] { named_sync(1, NC); };
    for (int it = 0; it < nmine; ++it) {
        const int b = it & 1;
        const Geo q = geo(it);
        const int i0 = q.i0;
        c2 *sPhi = bphi(b), *sPi = bpi(b);
        const c2 *sPiv = bpiv(b);
        T *sRt = brt(b);
        const int ok = (int)mbar_wait(&s_full[b], (unsigned)((it >> 1) & 1), kWaitLimit);
        if (!named_sync_and(1, NC, ok)) {
            if (tid == 0) atomicOr(&p.ctl->flags, FLAG_TIMEOUT);
            return;
        }
        // off-grid rows and r-table entries (first and last tile) are zero
        if (q.la > 0 || q.la + q.nrows < R) {
            for (int lr = t_lr, j = t_j; lr < R;) {
                if (lr < q.la || lr >= q.la + q.nrows) {
                    sPhi[lr * P + j] = zero;
                    sPi[lr * P + j] = zero;
                }
                lr += d_lr;
                j += d_j;
                if (j >= N) { j -= N; ++lr; }
            }
        }
        if (q.lp > 0 || q.lp + q.npos < 2 * R - 1) {
            for (int idx = tid; idx < (2 * R - 1) * NRF; idx += NC) {
                int e = idx / NRF;
                if (e < q.lp || e >= q.lp + q.npos) sRt[idx] = T(0);
            }
        }
        bar();
        // implicit step on all R rows
        for (int base = 0; base < R; base += rpp) {
            int lr = base + tid / G;
            bool in_tile = lr < R;
            int gi = i0 - 1 + lr;
            bool active = in_tile && gi >= 1 && gi <= Nr - 2;
            int lrc = in_tile ? lr : 0;
            implicit_row_group<T, S>(K, sPhi + lrc * P, sPi + lrc * P, sPiv + lrc * P, sRt + 2 * lrc * NRF, sTh, N,
                                     active, in_tile, g, G, vec, active ? K.plan[gi] : 0);
        }
        bar();
        // The extraction row (its r-table entry and, after the Lax-Wendroff
        // phase, its state) is copied out for the sample below: the buffer
        // is refilled once it is handed back.
        const bool ext = p.i_ext >= i0 && p.i_ext < i0 + TR && p.i_ext < Nr;
        const int lx = p.i_ext - i0 + 1;
        if (ext && tid < NRF) xF[tid] = sRt[2 * lx * NRF + tid];
        const bool src = p.patch_np > 0 && i0 + TR >= p.patch_p0 && i0 - 1 <= p.patch_p0 + p.patch_np;
        lw_phase<T, false>(p, sPhi, sPi, sRt, sTh, 1, TR, i0 - 1, tid, NC, src, ph1, ph2, bar);
        bar();
        if (ext && tid < 32) {
            for (int j = tid; j < N; j += 32) {
                xPhi[j] = sPhi[lx * P + j];
                xPi[j] = sPi[lx * P + j];
            }
        }
        fence_proxy_async();   // this thread's shared-memory writes become visible to the bulk store
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&s_empty[b]);
        // physical sample u_{n+1} = C_{dt/2} s_{n+1} on the extraction row
        if (ext && tid < 32) {
            bool mine = tid < G;
            bool active = mine && p.i_ext >= 1 && p.i_ext <= Nr - 2;
            implicit_row_group<T, S>(p.half, xPhi, xPi, p.half.piv + (size_t)p.i_ext * N, xF, sTh, N, active, mine,
                                     tid % G, G, vec, p.half.plan[p.i_ext]);
            __syncwarp();
            extract_warp<T>(p, xPhi, s_n + 1);
        }
    }
}

// ---------------------------------------------------------------- adjoint

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

// h = E u with u = s (physical) or u = C_{dt/2} s on the extraction row; one
// warp.  The sum is the one the step kernels write to the waveform buffer.
// Stored scan plans: the levels scan_plan chooses for every row of the
// grid and both implicit steps (dt and dt/2), from the same coefficient path
// as implicit_row_group (r table, theta tables and pivots as the step
// kernels stage them).  One CTA of 256 threads covers 256 / G rows.
template <typename T, int S>
__global__ void __launch_bounds__(256) k_scan_plans(const StepParams<T> p, int *plan_full, int *plan_half)
{
    typedef typename V2<T>::t c2;
    const int N = p.Nth, Nr = p.Nr, G = p.group;
    const int tid = threadIdx.x, g = tid % G;
    const int gi = (int)blockIdx.x * ((int)blockDim.x / G) + tid / G;
    const bool in_grid = gi < Nr;
    const bool active = in_grid && gi >= 1 && gi <= Nr - 2;
    const int gr = in_grid ? gi : 0;
    const int j0 = g * S;
    int len = N - j0;
    len = len < 0 ? 0 : (len > S ? S : len);
    if (!active) len = 0;
    for (int h = 0; h < 2; ++h) {
        const ImpConst<T> &K = h ? p.half : p.full;
        const c2 *prow = K.piv + (size_t)gr * N;
        RowCoef<T, S> C;
        c2 w[S], y[S];
        // the state rows are not needed: the pivot row stands in for them
        row_load<T, S>(K, prow, prow, prow, p.rtab + (size_t)(2 * gr) * NRF, p.thtab, N, len, j0, G, p.vec != 0, C, w, y);
        const ScanPlan<T> P = scan_plan<T, S>(C.m, C.fk, g, G);
        if (in_grid && g == 0) (h ? plan_half : plan_full)[gi] = P.nf | (P.nb << 8);
    }
}

template <typename T, int S>
__global__ void __launch_bounds__(32) k_sample(const StepParams<T> p, const typename V2<T>::t *s, int physical,
                                               double2 *h_out)
{
    typedef typename V2<T>::t c2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = p.Nth, Nr = p.Nr, i = p.i_ext, tid = threadIdx.x;
    c2 *xPhi = (c2 *)smem_raw;
    c2 *xPi = xPhi + ((N + 1) & ~1);
    T *xF = (T *)(xPi + ((N + 1) & ~1));
    T *xTh = xF + NRF;
    for (int j = tid; j < N; j += 32) {
        xPhi[j] = s[(size_t)i * N + j];
        xPi[j] = s[((size_t)Nr + i) * N + j];
    }
    if (tid < NRF) xF[tid] = p.rtab[(size_t)(2 * i) * NRF + tid];
    for (int k = tid; k < NTF * N; k += 32) xTh[k] = p.thtab[k];
    __syncwarp();
    if (!physical) {
        const int G = p.group;
        const bool mine = tid < G;
        const bool active = mine && i >= 1 && i <= Nr - 2;
        implicit_row_group<T, S>(p.half, xPhi, xPi, p.half.piv + (size_t)i * N, xF, xTh, N, active, mine, tid % G, G,
                                 p.vec != 0, p.half.plan[i]);
        __syncwarp();
    }
    double2 h = sample_warp<T>(p, xPhi);
    if (tid == 0) *h_out = h;
}

// Adds conj(lam) * coef * (unit source) * phase to the amplitude sum cA and
// conj(lam) * coef * (source) * (rho d r0*/d r0 - i m Omega' t) to the orbit
// sum cr (rho = (r* - r0*)/sigma_r^2): the derivatives of the source term
// A F_pref G(r*, theta) e^{-i m Omega t} with respect to A and r0.
template <typename T>
__device__ __forceinline__ void source_grad(const StepParams<T> &p, typename V2<T>::t lam, double coef,
                                            typename V2<T>::t u, double2 ph, double rs, double t, double2 &cA,
                                            double2 &cr)
{
    const double lr = (double)lam.x, li = -(double)lam.y;             // conj(lam)
    const double ur = (double)u.x * ph.x - (double)u.y * ph.y, ui = (double)u.x * ph.y + (double)u.y * ph.x;
    const double vr = coef * (lr * ur - li * ui), vi = coef * (lr * ui + li * ur);   // conj(lam) coef U ph
    cA.x += vr;
    cA.y += vi;
    const double fr = p.amp_re * vr - p.amp_im * vi, fi = p.amp_re * vi + p.amp_im * vr;   // times A
    const double zr = (rs - p.rs0) * p.inv_sig_r2 * p.drs0_dr0, zi = -p.m_dOmega * t;
    cr.x += fr * zr - fi * zi;
    cr.y += fr * zi + fi * zr;
}

// Hermitian adjoint of one split step s_n -> s_{n+1} = LW_n C_h s_n (h = dt;
// h = dt/2 and a physical input when p.first), plus the extraction seed:
//   lam_n = C_h^H LW^H lam_{n+1} + C_{dt/2}^H E^H g_n     (E^H g_0 when first)
// where LW is the linear part of the two Lax-Wendroff stages (Eqs. 13-14)
// and E u = sum_j w_j Phi_{i_ext, j}.  p.uin holds lam_{n+1}, p.uout gets
// lam_n, p.nfix = n.  Each CTA owns TR output rows and reads one halo row on
// either side.  The transposed stages are written in gather form: every
// midpoint adjoint (mF, mG) from its two nodes, then every node from its two
// midpoints.  The CTA's contributions to the source derivatives
// (sum over steps of <lam_{n+1}, dF_n/dp> for p = Re A, Im A, r0) go to
// part[4 blockIdx.x + (0..3)] = (Re cA, Im cA, Re cr, Im cr).
template <typename T, int S>
__global__ void __launch_bounds__(256, 1) k_adjoint_step(const StepParams<T> p, const double2 *gseed, double *part)
{
    typedef typename V2<T>::t c2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double s_red[8][4];
    const int Nr = p.Nr, N = p.Nth, TR = p.tile_rows, R = TR + 2, P = N;
    const int tid = threadIdx.x, NT = blockDim.x;
    const int i0 = blockIdx.x * TR;
    const int G = p.group;
    const bool first = p.first != 0;
    const ImpConst<T> &K = first ? p.half : p.full;
    const long long n = p.nfix;
    const T hdt = p.half_dt, dt = p.dt, ri = p.drs_inv;
    const c2 zero = cmk<c2>(T(0), T(0));

    const unsigned plane = (unsigned)R * (unsigned)N;
    c2 *lF = (c2 *)smem_raw;
    c2 *lG = lF + plane;
    c2 *mF = lG + plane;
    c2 *mG = mF + plane;
    T *sRt = (T *)(mG + plane);
    T *sTh = sRt + (2 * R - 1) * NRF;

    // ---- load lam_{n+1} on rows i0-1 .. i0+TR, the r and theta tables
    for (int idx = tid; idx < R * N; idx += NT) {
        int lr = idx / N, j = idx - lr * N;
        int gi = i0 - 1 + lr;
        c2 f = zero, g = zero;
        if (gi >= 0 && gi < Nr) {
            f = p.uin[(size_t)gi * N + j];
            g = p.uin[((size_t)Nr + gi) * N + j];
        }
        lF[idx] = f;
        lG[idx] = g;
    }
    {
        const long long pbase = 2LL * (i0 - 1), pmax = 2LL * Nr - 2;
        for (int idx = tid; idx < (2 * R - 1) * NRF; idx += NT) {
            int e = idx / NRF, q = idx - e * NRF;
            long long pos = pbase + e;
            sRt[idx] = (pos >= 0 && pos <= pmax) ? p.rtab[(size_t)pos * NRF + q] : T(0);
        }
    }
    for (int idx = tid; idx < NTF * N; idx += NT) sTh[idx] = p.thtab[idx];
    __syncthreads();

    const bool src = p.unit_np > 0 && i0 + TR >= p.unit_p0 && i0 - 1 <= p.unit_p0 + p.unit_np;
    double2 ph1 = make_double2(0.0, 0.0), ph2 = ph1;
    const double t1 = (double)n * p.dt64, t2 = t1 + 0.5 * p.dt64;
    if (src) {
        ph1 = phase_at(p.mOmega, t1);
        ph2 = phase_at(p.mOmega, t2);
    }
    double2 cA = make_double2(0.0, 0.0), cr = cA;
    auto node_bK = [&](int lr, int j, T &b, c2 &Kc) {
        T f[12];
        vload<12>(f, sRt + 2 * lr * NRF);
        const T S2 = sTh[TF_S2 * N + j], C = sTh[TF_C * N + j];
        bK<T>(f, rsq_(fma(-f[RF_AD], S2, f[RF_R2])), S2, C, b, Kc);
    };
    auto half_bK = [&](int k, int j, T &b, c2 &Kc) {
        T f[12];
        vload<12>(f, sRt + (2 * k + 1) * NRF);
        const T S2 = sTh[TF_S2 * N + j], C = sTh[TF_C * N + j];
        bK<T>(f, rsq_(fma(-f[RF_AD], S2, f[RF_R2])), S2, C, b, Kc);
    };

    // ---- adjoints of the midpoints k = 0 .. R-2 (between tile rows k, k+1)
    for (int idx = tid; idx < (R - 1) * N; idx += NT) {
        int k = idx / N, j = idx - k * N;
        int gl = i0 - 1 + k;
        c2 vF = zero, vG = zero;
        if (gl >= 0 && gl <= Nr - 2) {
            if (gl >= 1) {   // lower node interior (gl <= Nr - 2 holds)
                T b;
                c2 Kc;
                node_bK(k, j, b, Kc);
                const c2 lf = lF[k * P + j], lg = lG[k * P + j];
                const T cb = dt * b * ri;
                const c2 cK = cscale<c2>(dt * ri, Kc);
                vF = csub(cmul(conj_c(cK), lg), cscale<c2>(cb, lf));
                vG = cscale<c2>(cb, lg);
            }
            if (gl + 1 <= Nr - 2) {   // upper node interior (gl + 1 >= 1 holds)
                T b;
                c2 Kc;
                node_bK(k + 1, j, b, Kc);
                const c2 lf = lF[(k + 1) * P + j], lg = lG[(k + 1) * P + j];
                const T cb = dt * b * ri;
                const c2 cK = cscale<c2>(dt * ri, Kc);
                vF = cadd(vF, csub(cscale<c2>(cb, lf), cmul(conj_c(cK), lg)));
                vG = csub(vG, cscale<c2>(cb, lg));
            }
            // stage-1 source at this midpoint (owned by the tile of its lower node)
            if (src && k >= 1 && k <= TR) {
                int pr = gl - p.unit_p0;
                if (pr >= 0 && pr < p.unit_np)
                    source_grad<T>(p, vG, (double)hdt, p.patchu[((size_t)pr * 2 + 1) * N + j], ph1,
                                   p.rs_min64 + ((double)gl + 0.5) * p.drs64, t1, cA, cr);
            }
        }
        mF[idx] = vF;
        mG[idx] = vG;
    }
    __syncthreads();

    // ---- adjoints of the nodes (inputs of the Lax-Wendroff stages), rows 1..TR
    for (int idx = tid; idx < TR * N; idx += NT) {
        int lr = 1 + idx / N, j = idx - (lr - 1) * N;
        int gi = i0 - 1 + lr;
        if (gi >= Nr) continue;
        const c2 lf = lF[lr * P + j], lg = lG[lr * P + j];
        const bool interior = gi >= 1 && gi <= Nr - 2;
        c2 vF = interior ? lf : zero, vG = interior ? lg : zero;
        if (gi <= Nr - 2) {   // midpoint lr (to the next row)
            T b;
            c2 Kc;
            half_bK(lr, j, b, Kc);
            const T c = hdt * b * ri;
            const c2 kap = cscale<c2>(hdt * ri, Kc);
            const c2 mf = mF[lr * P + j], mg = mG[lr * P + j];
            vF = cadd(vF, csub(cscale<c2>(T(0.5) + c, mf), cmul(conj_c(kap), mg)));
            vG = cadd(vG, cscale<c2>(T(0.5) - c, mg));
        }
        if (gi >= 1) {   // midpoint lr - 1 (to the previous row)
            T b;
            c2 Kc;
            half_bK(lr - 1, j, b, Kc);
            const T c = hdt * b * ri;
            const c2 kap = cscale<c2>(hdt * ri, Kc);
            const c2 mf = mF[(lr - 1) * P + j], mg = mG[(lr - 1) * P + j];
            vF = cadd(vF, cadd(cscale<c2>(T(0.5) - c, mf), cmul(conj_c(kap), mg)));
            vG = cadd(vG, cscale<c2>(T(0.5) + c, mg));
        }
        // stage-2 source at this node
        if (src && interior) {
            int pr = gi - p.unit_p0;
            if (pr >= 0 && pr < p.unit_np)
                source_grad<T>(p, lg, (double)dt, p.patchu[((size_t)pr * 2) * N + j], ph2,
                               p.rs_min64 + (double)gi * p.drs64, t2, cA, cr);
        }
        lF[lr * P + j] = vF;
        lG[lr * P + j] = vG;
    }
    __syncthreads();

    // ---- C_h^H on the output rows
    {
        const int rpp = NT / G;
        const int g = tid % G;
        const bool vec = p.vec != 0;
        for (int base = 1; base <= TR; base += rpp) {
            int lr = base + tid / G;
            bool in_tile = lr <= TR && i0 - 1 + lr < Nr;
            int gi = i0 - 1 + lr;
            bool active = in_tile && gi >= 1 && gi <= Nr - 2;
            int lrc = in_tile ? lr : 1;
            implicit_row_adjoint<T, S>(K, lF + lrc * P, lG + lrc * P, K.piv + (size_t)(active ? gi : 1) * N,
                                       sRt + 2 * lrc * NRF, sTh, N, active, in_tile, g, G, vec);
        }
    }
    __syncthreads();

    // ---- extraction seed: C_{dt/2}^H E^H g_n (E^H g_0 for a physical input)
    const bool ext = gseed != nullptr && p.i_ext >= i0 && p.i_ext < i0 + TR && p.i_ext < Nr;
    if (ext) {
        const int lx = p.i_ext - i0 + 1;
        c2 *xF = mF, *xG = mG;
        if (tid < 32) {
            const double2 gv = *gseed;
            for (int j = tid; j < N; j += 32) {
                const double w = p.w[j];
                xF[j] = cmk<c2>((T)(w * gv.x), (T)(w * gv.y));
                xG[j] = zero;
            }
            __syncwarp();
            if (!first) {
                const bool mine = tid < G;
                const bool active = mine && p.i_ext >= 1 && p.i_ext <= Nr - 2;
                implicit_row_adjoint<T, S>(p.half, xF, xG, p.half.piv + (size_t)p.i_ext * N, sRt + 2 * lx * NRF, sTh,
                                           N, active, mine, tid % G, G, p.vec != 0);
                __syncwarp();
            }
            for (int j = tid; j < N; j += 32) {
                lF[lx * P + j] = cadd(lF[lx * P + j], xF[j]);
                lG[lx * P + j] = cadd(lG[lx * P + j], xG[j]);
            }
        }
        __syncthreads();
    }

    // ---- store lam_n
    for (int idx = tid; idx < TR * N; idx += NT) {
        int lr = 1 + idx / N, j = idx - (lr - 1) * N;
        int gi = i0 - 1 + lr;
        if (gi >= Nr) continue;
        p.uout[(size_t)gi * N + j] = lF[lr * P + j];
        p.uout[((size_t)Nr + gi) * N + j] = lG[lr * P + j];
    }

    // ---- this CTA's source-derivative sums (fixed-order reduction)
    double v[4] = {cA.x, cA.y, cr.x, cr.y};
#pragma unroll
    for (int c = 0; c < 4; ++c)
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
    if ((tid & 31) == 0)
        for (int c = 0; c < 4; ++c) s_red[tid >> 5][c] = v[c];
    __syncthreads();
    if (tid < 4) {
        double acc = 0.0;
        for (int w = 0; w < NT / 32; ++w) acc += s_red[w][tid];
        part[4 * blockIdx.x + tid] = acc;
    }
}

// acc[c] += sum over the nblk CTAs of part[4 b + c], in a fixed order.
__global__ void __launch_bounds__(32) k_part_reduce(const double *part, int nblk, double *acc)
{
    const int lane = threadIdx.x;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = lane; b < nblk; b += 32)
        for (int c = 0; c < 4; ++c) v[c] += part[4 * b + c];
    for (int c = 0; c < 4; ++c)
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
    if (lane == 0)
        for (int c = 0; c < 4; ++c) acc[c] += v[c];
}

// Deterministic <x, y - z> = sum conj(x_k) (y_k - z_k) in FP64 (z may be
// null): per-CTA partial sums over a fixed grid, then one warp adds them in
// a fixed order.
constexpr int kDotBlocks = 256;
template <typename T>
__global__ void __launch_bounds__(256) k_dot_part(const typename V2<T>::t *x, const typename V2<T>::t *y,
                                                  const typename V2<T>::t *z, size_t n, double *part)
{
    __shared__ double red[8][2];
    double re = 0.0, im = 0.0;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const double xr = x[k].x, xi = x[k].y;
        double yr = y[k].x, yi = y[k].y;
        if (z) {   // y - z, exact in FP64 for FP32 data
            yr -= (double)z[k].x;
            yi -= (double)z[k].y;
        }
        re = fma(xr, yr, fma(xi, yi, re));
        im = fma(xr, yi, fma(-xi, yr, im));
    }
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5][0] = re;
        red[threadIdx.x >> 5][1] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += red[w][0];
            b += red[w][1];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

__global__ void __launch_bounds__(32) k_dot_final(const double *part, int nblk, double2 *out)
{
    double re = 0.0, im = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) {
        re += part[2 * b];
        im += part[2 * b + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (threadIdx.x == 0) *out = make_double2(re, im);
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
    T rs = rsq_(fma(-f[RF_AD], S2, f[RF_R2]));
    c2 K;
    bK<T>(f, rs, S2, C, b, K);
    Loc<T> L = local_coef<T>(rs * rs, f, C, T(0));
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

// ------------------------------------------- literal step, static scratch
// Midpoint scratch of the literal scheme for callers that cannot allocate
// device memory (see teuk_literal_step_static): a fixed array in the
// library's own device image, present on every GPU that loads the library
// until the process exits.  Device code may name it directly; host code
// must obtain its device address with cudaGetSymbolAddress.
constexpr size_t kStaticScratchBytes = (size_t)8 << 20;
static __device__ __align__(256) unsigned char g_literal_scratch[kStaticScratchBytes];

// Same arithmetic as k_literal_mid / k_literal_node, with the step index
// passed in (no control block) and the midpoints in caller-given scratch.
template <typename T>
__global__ void k_literal_mid_static(const StepParams<T> p, typename V2<T>::t *mid, long long n)
{
    typedef typename V2<T>::t c2;
    const int N = p.Nth, Nr = p.Nr;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (Nr - 1) * N) return;
    int i = idx / N, j = idx - i * N;
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
    c2 *mPhi = mid, *mPi = mid + (size_t)(Nr - 1) * N;
    mPhi[idx] = cadd(f0, cscale<c2>(p.half_dt, csub(gbar, cscale<c2>(b, df))));
    mPi[idx] = cadd(gbar, cscale<c2>(p.half_dt, cadd(cscale<c2>(b, dg), S)));
}

template <typename T>
__global__ void k_literal_node_static(const StepParams<T> p, const typename V2<T>::t *mid, long long n)
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
    const c2 *Phi = p.uin, *Pi = p.uin + (size_t)Nr * N;
    const c2 *mPhi = mid, *mPi = mid + (size_t)(Nr - 1) * N;
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

// Raise a kernel's dynamic shared-memory limit to the device maximum, once
// per kernel and device.  Occupancy queries and launches never lower it, so
// a launch within the maximum is valid whatever was queried before it.
static cudaError_t smem_limit_max(const void *fn)
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

template <typename T>
size_t split_smem_bytes(int tile_rows, int Nth)
{
    return split_smem_plan(tile_rows + 2, Nth, (int)sizeof(T)).total;
}

// Two steps per launch: R = TR + 4 rows plus a copy of the extraction row.
template <typename T>
size_t split2_smem_bytes(int tile_rows, int Nth)
{
    return split_smem_plan(tile_rows + 4, Nth, (int)sizeof(T)).total + 2 * (size_t)Nth * sizeof(typename V2<T>::t);
}

int implicit_seg(int Nth) { return Nth <= 128 ? kSegNarrow : (Nth <= 256 ? kSeg : kSegWide); }

int implicit_group(int Nth)
{
    int seg = implicit_seg(Nth);
    int need = (Nth + seg - 1) / seg;
    int G = 1;
    while (G < need) G <<= 1;
    return G;
}

template <typename T>
int split_blocks_per_sm(int Nth, int threads, size_t smem)
{
    const int seg = implicit_seg(Nth);
    auto fn = seg == kSegNarrow ? k_split_step<T, kSegNarrow> : (seg == kSeg ? k_split_step<T, kSeg> : k_split_step<T, kSegWide>);
    if (smem_limit_max((const void *)fn) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

template <typename T>
cudaError_t launch_split_step(const StepParams<T> &p, int threads, size_t smem, cudaStream_t st)
{
    const int seg = implicit_seg(p.Nth);
    const int v = seg == kSegNarrow ? 0 : (seg == kSeg ? 1 : 2);
    auto fn = v == 0 ? k_split_step<T, kSegNarrow> : (v == 1 ? k_split_step<T, kSeg> : k_split_step<T, kSegWide>);
    cudaError_t e = smem_limit_max((const void *)fn);
    if (e != cudaSuccess) return e;
    int grid = (p.Nr + p.tile_rows - 1) / p.tile_rows;
    fn<<<grid, threads, smem, st>>>(p);
    return cudaGetLastError();
}

template <typename T>
bool persist_available(int Nth, int nc)
{
    return sizeof(T) == 4 && implicit_seg(Nth) == kSegNarrow && (nc == 384 || nc == 480);
}

template <typename T>
size_t persist_smem_bytes(int tile_rows, int Nth)
{
    return persist_smem_plan(tile_rows + 2, Nth, (int)sizeof(T)).total;
}

// The persistent kernel for (T, nc), or nullptr.
template <typename T>
static void (*persist_fn(int Nth, int nc))(const StepParams<T>)
{
    if constexpr (sizeof(T) == 4) {
        if (!persist_available<T>(Nth, nc)) return nullptr;
        return nc == 384 ? k_split_persist<T, kSegNarrow, 384> : k_split_persist<T, kSegNarrow, 480>;
    } else {
        return nullptr;
    }
}

template <typename T>
int persist_blocks_per_sm(int Nth, int nc, size_t smem)
{
    auto fn = persist_fn<T>(Nth, nc);
    if (!fn) return 0;
    if (smem_limit_max((const void *)fn) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, nc + 32, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

template <typename T>
void persist_explain(int Nth, int nc, size_t smem, char *buf, size_t len)
{
    auto fn = persist_fn<T>(Nth, nc);
    if (!fn) {
        snprintf(buf, len, "no persistent kernel for this precision, Ntheta and consumer count");
        return;
    }
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, fn);
    if (e != cudaSuccess) {
        cudaGetLastError();
        snprintf(buf, len, "cudaFuncGetAttributes: %s", cudaGetErrorString(e));
        return;
    }
    e = smem_limit_max((const void *)fn);
    cudaGetLastError();
    int nb = -1;
    cudaError_t e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, nc + 32, smem);
    cudaGetLastError();
    snprintf(buf, len,
             "persistent kernel: %d registers/thread, max %d threads/block, %zu B static shared, %zu B local; "
             "needs %d threads and %zu B dynamic shared (set: %s); blocks per SM %d (%s)",
             a.numRegs, a.maxThreadsPerBlock, (size_t)a.sharedSizeBytes, (size_t)a.localSizeBytes, nc + 32, smem,
             cudaGetErrorString(e), nb, cudaGetErrorString(e2));
}

template <typename T>
cudaError_t launch_split_persist(const StepParams<T> &p, int nc, int grid, size_t smem, cudaStream_t st)
{
    auto fn = persist_fn<T>(p.Nth, nc);
    if (!fn || !p.bulk || grid < 1) return cudaErrorInvalidConfiguration;
    cudaError_t e = smem_limit_max((const void *)fn);
    if (e != cudaSuccess) return e;
    fn<<<grid, nc + 32, smem, st>>>(p);
    return cudaGetLastError();
}

template <typename T>
static void (*batch_fn(int seg, int ks))(const StepParams<T> *, const int2 *)
{
    // two steps per launch for segments of up to 8 elements (Ntheta <= 256)
    if (ks == 2) return seg == kSegNarrow ? k_split_batch<T, kSegNarrow, 2> : (seg == kSeg ? k_split_batch<T, kSeg, 2> : nullptr);
    return seg == kSegNarrow ? k_split_batch<T, kSegNarrow, 1>
                             : (seg == kSeg ? k_split_batch<T, kSeg, 1> : k_split_batch<T, kSegWide, 1>);
}

bool split_batch_available(int seg, int ks) { return ks == 1 || (ks == 2 && seg != kSegWide); }

template <typename T>
int split_batch_blocks_per_sm(int seg, size_t smem, int ks)
{
    auto fn = batch_fn<T>(seg, ks);
    if (!fn) return 0;
    if (smem_limit_max((const void *)fn) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 256, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

template <typename T>
cudaError_t launch_split_batch(const StepParams<T> *d_params, const int2 *d_tiles, int ntiles, int seg, size_t smem,
                               int ks, cudaStream_t st)
{
    auto fn = batch_fn<T>(seg, ks);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = smem_limit_max((const void *)fn);
    if (e != cudaSuccess) return e;
    if (ntiles < 1) return cudaSuccess;
    fn<<<ntiles, 256, smem, st>>>(d_params, d_tiles);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply_step(const StepParams<T> &p, int threads, size_t smem, cudaStream_t st)
{
    if (p.nfix < 0) return cudaErrorInvalidValue;
    return launch_split_step<T>(p, threads, smem, st);
}

template <typename T>
cudaError_t launch_sample(const StepParams<T> &p, const typename V2<T>::t *s, int physical, double2 *h_out,
                          cudaStream_t st)
{
    typedef typename V2<T>::t c2;
    const int seg = implicit_seg(p.Nth);
    auto fn = seg == kSegNarrow ? k_sample<T, kSegNarrow> : (seg == kSeg ? k_sample<T, kSeg> : k_sample<T, kSegWide>);
    cudaError_t e = smem_limit_max((const void *)fn);
    if (e != cudaSuccess) return e;
    const size_t row = (size_t)((p.Nth + 1) & ~1);
    const size_t smem = 2 * row * sizeof(c2) + ((size_t)NRF + (size_t)NTF * p.Nth) * sizeof(T);
    fn<<<1, 32, smem, st>>>(p, s, physical, h_out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scan_plans(const StepParams<T> &p, int *plan_full, int *plan_half, cudaStream_t st)
{
    const int seg = implicit_seg(p.Nth);
    auto fn = seg == kSegNarrow ? k_scan_plans<T, kSegNarrow>
                                : (seg == kSeg ? k_scan_plans<T, kSeg> : k_scan_plans<T, kSegWide>);
    const int rows = 256 / p.group;
    fn<<<(p.Nr + rows - 1) / rows, 256, 0, st>>>(p, plan_full, plan_half);
    return cudaGetLastError();
}

template <typename T>
size_t adjoint_smem_bytes(int tile_rows, int Nth)
{
    const size_t R = (size_t)tile_rows + 2;
    return 4 * R * Nth * sizeof(typename V2<T>::t) + ((2 * R - 1) * NRF + (size_t)NTF * Nth) * sizeof(T);
}

template <typename T>
int adjoint_grid(int Nr, int tile_rows)
{
    return (Nr + tile_rows - 1) / tile_rows;
}

template <typename T>
cudaError_t launch_adjoint_step(const StepParams<T> &p, int tile_rows, const double2 *gseed, double *part,
                                double *acc, cudaStream_t st)
{
    const int seg = implicit_seg(p.Nth);
    auto fn = seg == kSegNarrow ? k_adjoint_step<T, kSegNarrow>
                                : (seg == kSeg ? k_adjoint_step<T, kSeg> : k_adjoint_step<T, kSegWide>);
    cudaError_t e = smem_limit_max((const void *)fn);
    if (e != cudaSuccess) return e;
    StepParams<T> q = p;
    q.tile_rows = tile_rows;
    const int grid = adjoint_grid<T>(p.Nr, tile_rows);
    fn<<<grid, 256, adjoint_smem_bytes<T>(tile_rows, p.Nth), st>>>(q, gseed, part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_part_reduce<<<1, 32, 0, st>>>(part, grid, acc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dot(const typename V2<T>::t *x, const typename V2<T>::t *y, const typename V2<T>::t *z,
                       size_t n, double *part, double2 *out, cudaStream_t st)
{
    k_dot_part<T><<<kDotBlocks, 256, 0, st>>>(x, y, z, n, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_dot_final<<<1, 32, 0, st>>>(part, kDotBlocks, out);
    return cudaGetLastError();
}

template <typename T>
static void (*split2_fn(int Nth))(const StepParams<T>)
{
    const int seg = implicit_seg(Nth);
    return seg == kSegNarrow ? k_split_step2<T, kSegNarrow>
                             : (seg == kSeg ? k_split_step2<T, kSeg> : k_split_step2<T, kSegWide>);
}

template <typename T>
int split2_blocks_per_sm(int Nth, int threads, size_t smem)
{
    auto fn = split2_fn<T>(Nth);
    if (smem_limit_max((const void *)fn) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

template <typename T>
cudaError_t launch_split_step2(const StepParams<T> &p, int threads, size_t smem, cudaStream_t st)
{
    if (p.first || p.imp_only) return cudaErrorInvalidValue;   // two full steps only
    auto fn = split2_fn<T>(p.Nth);
    cudaError_t e = smem_limit_max((const void *)fn);
    if (e != cudaSuccess) return e;
    int grid = (p.Nr + p.tile_rows - 1) / p.tile_rows;
    fn<<<grid, threads, smem, st>>>(p);
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

size_t literal_static_scratch_bytes() { return kStaticScratchBytes; }

// Device address of g_literal_scratch, looked up once per device with that
// device current (a host-side symbol is not a device address).
static cudaError_t static_scratch_address(void **out)
{
    static std::mutex mu;
    static void *addr[64] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_literal_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = ptr;
    }
    *out = addr[dev];
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_literal_step_static(const StepParams<T> &p, long long n, cudaStream_t st)
{
    typedef typename V2<T>::t c2;
    void *scratch = nullptr;
    cudaError_t e = static_scratch_address(&scratch);
    if (e != cudaSuccess) return e;
    int nm = (p.Nr - 1) * p.Nth, nn = p.Nr * p.Nth;
    k_literal_mid_static<T><<<(nm + 255) / 256, 256, 0, st>>>(p, (c2 *)scratch, n);
    k_literal_node_static<T><<<(nn + 255) / 256, 256, 0, st>>>(p, (const c2 *)scratch, n);
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

template cudaError_t launch_apply_step<float>(const StepParams<float> &, int, size_t, cudaStream_t);
template cudaError_t launch_apply_step<double>(const StepParams<double> &, int, size_t, cudaStream_t);
template cudaError_t launch_scan_plans<float>(const StepParams<float> &, int *, int *, cudaStream_t);
template cudaError_t launch_scan_plans<double>(const StepParams<double> &, int *, int *, cudaStream_t);
template cudaError_t launch_sample<float>(const StepParams<float> &, const float2 *, int, double2 *, cudaStream_t);
template cudaError_t launch_sample<double>(const StepParams<double> &, const double2 *, int, double2 *, cudaStream_t);
template size_t adjoint_smem_bytes<float>(int, int);
template size_t adjoint_smem_bytes<double>(int, int);
template int adjoint_grid<float>(int, int);
template int adjoint_grid<double>(int, int);
template cudaError_t launch_adjoint_step<float>(const StepParams<float> &, int, const double2 *, double *, double *,
                                                cudaStream_t);
template cudaError_t launch_adjoint_step<double>(const StepParams<double> &, int, const double2 *, double *, double *,
                                                 cudaStream_t);
template cudaError_t launch_dot<float>(const float2 *, const float2 *, const float2 *, size_t, double *, double2 *,
                                       cudaStream_t);
template cudaError_t launch_dot<double>(const double2 *, const double2 *, const double2 *, size_t, double *,
                                        double2 *, cudaStream_t);
template int split_batch_blocks_per_sm<float>(int, size_t, int);
template int split_batch_blocks_per_sm<double>(int, size_t, int);
template cudaError_t launch_split_batch<float>(const StepParams<float> *, const int2 *, int, int, size_t, int,
                                               cudaStream_t);
template cudaError_t launch_split_batch<double>(const StepParams<double> *, const int2 *, int, int, size_t, int,
                                                cudaStream_t);
template bool persist_available<float>(int, int);
template bool persist_available<double>(int, int);
template size_t persist_smem_bytes<float>(int, int);
template size_t persist_smem_bytes<double>(int, int);
template void persist_explain<float>(int, int, size_t, char *, size_t);
template void persist_explain<double>(int, int, size_t, char *, size_t);
template int persist_blocks_per_sm<float>(int, int, size_t);
template int persist_blocks_per_sm<double>(int, int, size_t);
template cudaError_t launch_split_persist<float>(const StepParams<float> &, int, int, size_t, cudaStream_t);
template cudaError_t launch_split_persist<double>(const StepParams<double> &, int, int, size_t, cudaStream_t);
template size_t split2_smem_bytes<float>(int, int);
template size_t split2_smem_bytes<double>(int, int);
template int split2_blocks_per_sm<float>(int, int, size_t);
template int split2_blocks_per_sm<double>(int, int, size_t);
template cudaError_t launch_split_step2<float>(const StepParams<float> &, int, size_t, cudaStream_t);
template cudaError_t launch_split_step2<double>(const StepParams<double> &, int, size_t, cudaStream_t);
template int split_blocks_per_sm<float>(int, int, size_t);
template int split_blocks_per_sm<double>(int, int, size_t);
template size_t split_smem_bytes<float>(int, int);
template size_t split_smem_bytes<double>(int, int);
template cudaError_t launch_split_step<float>(const StepParams<float> &, int, size_t, cudaStream_t);
template cudaError_t launch_split_step<double>(const StepParams<double> &, int, size_t, cudaStream_t);
template cudaError_t launch_literal_step_static<float>(const StepParams<float> &, long long, cudaStream_t);
template cudaError_t launch_literal_step_static<double>(const StepParams<double> &, long long, cudaStream_t);
template cudaError_t launch_literal_step<float>(const StepParams<float> &, cudaStream_t);
template cudaError_t launch_literal_step<double>(const StepParams<double> &, cudaStream_t);
template cudaError_t launch_extract<float>(const StepParams<float> &, const float2 *, long long, cudaStream_t);
template cudaError_t launch_extract<double>(const StepParams<double> &, const double2 *, long long, cudaStream_t);

}  // namespace teuk
