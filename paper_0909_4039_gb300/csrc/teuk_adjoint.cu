// teuk_adjoint.cu -- the step's waveform sample as an operator, the Hermitian
// adjoint of one split-scheme step with the source-parameter derivatives,
// and deterministic FP64 inner products (gradients of waveform losses).
#include "teuk_dev.cuh"

namespace teuk {
namespace {

// Tile of CTA b among nt: the tile holding the extraction row goes first.
// Its CTA also runs the sample's adjoint on that row (FP64 solves of one row
// by one warp), which then overlaps the other tiles instead of trailing the
// last wave (FP64 adjoint step with the spin term on 4096 x 64: the SMs were
// busy 70 % of the launch before).
__device__ __forceinline__ int tile_of_block(int b, int nt, int i_ext, int tile_rows)
{
    int e = i_ext / tile_rows;
    e = e < nt ? e : nt - 1;
    b += e;
    return b < nt ? b : b - nt;
}

// h = E u with u = s (physical) or u = C_{dt/2} s on the extraction row; one
// warp.  The sum is the one the step kernels write to the waveform buffer.
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
    T *xTh = xF + NSF;
    for (int j = tid; j < N; j += 32) {
        xPhi[j] = s[(size_t)i * N + j];
        xPi[j] = s[((size_t)Nr + i) * N + j];
    }
    if (tid < NSF) xF[tid] = p.stab[(size_t)(2 * i) * NSF + tid];
    for (int k = tid; k < NTF * N; k += 32) xTh[k] = p.thtab[k];
    __syncwarp();
    if (!physical) {
        const int G = p.group;
        const bool mine = tid < G;
        const bool active = mine && i >= 1 && i <= Nr - 2;
        implicit_row_fwd<T, S>(p.half, xPhi, xPi, p.half.piv + (size_t)i * N, xF, xTh, N, active, mine, tid % G, G,
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
// part[4 tile + (0..3)] = (Re cA, Im cA, Re cr, Im cr); the extraction
// row's tile runs first (see tile_of_block).
template <typename T, int S>
__global__ void __launch_bounds__(256, 1) k_adjoint_step(const StepParams<T> p, const double2 *gseed, double *part)
{
    typedef typename V2<T>::t c2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double s_red[8][4];
    const int Nr = p.Nr, N = p.Nth, TR = p.tile_rows, R = TR + 2, P = N;
    const int tid = threadIdx.x, NT = blockDim.x;
    const int tile = tile_of_block((int)blockIdx.x, (int)gridDim.x, p.i_ext, TR);
    const int i0 = tile * TR;
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
        part[4 * tile + tid] = acc;
    }
}

// ---------------------------------------------------- the spin derivative
//
// dL/da = sum_n Re <lam_{n+1}, (d M_n/d a) s_n> + Re <g_n, d(E C_{dt/2})/d a s_n>
// by contraction with the forward stage values, inside the adjoint step
// (no extra step applications).  With A = I - gh J, J u = (Pi, -W Phi - c_t Pi)
// and c = (1 - gamma) h, the implicit step is C_h = A^{-1}(I + c J A^{-1}):
// U1 = A^{-1} u, U2 = C_h u.  For an adjoint mu of its output,
//   <mu, dC_h u> = gh <nu2, dJ U2> + c <nu2, dJ U1> + gh <nu1, dJ U1>,
//   nu2 = A^{-H} mu,  nu1 = A^{-H}(c J^H nu2),  C_h^H mu = nu2 + nu1,
// dJ x = (0, -(dW x_Phi + dc_t x_Pi)).  A^{-H} is solved Pi-first,
// M^H nu_Pi = b_Pi + gh b_Phi, nu_Phi = b_Phi - gh W^H nu_Pi, with the LU
// of M = (1 + gh c_t) + gh^2 W.  The Lax-Wendroff stages contribute
// <adjoint of each stage output, d(stage)/da> with the stage inputs of the
// forward step; the coefficient derivatives come from the step table's
// spin derivative (dstab, exact forward-mode derivatives of the FP64
// table generator, r(r*; a) by implicit differentiation of Eq. 2).

// The source term of a stage, S = F ph (ph: the scaled phase), as the
// forward step forms it, and dS/da: F = SRC sg (SR2 GTH + GA2) through its
// factors and 1/Sigma^2, the phase through Omega(a) (mdt = m t dOmega/da).
template <typename T>
__device__ __forceinline__ void src_da(const T *f, const T *df, T sg, T dsg, T gth, T ga2, T dga2,
                                       typename V2<T>::t ph, T mdt, typename V2<T>::t &Sv, typename V2<T>::t &dS)
{
    typedef typename V2<T>::t c2;
    const T X = fma(f[SF_SR2], gth, ga2), dX = fma(df[SF_SR2], gth, dga2);
    const c2 src = cmk<c2>(f[SF_SRE], f[SF_SIM]), dsrc = cmk<c2>(df[SF_SRE], df[SF_SIM]);
    const c2 F = cscale<c2>(sg * X, src);
    const c2 dF = cadd(cscale<c2>(sg * X, dsrc), cscale<c2>(fma(dsg, X, sg * dX), src));
    Sv = cmul(F, ph);
    // d/da e^{-i m Omega t} = -i m t (dOmega/da) e^{-i m Omega t}
    dS = cadd(cmul(dF, ph), cmk<c2>(Sv.y * mdt, -Sv.x * mdt));
}

// Loads the lane's segment of a row (zero past its end).
template <typename T, int S>
__device__ __forceinline__ void seg_load(const typename V2<T>::t *row, int j0, int len, bool vec,
                                         typename V2<T>::t (&v)[S])
{
    typedef typename V2<T>::t c2;
    if (vec && len == S) {
        vload<S>(v, row + j0);
    } else {
#pragma unroll
        for (int k = 0; k < S; ++k) v[k] = k < len ? row[j0 + k] : cmk<c2>(T(0), T(0));
    }
}

// C_h^H on one row in the block form above (lf, lg: mu on entry, C_h^H mu on
// exit), and this lane's part of <mu, dC_h u> from the forward stage values
// (u1f, u1g) = U1 and (u2f, u2g) = U2 of the same row; f, df: the row's
// step-table entry and its spin derivative.
template <typename T, int S, bool MAT = false, bool SPIN = true>
__device__ double implicit_row_adj_spin(const ImpConst<T> &K, typename V2<T>::t *lf, typename V2<T>::t *lg,
                                        const typename V2<T>::t *u1f, const typename V2<T>::t *u1g,
                                        const typename V2<T>::t *u2f, const typename V2<T>::t *u2g,
                                        const typename V2<T>::t *prow, const T *f, const T *df, const T *th, int N,
                                        bool active, bool in_tile, int g, int G, bool vec,
                                        const AdjPlanes<T> *A = nullptr, int gi = 0)
{
    typedef typename V2<T>::t c2;
    const c2 zero = cmk<c2>(T(0), T(0));
    const int j0 = g * S;
    int len = N - j0;
    len = len < 0 ? 0 : (len > S ? S : len);
    const int lenw = len;
    if (!active) len = 0;
    const T gh = K.gh, c = K.h1g;
    ImpCoef<T, S> C;
    c2 w[S], y[S];   // mu_Phi, mu_Pi
    if constexpr (MAT)
        imp_load_mat<T, S>(A->m, lf, lg, prow, gi, N, len, j0, vec, C, w, y);
    else
        imp_load<T, S>(K, lf, lg, prow, f, th, N, len, j0, vec, C, w, y);
    // multipliers of M^H = U^H L^H and the rows of W^H (qap_{j-1}, conj(dg_j), qam_{j+1})
    c2 fm[S], pm[S], bm[S];
    T qapp[S], qamn[S];
    {
        const c2 fk_prev = shfl_up_c(C.fk[S - 1], 1, G);
        const T sub_next = __shfl_down_sync(0xffffffffu, C.sub[0], 1, G);
        T qap_prev = __shfl_up_sync(0xffffffffu, C.qap[S - 1], 1, G);
        T qam_next = __shfl_down_sync(0xffffffffu, C.qam[0], 1, G);
        if (g == 0) qap_prev = T(0);
        if (g == G - 1) qam_next = T(0);
#pragma unroll
        for (int k = 0; k < S; ++k) {
            const c2 fkp = k ? C.fk[k - 1] : fk_prev;
            const T subn = (k + 1 < S) ? C.sub[(k + 1) < S ? k + 1 : S - 1] : sub_next;
            fm[k] = (g == 0 && k == 0) ? zero : conj_c(fkp);
            pm[k] = conj_c(C.e[k]);
            bm[k] = (g == G - 1 && k == S - 1) ? zero : cscale<c2>(subn, conj_c(C.e[k]));
            qapp[k] = k ? C.qap[k - 1] : qap_prev;
            qamn[k] = (k + 1 < S) ? C.qam[(k + 1) < S ? k + 1 : S - 1] : qam_next;
        }
    }
    const ScanPlan<T> P = scan_plan<T, S>(fm, bm, g, G);
    auto apply_WH = [&](const c2 (&v)[S], c2 (&out)[S]) {
        c2 vl = shfl_up_c(v[S - 1], 1, G), vr = shfl_down_c(v[0], 1, G);
        if (g == 0) vl = zero;
        if (g == G - 1) vr = zero;
#pragma unroll
        for (int k = 0; k < S; ++k) {
            const c2 vm = k ? v[k - 1] : vl;
            const c2 vp = (k + 1 < S) ? v[(k + 1) < S ? k + 1 : S - 1] : vr;
            out[k] = cfma(conj_c(C.dg[k]), v[k], caxpy(qamn[k], vp, cscale<c2>(qapp[k], vm)));
        }
    };
    // nu2 = A^{-H} mu
    c2 n2p[S], n2f[S], Y[S];
#pragma unroll
    for (int k = 0; k < S; ++k) n2p[k] = caxpy(gh, w[k], y[k]);
    seg_solve<T, S>(n2p, fm, pm, bm, P, g, G);
    apply_WH(n2p, Y);
#pragma unroll
    for (int k = 0; k < S; ++k) n2f[k] = caxpy(-gh, Y[k], w[k]);
    // xi = c J^H nu2 = c (-W^H nu2_Pi, nu2_Phi - conj(c_t) nu2_Pi); nu1 = A^{-H} xi
    c2 xf[S], n1p[S];
#pragma unroll
    for (int k = 0; k < S; ++k) {
        xf[k] = cscale<c2>(-c, Y[k]);
        const c2 xp = cfnma(conj_c(C.ct[k]), n2p[k], cscale<c2>(c, n2f[k]));   // ct holds c c_t
        n1p[k] = caxpy(gh, xf[k], xp);
    }
    seg_solve<T, S>(n1p, fm, pm, bm, P, g, G);
    apply_WH(n1p, Y);
    // C_h^H mu = nu2 + nu1
#pragma unroll
    for (int k = 0; k < S; ++k) {
        w[k] = cadd(n2f[k], caxpy(-gh, Y[k], xf[k]));
        y[k] = cadd(n2p[k], n1p[k]);
    }
    if constexpr (!SPIN) {
        if (in_tile) row_store<T, S>(lf, lg, w, y, j0, lenw, vec);
        return 0.0;
    }
    // derivative coefficients dW (dqam, ddg, dqap) and dc_t of the row
    c2 ddg[S], dct[S];
    T dqam[S], dqap[S];
    if constexpr (MAT) {
#pragma unroll
        for (int k = 0; k < S; ++k) {
            T v[8];
            if (k < len) {
                vload<8>(v, A->dimp + ((size_t)gi * N + j0 + k) * 8);
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = T(0);
            }
            ddg[k] = cmk<c2>(v[0], v[1]);
            dct[k] = cmk<c2>(v[2], v[3]);
            dqam[k] = v[4];
            dqap[k] = v[5];
        }
    } else {
        const ImpRow<T> r = imp_row(K, f);
        T fr[8], dfr[8];
        vload<8>(fr, f);
        vload<8>(dfr, df);
#pragma unroll
        for (int k = 0; k < S; ++k) {
            if (k < len) {
                const int j = j0 + k;
                imp_da<T>(r, fr, dfr, th[TF_S2 * N + j], th[TF_C * N + j], th[TF_AM * N + j], th[TF_A0 * N + j],
                          th[TF_AP * N + j], ddg[k], dct[k], dqam[k], dqap[k]);
            } else {
                dqam[k] = dqap[k] = T(0);
                ddg[k] = dct[k] = zero;
            }
        }
    }
    // Q = dW x_Phi + dc_t x_Pi for the stage values
    auto apply_dQ = [&](const c2 (&xf_)[S], const c2 (&xp_)[S], c2 (&out)[S]) {
        c2 vl = shfl_up_c(xf_[S - 1], 1, G), vr = shfl_down_c(xf_[0], 1, G);
        if (g == 0) vl = zero;
        if (g == G - 1) vr = zero;
#pragma unroll
        for (int k = 0; k < S; ++k) {
            const c2 vm = k ? xf_[k - 1] : vl;
            const c2 vp = (k + 1 < S) ? xf_[(k + 1) < S ? k + 1 : S - 1] : vr;
            out[k] = cfma(dct[k], xp_[k], cfma(ddg[k], xf_[k], caxpy(dqap[k], vp, cscale<c2>(dqam[k], vm))));
        }
    };
    double acc = 0.0;
    {
        c2 a[S], b[S], Q1[S], Q2[S];
        seg_load<T, S>(u1f, j0, len, vec, a);
        seg_load<T, S>(u1g, j0, len, vec, b);
        apply_dQ(a, b, Q1);
        seg_load<T, S>(u2f, j0, len, vec, a);
        seg_load<T, S>(u2g, j0, len, vec, b);
        apply_dQ(a, b, Q2);
#pragma unroll
        for (int k = 0; k < S; ++k) {
            // gh <nu2, dJ U2> + c <nu2, dJ U1> + gh <nu1, dJ U1>, <nu, dJ x> = -Re conj(nu_Pi) Q
            const c2 z2 = caxpy(c, Q1[k], cscale<c2>(gh, Q2[k]));
            const c2 z1 = cscale<c2>(gh, Q1[k]);
            acc -= (double)n2p[k].x * (double)z2.x + (double)n2p[k].y * (double)z2.y;
            acc -= (double)n1p[k].x * (double)z1.x + (double)n1p[k].y * (double)z1.y;
        }
    }
    if (in_tile) row_store<T, S>(lf, lg, w, y, j0, lenw, vec);
    return acc;
}

// Adjoint step with the spin derivative: lam_n as k_adjoint_step (here
// through the block form of C_h^H), the source derivatives (amplitude and
// r0) as k_adjoint_step, and the step's part of dL/da.  p.uin = lam_{n+1},
// p.uout = lam_n, sin = s_n (the step's input state), p.nfix = n.  Per CTA:
// part[NPART b + (0 .. 4)] = (Re cA, Im cA, Re cr, Im cr, spin term).
// Tile rows i0-1 .. i0+TR: lam_{n+1} (lF, lG), the stage values U2 = C_h s_n
// (vF, vG) and U1 (u1F, u1G), the midpoint adjoints (mF, mG).
constexpr int kNPart = 6;

template <typename T, int S, bool MAT, bool SPIN>
__global__ void __launch_bounds__(256, 1) k_adjoint_spin(const StepParams<T> p, const typename V2<T>::t *sin,
                                                         const typename V2<T>::t *tape, const double2 *gseed,
                                                         const AdjPlanes<T> A, double *part)
{
    typedef typename V2<T>::t c2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double s_red[8][kNPart];
    const int Nr = p.Nr, N = p.Nth, TR = p.tile_rows, R = TR + 2, P = N;
    const int tid = threadIdx.x, NT = blockDim.x;
    const int tile = tile_of_block((int)blockIdx.x, (int)gridDim.x, p.i_ext, TR);
    const int i0 = tile * TR;
    const int G = p.group;
    const bool first = p.first != 0;
    const ImpConst<T> &K = first ? p.half : p.full;
    const long long n = p.nfix;
    const c2 zero = cmk<c2>(T(0), T(0));
    const T dtT = p.dt, hdtT = p.half_dt;
    const bool vec = p.vec != 0;
    const int g = tid % G;

    const unsigned plane = (unsigned)R * (unsigned)N;
    c2 *lF = (c2 *)smem_raw;
    c2 *lG = lF + plane;
    c2 *mF = lG + plane;
    c2 *mG = mF + plane;
    c2 *vF = mG + plane;
    c2 *vG = vF + plane;
    c2 *u1F = vG + plane;
    c2 *u1G = u1F + plane;
    c2 *fmF = u1G + plane;   // forward midpoints (Lax-Wendroff stage 1 of U2)
    c2 *fmG = fmF + plane;
    T *sSt = (T *)(fmG + plane);
    T *sDSt = sSt + (2 * R - 1) * NSF;
    T *sTh = sDSt + (2 * R - 1) * NSF;

    // ---- lam_{n+1} and s_n (with a tape: the forward stage values U2 and U1
    // the forward step recorded) on rows i0-1 .. i0+TR, the step tables,
    // theta tables
    const c2 *tp1 = tape, *tp2 = tape ? tape + tape_u2_off(Nr, N) : nullptr;
    for (int idx = tid; idx < R * N; idx += NT) {
        const int lr = idx / N, j = idx - lr * N;
        const int gi = i0 - 1 + lr;
        c2 a = zero, b = zero, sa = zero, sb = zero, ua = zero, ub = zero;
        if (gi >= 0 && gi < Nr) {
            const size_t qf = (size_t)gi * N + j, qg = ((size_t)Nr + gi) * N + j;
            a = p.uin[qf];
            b = p.uin[qg];
            if (!SPIN) {
            } else if (tape) {
                sa = tp2[qf];
                sb = tp2[qg];
                ua = tp1[qf];
                ub = tp1[qg];
            } else {
                sa = sin[qf];
                sb = sin[qg];
            }
        }
        lF[idx] = a;
        lG[idx] = b;
        vF[idx] = sa;
        vG[idx] = sb;
        if (tape) {
            u1F[idx] = ua;
            u1G[idx] = ub;
        }
    }
    {
        const long long pbase = 2LL * (i0 - 1), pmax = 2LL * Nr - 2;
        for (int idx = tid; idx < (2 * R - 1) * NSF; idx += NT) {
            const int e = idx / NSF, q = idx - e * NSF;
            const long long pos = pbase + e;
            const bool on = pos >= 0 && pos <= pmax;
            sSt[idx] = on ? p.stab[(size_t)pos * NSF + q] : T(0);
            sDSt[idx] = on ? p.dstab[(size_t)pos * NSF + q] : T(0);
        }
    }
    for (int idx = tid; idx < NTF * N; idx += NT) sTh[idx] = p.thtab[idx];
    __syncthreads();

    // ---- forward implicit stage on all rows: (vF, vG) <- U2 = C_h s_n, (u1F, u1G) <- U1
    if (SPIN && !tape) {
        const int rpp = NT / G;
        for (int base = 0; base < R; base += rpp) {
            const int lr = base + tid / G;
            const bool in_tile = lr < R;
            const int gi = i0 - 1 + lr;
            const bool active = in_tile && gi >= 1 && gi <= Nr - 2;
            const int lrc = in_tile ? lr : 0;
            implicit_row_fwd<T, S, MAT>(K, vF + lrc * P, vG + lrc * P, K.piv + (size_t)(active ? gi : 1) * N,
                                        sSt + 2 * lrc * NSF, sTh, N, active, in_tile, g, G, vec,
                                        active ? K.plan[gi] : 0, &A.m, active ? gi : 1, u1F + lrc * P,
                                        u1G + lrc * P);
        }
    }
    __syncthreads();

    const bool src = p.patch_np > 0 && i0 + TR >= p.patch_p0 && i0 - 1 <= p.patch_p0 + p.patch_np;
    const bool srcu = p.unit_np > 0 && i0 + TR >= p.unit_p0 && i0 - 1 <= p.unit_p0 + p.unit_np;
    const double t1 = (double)n * p.dt64, t2 = t1 + 0.5 * p.dt64;
    double2 ph1 = make_double2(0.0, 0.0), ph2 = ph1;
    if (src || srcu) {
        ph1 = phase_at(p.mOmega, t1);
        ph2 = phase_at(p.mOmega, t2);
    }
    // scaled phases of the forward stages (dt/2 and dt), as the step kernels form them
    const c2 sph1 = from_d2<T>(make_double2(0.5 * p.dt64 * ph1.x, 0.5 * p.dt64 * ph1.y));
    const c2 sph2 = from_d2<T>(make_double2(p.dt64 * ph2.x, p.dt64 * ph2.y));
    const T mdt1 = (T)(p.m_dOmega_da * t1), mdt2 = (T)(p.m_dOmega_da * t2);
    double2 cA = make_double2(0.0, 0.0), cr = cA;
    double spin = 0.0;

    // beta, kap, 1/Sigma^2 and their spin derivatives at tile position e
    // (2 lr: node, 2 k + 1: half node) and theta j
    auto lwc = [&](int e, int j, T S2, T Cc) -> LwDa<T> {
        if constexpr (MAT) {
            const size_t o = ((size_t)(2 * (i0 - 1) + e) * N + j) * 4;
            T v[4], dv[4];
            vload<4>(v, A.m.lw + o);
            vload<4>(dv, A.dlw + o);
            LwDa<T> r;
            r.beta = v[0];
            r.kap = cmk<c2>(v[1], v[2]);
            r.sg = v[3];
            r.dbeta = dv[0];
            r.dkap = cmk<c2>(dv[1], dv[2]);
            r.dsg = dv[3];
            return r;
        } else {
            return lw_coef_da<T>(sSt + e * NSF, sDSt + e * NSF, S2, Cc);
        }
    };

    // ---- adjoints of the midpoints k = 0 .. R-2, and their spin terms
    for (int idx = tid; idx < (R - 1) * N; idx += NT) {
        const int k = idx / N, j = idx - k * N;
        const int gl = i0 - 1 + k;
        const T S2 = sTh[TF_S2 * N + j], Cc = sTh[TF_C * N + j];
        c2 wF = zero, wG = zero;
        if (gl >= 0 && gl <= Nr - 2) {
            if (gl >= 1) {   // lower node interior
                const LwDa<T> nd = lwc(2 * k, j, S2, Cc);
                const c2 lf = lF[k * P + j], lg = lG[k * P + j];
                wF = csub(cmul(conj_c(nd.kap), lg), cscale<c2>(nd.beta, lf));
                wG = cscale<c2>(nd.beta, lg);
            }
            if (gl + 1 <= Nr - 2) {   // upper node interior
                const LwDa<T> nd = lwc(2 * (k + 1), j, S2, Cc);
                const c2 lf = lF[(k + 1) * P + j], lg = lG[(k + 1) * P + j];
                wF = cadd(wF, csub(cscale<c2>(nd.beta, lf), cmul(conj_c(nd.kap), lg)));
                wG = csub(wG, cscale<c2>(nd.beta, lg));
            }
            // the source derivatives of this midpoint (owned by the tile of its lower node)
            if (srcu && k >= 1 && k <= TR) {
                const int pr = gl - p.unit_p0;
                if (pr >= 0 && pr < p.unit_np)
                    source_grad<T>(p, wG, (double)hdtT, p.patchu[((size_t)pr * 2 + 1) * N + j], ph1,
                                   p.rs_min64 + ((double)gl + 0.5) * p.drs64, t1, cA, cr);
            }
            if constexpr (SPIN) {
                // the forward midpoint from U2, as the step forms it (stored for
                // the node stage's spin terms), and this midpoint's spin term
                const LwDa<T> h = lwc(2 * k + 1, j, S2, Cc);
                const c2 fa = vF[k * P + j], fb = vF[(k + 1) * P + j], ga = vG[k * P + j], gb = vG[(k + 1) * P + j];
                const c2 Df = csub(fb, fa), Dg = csub(gb, ga);
                c2 Sv = zero, dS = zero;
                if (src && gl >= p.patch_p0 && gl < p.patch_p0 + p.patch_np)
                    src_da<T>(sSt + (2 * k + 1) * NSF, sDSt + (2 * k + 1) * NSF, h.sg, h.dsg, sTh[TF_GTH * N + j],
                              sTh[TF_GA2 * N + j], sTh[TF_DGA2 * N + j], sph1, mdt1, Sv, dS);
                fmF[idx] = caxpy(-h.beta, Df, cscale<c2>(T(0.5), cadd(fa, fb)));
                fmG[idx] = cfma(h.kap, Df, cadd(caxpy(h.beta, Dg, cscale<c2>(T(0.5), cadd(ga, gb))), Sv));
                if (k >= 1 && k <= TR) {
                    // d(Phi*) = -dbeta Df,  d(Pi*) = dbeta Dg + dkap Df + dS
                    const c2 dmf = cscale<c2>(-h.dbeta, Df);
                    const c2 dmg = cadd(cfma(h.dkap, Df, cscale<c2>(h.dbeta, Dg)), dS);
                    spin += (double)wF.x * (double)dmf.x + (double)wF.y * (double)dmf.y +
                            (double)wG.x * (double)dmg.x + (double)wG.y * (double)dmg.y;
                }
            }
        }
        mF[idx] = wF;
        mG[idx] = wG;
    }
    __syncthreads();

    // ---- adjoints of the nodes (the Lax-Wendroff inputs), rows 1..TR, and their spin terms
    for (int idx = tid; idx < TR * N; idx += NT) {
        const int lr = 1 + idx / N, j = idx - (lr - 1) * N;
        const int gi = i0 - 1 + lr;
        if (gi >= Nr) continue;
        const T S2 = sTh[TF_S2 * N + j], Cc = sTh[TF_C * N + j];
        const c2 lf = lF[lr * P + j], lg = lG[lr * P + j];
        const bool interior = gi >= 1 && gi <= Nr - 2;
        c2 wF = interior ? lf : zero, wG = interior ? lg : zero;
        LwDa<T> hu, hd;
        if (gi <= Nr - 2) {   // midpoint lr (to the next row)
            hu = lwc(2 * lr + 1, j, S2, Cc);
            const c2 mf = mF[lr * P + j], mg = mG[lr * P + j];
            wF = cadd(wF, csub(cscale<c2>(T(0.5) + hu.beta, mf), cmul(conj_c(hu.kap), mg)));
            wG = cadd(wG, cscale<c2>(T(0.5) - hu.beta, mg));
        }
        if (gi >= 1) {   // midpoint lr - 1 (to the previous row)
            hd = lwc(2 * lr - 1, j, S2, Cc);
            const c2 mf = mF[(lr - 1) * P + j], mg = mG[(lr - 1) * P + j];
            wF = cadd(wF, cadd(cscale<c2>(T(0.5) - hd.beta, mf), cmul(conj_c(hd.kap), mg)));
            wG = cadd(wG, cscale<c2>(T(0.5) + hd.beta, mg));
        }
        if (interior) {
            if (srcu) {
                const int pr = gi - p.unit_p0;
                if (pr >= 0 && pr < p.unit_np)
                    source_grad<T>(p, lg, (double)dtT, p.patchu[((size_t)pr * 2) * N + j], ph2,
                                   p.rs_min64 + (double)gi * p.drs64, t2, cA, cr);
            }
            if constexpr (SPIN) {
            // spin terms of the node stage: d(Phi') = -dbeta dMf,
            // d(Pi') = dbeta dMg + dkap dMf + dS, dM the forward midpoint difference
            const LwDa<T> nd = lwc(2 * lr, j, S2, Cc);
            const c2 dMf = csub(fmF[lr * P + j], fmF[(lr - 1) * P + j]);
            const c2 dMg = csub(fmG[lr * P + j], fmG[(lr - 1) * P + j]);
            const c2 dnf = cscale<c2>(-nd.dbeta, dMf);
            c2 dng = cfma(nd.dkap, dMf, cscale<c2>(nd.dbeta, dMg));
            if (src && gi >= p.patch_p0 && gi < p.patch_p0 + p.patch_np) {
                c2 Sv, dS;
                src_da<T>(sSt + 2 * lr * NSF, sDSt + 2 * lr * NSF, nd.sg, nd.dsg, sTh[TF_GTH * N + j],
                          sTh[TF_GA2 * N + j], sTh[TF_DGA2 * N + j], sph2, mdt2, Sv, dS);
                dng = cadd(dng, dS);
            }
            spin += (double)lf.x * (double)dnf.x + (double)lf.y * (double)dnf.y + (double)lg.x * (double)dng.x +
                    (double)lg.y * (double)dng.y;
            }
        }
        lF[lr * P + j] = wF;
        lG[lr * P + j] = wG;
    }
    __syncthreads();

    // ---- C_h^H on the output rows with the implicit stage's spin terms
    {
        const int rpp = NT / G;
        for (int base = 1; base <= TR; base += rpp) {
            const int lr = base + tid / G;
            const bool in_tile = lr <= TR && i0 - 1 + lr < Nr;
            const int gi = i0 - 1 + lr;
            const bool active = in_tile && gi >= 1 && gi <= Nr - 2;
            const int lrc = in_tile ? lr : 1;
            const double d = implicit_row_adj_spin<T, S, MAT, SPIN>(
                K, lF + lrc * P, lG + lrc * P, u1F + lrc * P, u1G + lrc * P, vF + lrc * P, vG + lrc * P,
                K.piv + (size_t)(active ? gi : 1) * N, sSt + 2 * lrc * NSF, sDSt + 2 * lrc * NSF, sTh, N, active,
                in_tile, g, G, vec, &A, active ? gi : 1);
            if (active) spin += d;
        }
    }
    __syncthreads();

    // ---- extraction seed C_{dt/2}^H E^H g_n (E^H g_0 for a physical input), and
    // the sample's spin term <E^H g_n, dC_{dt/2} s_n>
    const bool ext = gseed != nullptr && p.i_ext >= i0 && p.i_ext < i0 + TR && p.i_ext < Nr;
    if (ext) {
        const int lx = p.i_ext - i0 + 1;
        // row buffers: mF/mG rows 0, 1 (the midpoint adjoints are no longer needed)
        c2 *xF = mF, *xG = mG, *sF = mF + N, *sG = mG + N, *aF = mF + 2 * N, *aG = mG + 2 * N;
        if (tid < 32) {
            const double2 gv = *gseed;
            for (int j = tid; j < N; j += 32) {
                const double w = p.w[j];
                xF[j] = cmk<c2>((T)(w * gv.x), (T)(w * gv.y));
                xG[j] = zero;
                if (!SPIN) {
                } else if (tape) {
                    sF[j] = tape[tape_x_off(Nr, N) + j];
                    sG[j] = tape[tape_x_off(Nr, N) + N + j];
                } else {
                    sF[j] = sin[(size_t)p.i_ext * N + j];
                    sG[j] = sin[((size_t)Nr + p.i_ext) * N + j];
                }
            }
            __syncwarp();
            if (!first) {
                const bool mine = tid < G;
                const bool active = mine && p.i_ext >= 1 && p.i_ext <= Nr - 2;
                // forward C_{dt/2} on the row of s_n: (sF, sG) <- U2, (aF, aG) <- U1
                if constexpr (SPIN)
                    implicit_row_fwd<T, S>(p.half, sF, sG, p.half.piv + (size_t)p.i_ext * N, sSt + 2 * lx * NSF, sTh,
                                           N, active, mine, tid % G, G, vec, active ? p.half.plan[p.i_ext] : 0,
                                           nullptr, 0, aF, aG);
                __syncwarp();
                const double d = implicit_row_adj_spin<T, S, false, SPIN>(p.half, xF, xG, aF, aG, sF, sG,
                                                             p.half.piv + (size_t)p.i_ext * N, sSt + 2 * lx * NSF,
                                                             sDSt + 2 * lx * NSF, sTh, N, active, mine, tid % G, G,
                                                             vec);
                if (active) spin += d;
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
        const int lr = 1 + idx / N, j = idx - (lr - 1) * N;
        const int gi = i0 - 1 + lr;
        if (gi >= Nr) continue;
        p.uout[(size_t)gi * N + j] = lF[lr * P + j];
        p.uout[((size_t)Nr + gi) * N + j] = lG[lr * P + j];
    }

    // ---- this CTA's sums (fixed-order reduction)
    double v[kNPart] = {cA.x, cA.y, cr.x, cr.y, spin, 0.0};
#pragma unroll
    for (int c = 0; c < kNPart; ++c)
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
    if ((tid & 31) == 0)
        for (int c = 0; c < kNPart; ++c) s_red[tid >> 5][c] = v[c];
    __syncthreads();
    if (tid < kNPart) {
        double acc = 0.0;
        for (int w = 0; w < NT / 32; ++w) acc += s_red[w][tid];
        part[kNPart * tile + tid] = acc;
    }
}

// acc[c] += sum over the nblk CTAs of part[kNPart b + c], c < kNPart, in a fixed order.
__global__ void __launch_bounds__(32) k_part_reduce6(const double *part, int nblk, double *acc)
{
    const int lane = threadIdx.x;
    double v[kNPart] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = lane; b < nblk; b += 32)
        for (int c = 0; c < kNPart; ++c) v[c] += part[kNPart * b + c];
    for (int c = 0; c < kNPart; ++c)
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
    if (lane == 0)
        for (int c = 0; c < kNPart; ++c) acc[c] += v[c];
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

}  // namespace

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
    const size_t smem = 2 * row * sizeof(c2) + ((size_t)NSF + (size_t)NTF * p.Nth) * sizeof(T);
    fn<<<1, 32, smem, st>>>(p, s, physical, h_out);
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
size_t adjoint_spin_smem_bytes(int tile_rows, int Nth)
{
    const size_t R = (size_t)tile_rows + 2;
    return 10 * R * Nth * sizeof(typename V2<T>::t) + (2 * (2 * R - 1) * NSF + (size_t)NTF * Nth) * sizeof(T);
}

template <typename T, bool MAT, bool SPIN = true>
static void (*adjoint_spin_fn(int Nth))(const StepParams<T>, const typename V2<T>::t *, const typename V2<T>::t *,
                                        const double2 *, const AdjPlanes<T>, double *)
{
    const int seg = implicit_seg(Nth);
    return seg == kSegNarrow ? k_adjoint_spin<T, kSegNarrow, MAT, SPIN>
                             : (seg == kSeg ? k_adjoint_spin<T, kSeg, MAT, SPIN> : k_adjoint_spin<T, kSegWide, MAT, SPIN>);
}

template <typename T>
cudaError_t launch_adjoint_spin(const StepParams<T> &p, int tile_rows, const typename V2<T>::t *sin,
                                const typename V2<T>::t *tape, const double2 *gseed, const AdjPlanes<T> &A,
                                double *part, double *acc, cudaStream_t st)
{
    // the planes (FP64) hold the full step's coefficients; a first step
    // (dt/2) and the FP32 adjoint form their own from the tables
    auto fn = adjoint_spin_fn<T, false>(p.Nth);
    if constexpr (sizeof(T) == 8)
        if (!p.first) fn = adjoint_spin_fn<T, true>(p.Nth);
    cudaError_t e = smem_limit_max((const void *)fn);
    if (e != cudaSuccess) return e;
    StepParams<T> q = p;
    q.tile_rows = tile_rows;
    const int grid = adjoint_grid<T>(p.Nr, tile_rows);
    fn<<<grid, 256, adjoint_spin_smem_bytes<T>(tile_rows, p.Nth), st>>>(q, sin, tape, gseed, A, part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_part_reduce6<<<1, 32, 0, st>>>(part, grid, acc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adjoint_planes(const StepParams<T> &p, int tile_rows, const double2 *gseed, const AdjPlanes<T> &A,
                                  double *part, double *acc, cudaStream_t st)
{
    if constexpr (sizeof(T) != 8) {
        return cudaErrorInvalidValue;
    } else {
        if (p.first) return cudaErrorInvalidValue;
        auto fn = adjoint_spin_fn<T, true, false>(p.Nth);
        cudaError_t e = smem_limit_max((const void *)fn);
        if (e != cudaSuccess) return e;
        StepParams<T> q = p;
        q.tile_rows = tile_rows;
        const int grid = adjoint_grid<T>(p.Nr, tile_rows);
        fn<<<grid, 256, adjoint_spin_smem_bytes<T>(tile_rows, p.Nth), st>>>(q, nullptr, nullptr, gseed, A, part);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_part_reduce6<<<1, 32, 0, st>>>(part, grid, acc);
        return cudaGetLastError();
    }
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
template size_t adjoint_spin_smem_bytes<float>(int, int);
template size_t adjoint_spin_smem_bytes<double>(int, int);
template cudaError_t launch_adjoint_spin<float>(const StepParams<float> &, int, const float2 *, const float2 *,
                                                const double2 *, const AdjPlanes<float> &, double *, double *,
                                                cudaStream_t);
template cudaError_t launch_adjoint_spin<double>(const StepParams<double> &, int, const double2 *, const double2 *,
                                                 const double2 *, const AdjPlanes<double> &, double *, double *,
                                                 cudaStream_t);
template cudaError_t launch_adjoint_planes<double>(const StepParams<double> &, int, const double2 *,
                                                   const AdjPlanes<double> &, double *, double *, cudaStream_t);
template cudaError_t launch_dot<float>(const float2 *, const float2 *, const float2 *, size_t, double *, double2 *,
                                       cudaStream_t);
template cudaError_t launch_dot<double>(const double2 *, const double2 *, const double2 *, size_t, double *,
                                        double2 *, cudaStream_t);

}  // namespace teuk
