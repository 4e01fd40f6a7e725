// teuk_adjoint.cu -- the step's waveform sample as an operator, the Hermitian
// adjoint of one split-scheme step with the source-parameter derivatives,
// and deterministic FP64 inner products (gradients of waveform losses).
#include "teuk_dev.cuh"

namespace teuk {
namespace {

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
template cudaError_t launch_dot<float>(const float2 *, const float2 *, const float2 *, size_t, double *, double2 *,
                                       cudaStream_t);
template cudaError_t launch_dot<double>(const double2 *, const double2 *, const double2 *, size_t, double *,
                                        double2 *, cudaStream_t);

}  // namespace teuk
