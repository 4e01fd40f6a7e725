// teuk_split.cuh -- split-scheme step kernels for sm_103a (tiled, two steps
// per launch, batched) and their launchers, for one state precision T;
// teuk_split_f32.cu and teuk_split_f64.cu instantiate them.
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
#pragma once

#include "teuk_dev.cuh"

namespace teuk {
namespace {

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

// Stored scan plans: the levels scan_plan chooses for every row of the
// grid and both implicit steps (dt and dt/2), for the multipliers of the LU
// solve of implicit_row_fwd (forward e_j sub_j, backward fk_j), from the
// same coefficient path (step table, theta tables and pivots as the step
// kernels read them).  One CTA of 256 threads covers 256 / G rows.
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
        ImpCoef<T, S> C;
        c2 w[S], y[S], fm[S];
        // the state rows are not needed: the pivot row stands in for them
        imp_load<T, S>(K, prow, prow, prow, p.stab + (size_t)(2 * gr) * NSF, p.thtab, N, len, j0, p.vec != 0, C, w, y);
#pragma unroll
        for (int k = 0; k < S; ++k) fm[k] = cscale<c2>(C.sub[k], C.e[k]);
        const ScanPlan<T> P = scan_plan<T, S>(fm, C.fk, g, G);
        if (in_grid && g == 0) (h ? plan_half : plan_full)[gi] = P.nf | (P.nb << 8);
    }
}

// Materialised coefficients of the FP64 path (MatPlanes): thread (e, j) of
// the grid covers step-table position e (node 2i or half node 2i+1) and
// theta j, forming exactly what the kernels would form in place (imp_row,
// imp_sg, imp_elem for the full step at nodes; lw_coef at every position).
template <typename T>
__global__ void __launch_bounds__(256) k_mat_coef(const StepParams<T> p, typename V2<T>::t *fk, typename V2<T>::t *dg,
                                                  typename V2<T>::t *ct, T *sub, T *qam, T *qap, T *lw)
{
    typedef typename V2<T>::t c2;
    const int N = p.Nth, Nr = p.Nr;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)(2 * Nr - 1) * N) return;
    const int e = (int)(idx / N), j = (int)(idx - (long long)e * N);
    const T *f = p.stab + (size_t)e * NSF;
    const T S2 = p.thtab[TF_S2 * N + j], C = p.thtab[TF_C * N + j];
    T beta;
    c2 kap;
    lw_coef<T>(f, S2, C, beta, kap);
    T *o = lw + ((size_t)e * N + j) * 4;
    o[0] = beta;
    o[1] = kap.x;
    o[2] = kap.y;
    o[3] = T(0);
    if (e & 1) return;
    const int i = e >> 1;
    const size_t q = (size_t)i * N + j;
    const c2 zero = cmk<c2>(T(0), T(0));
    if (i < 1 || i > Nr - 2) {
        // boundary rows: the step treats them as inactive and reads nothing here
        fk[q] = zero;
        dg[q] = zero;
        ct[q] = zero;
        sub[q] = qam[q] = qap[q] = T(0);
        return;
    }
    const ImpRow<T> r = imp_row(p.full, f);
    const T sg = imp_sg(r, S2);
    c2 vct, vdg, vfk;
    T vqam, vqap, vsub;
    imp_elem(p.full, r, sg, C, p.thtab[TF_AM * N + j], p.thtab[TF_A0 * N + j], p.thtab[TF_AP * N + j], p.full.piv[q],
             vct, vdg, vqam, vqap, vsub, vfk);
    fk[q] = vfk;
    dg[q] = vdg;
    ct[q] = vct;
    sub[q] = vsub;
    qam[q] = vqam;
    qap[q] = vqap;
}

}  // namespace

template <typename T>
cudaError_t launch_mat_coef(const StepParams<T> &p, cudaStream_t st)
{
    typedef typename V2<T>::t c2;
    if (!p.mat_on) return cudaSuccess;
    const long long n = (long long)(2 * p.Nr - 1) * p.Nth;
    k_mat_coef<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, (c2 *)p.mat.fk, (c2 *)p.mat.dg, (c2 *)p.mat.ct,
                                                              (T *)p.mat.sub, (T *)p.mat.qam, (T *)p.mat.qap,
                                                              (T *)p.mat.lw);
    return cudaGetLastError();
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
static void (*batch_fn(int seg, int ks))(const StepParams<T> *, const int2 *)
{
    // two steps per launch for segments of up to 8 elements (Ntheta <= 256)
    if (ks == 2) return seg == kSegNarrow ? k_split_batch<T, kSegNarrow, 2> : (seg == kSeg ? k_split_batch<T, kSeg, 2> : nullptr);
    return seg == kSegNarrow ? k_split_batch<T, kSegNarrow, 1>
                             : (seg == kSeg ? k_split_batch<T, kSeg, 1> : k_split_batch<T, kSegWide, 1>);
}

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

}  // namespace teuk
