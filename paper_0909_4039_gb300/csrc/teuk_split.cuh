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

// Three time steps per launch: the tile carries three halo rows on either
// side, and the state moves once per three steps.
template <typename T, int S>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && S <= 4) ? 2 : 1) k_split_step3(const StepParams<T> p)
{
    split_tile<T, S, 3>(p, (int)blockIdx.x, (int)gridDim.x);
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
__global__ void __launch_bounds__(256) k_scan_plans(const StepParams<T> p, int *plan_full, int *plan_half,
                                                    typename V2<T>::t *seg_full, typename V2<T>::t *seg_half)
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
        // the lane segment's multiplier products, formed as scan_plan_lu forms them
        const ScanPlan<T> Q = scan_plan_products<T, S>(C);
        if (in_grid) {
            c2 *o = (h ? seg_half : seg_full) + ((size_t)gi * G + g) * 2;
            o[0] = Q.Af0;
            o[1] = Q.Ab0;
        }
    }
}

// ---- Pipelined form of k_split_step2 (two time steps per launch).
//
// gridDim.x persistent CTAs (about two per SM) walk the tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ...  Each CTA holds two tile buffers in shared
// memory: while tile k computes in one, the bulk copies of tile k+1 (state
// rows, step-table entries, scan plans; its pivot rows are prefetched into
// L2, where the row solves read them) land in the other, so the
// loads of every tile but the first overlap the arithmetic.  The per-tile
// work is that of split_tile with KS = 2 (same device functions, same
// results bit for bit); the extraction row is sampled from a copy, so the
// bulk store of a tile never waits.  Per buffer b and chunk c the mbarrier
// s_full[b][c] completes when the chunk's rows (chunk 0: also the table
// entries and plans) have landed; the buffer's k-th use waits on parity
// (k / 2) & 1.  Thread 0 refills a buffer only after the bulk store that
// last read it has finished reading (cp.async.bulk.wait_group.read).
// Every wait is bounded: a copy that does not land sets FLAG_TIMEOUT, the
// CTA waits (bounded) for the copies it issued and returns.
constexpr int kPipeChunks = 4;

template <typename T, int S, int NTH>
__global__ void __launch_bounds__(NTH, (NTH == 256 && sizeof(T) == 4 && S <= 4) ? 2 : 1)
    k_split_pipe(const StepParams<T> p)
{
    typedef typename V2<T>::t c2;
    constexpr int KS = 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double2 sph[2 * KS];
    __shared__ long long s_n;
    __shared__ __align__(8) unsigned long long s_full[2][kPipeChunks];
    const int Nr = p.Nr, N = p.Nth, TR = p.tile_rows, R = TR + 2 * KS, P = p.pitch;
    const int tid = threadIdx.x, NT = blockDim.x, G = p.group;
    const int ntiles = (Nr + TR - 1) / TR;
    const PipeSmem L = pipe_smem_plan(R, N, (int)sizeof(T));
    T *sTh = (T *)(smem_raw + L.th);
    c2 *xPhi = (c2 *)(smem_raw + L.xphi);
    c2 *xPi = (c2 *)(smem_raw + L.xpi);
    const ImpConst<T> &K = p.full;
    const int rpp = NT / G;   // theta rows per implicit pass
    int cr = rpp;             // rows per chunk
    while ((R + cr - 1) / cr > kPipeChunks) cr += rpp;
    const int nch = (R + cr - 1) / cr;
    const int wait_lim = p.wait0 >= 0 ? p.wait0 : kWaitLimit;
    const c2 zero = cmk<c2>(T(0), T(0));

    // tile t: rows g0 .. g0+R-1, on the grid [ga, gb] from tile row la; the
    // plan copy starts at global row a0 (a 16-byte boundary)
    struct Geo {
        int i0, g0, ga, gb, la, nrows, a0;
    };
    auto geo = [&](int t) {
        Geo q;
        q.i0 = t * TR;
        q.g0 = q.i0 - KS;
        q.ga = q.g0 < 0 ? 0 : q.g0;
        q.gb = q.g0 + R - 1 > Nr - 1 ? Nr - 1 : q.g0 + R - 1;
        q.la = q.ga - q.g0;
        q.nrows = q.gb - q.ga + 1;
        q.a0 = q.ga & ~3;
        return q;
    };
    auto buf = [&](int b) { return smem_raw + L.buf + (unsigned)b * L.bsize; };
    // bulk copies of tile t into buffer b (thread 0)
    auto issue = [&](int t, int b) {
        const Geo q = geo(t);
        unsigned char *B = buf(b);
        c2 *bPhi = (c2 *)B, *bPi = (c2 *)(B + L.pi);
        T *bSt = (T *)(B + L.st);
        int *bPl = (int *)(B + L.plan);
        const int e0 = 2 * q.ga, e1 = 2 * q.gb + 1 > 2 * Nr - 2 ? 2 * Nr - 2 : 2 * q.gb + 1;
        const unsigned st_bytes = (unsigned)(e1 - e0 + 1) * NSF * (unsigned)sizeof(T);
        const unsigned pl_bytes = (unsigned)(((q.gb + 1 - q.a0) + 3) & ~3) * 4u;
        for (int c = 0; c < nch; ++c) {
            int r0 = c * cr, r1 = r0 + cr;
            if (r1 > R) r1 = R;
            if (r0 < q.la) r0 = q.la;
            if (r1 > q.la + q.nrows) r1 = q.la + q.nrows;
            const unsigned bytes = r1 > r0 ? (unsigned)(r1 - r0) * (unsigned)N * (unsigned)sizeof(c2) : 0u;
            mbar_expect_tx(&s_full[b][c], 2 * bytes + (c == 0 ? st_bytes + pl_bytes : 0u));
            if (bytes) {
                const size_t gr = (size_t)(q.ga + r0 - q.la);
                bulk_g2s(bPhi + r0 * P, p.uin + gr * N, bytes, &s_full[b][c]);
                bulk_g2s(bPi + r0 * P, p.uin + ((size_t)Nr + gr) * N, bytes, &s_full[b][c]);
                prefetch_l2(K.piv + gr * N, bytes);
            }
            if (c == 0) {
                bulk_g2s(bSt + (e0 - 2 * q.g0) * NSF, p.stab + (size_t)e0 * NSF, st_bytes, &s_full[b][0]);
                bulk_g2s(bPl, K.plan + q.a0, pl_bytes, &s_full[b][0]);
            }
        }
    };
    // bounded wait for every chunk of buffer b's use with parity par (thread 0, after a failure)
    auto drain = [&](int b, unsigned par) {
        for (int c = 0; c < nch; ++c) mbar_wait(&s_full[b][c], par, kWaitLimit);
    };

    if (tid == 0) {
        long long n = *((volatile long long *)&p.ctl->step);
        s_n = n;
        // the last CTA to read the step index advances it (one ticket per CTA)
        __threadfence();
        unsigned t = atomicAdd(&p.ctl->ticket, 1u);
        if (t == gridDim.x - 1u) {
            p.ctl->ticket = 0u;
            p.ctl->step = n + KS;
        }
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < nch; ++c) mbar_init(&s_full[b][c], 1);
        if ((int)blockIdx.x < ntiles) issue((int)blockIdx.x, 0);
    }
    for (int idx = tid; idx < NTF * N; idx += NT) sTh[idx] = p.thtab[idx];
    __syncthreads();

    const int g = tid % G;
    const bool vec = p.vec != 0;
    int ok = 1;
    int k = 0;
    for (int t = (int)blockIdx.x; t < ntiles; t += (int)gridDim.x, ++k) {
        const int b = k & 1;
        const unsigned par = (unsigned)((k >> 1) & 1);
        const Geo q = geo(t);
        unsigned char *B = buf(b);
        c2 *sPhi = (c2 *)B, *sPi = (c2 *)(B + L.pi);
        T *sSt = (T *)(B + L.st);
        const int *sPl = (const int *)(B + L.plan);
        const int tn = t + (int)gridDim.x;
        const int i0 = q.i0, g0 = q.g0;
        const bool src = p.patch_np > 0 && i0 + TR + KS - 1 >= p.patch_p0 && g0 <= p.patch_p0 + p.patch_np;
        if (tid == 0 && src)
            for (int s = 0; s < KS; ++s) {
                // phases of Eqs. 13 and 14 times their stage lengths dt/2 and dt
                const double tt = (double)(s_n + s) * p.dt64;
                const double2 e1 = phase_at(p.mOmega, tt), e2 = phase_at(p.mOmega, tt + 0.5 * p.dt64);
                sph[2 * s] = make_double2(0.5 * p.dt64 * e1.x, 0.5 * p.dt64 * e1.y);
                sph[2 * s + 1] = make_double2(p.dt64 * e2.x, p.dt64 * e2.y);
            }
        const bool ext = p.i_ext >= i0 && p.i_ext < i0 + TR && p.i_ext < Nr;
        const int lx = p.i_ext - g0;
        // implicit step on tile rows [lo, hi); the first step waits, pass by
        // pass, for the chunks holding the pass's rows.  Rows off the grid
        // and the boundary rows are inactive: the step writes zeros there.
        auto implicit_rows = [&](int lo, int hi, bool wait) {
            for (int base = lo; base < hi; base += rpp) {
                if (wait && ok) {
                    int last = base + rpp - 1;
                    if (last > hi - 1) last = hi - 1;
                    for (int c = base / cr; c <= last / cr; ++c) ok &= (int)mbar_wait(&s_full[b][c], par, wait_lim);
                }
                const int lr = base + tid / G;
                const bool in_tile = lr < hi;
                const int gi = g0 + lr;
                const bool active = in_tile && gi >= 1 && gi <= Nr - 2;
                const int lrc = in_tile ? lr : lo;
                const int plan = active ? sPl[gi - q.a0] : 0;
                if constexpr (sizeof(T) == 8) {
                    if (p.mat_on) {
                        implicit_row_fwd<T, S, true>(K, sPhi + lrc * P, sPi + lrc * P, K.piv + (size_t)(active ? gi : 1) * N, nullptr, nullptr,
                                                     N, active, in_tile, g, G, vec, plan, &p.mat, gi);
                        continue;
                    }
                }
                implicit_row_fwd<T, S>(K, sPhi + lrc * P, sPi + lrc * P, K.piv + (size_t)(active ? gi : 1) * N, sSt + 2 * lrc * NSF, sTh, N,
                                       active, in_tile, g, G, vec, plan);
            }
        };
        // Lax-Wendroff stages of step s on tile rows r0 .. r0+nr-1
        auto lw = [&](int s, int r0, int nr) {
            c2 ph1 = zero, ph2 = zero;
            if (src) {
                ph1 = from_d2<T>(sph[2 * s]);
                ph2 = from_d2<T>(sph[2 * s + 1]);
            }
            const auto sync_all = [] { __syncthreads(); };
            const bool interior = g0 >= 1 && g0 + R <= Nr - 1;
            if constexpr (sizeof(T) == 8) {
                if (p.mat_on) {
                    if (interior)
                        lw_phase<T, true, true>(p, sPhi, sPi, sSt, sTh, r0, nr, g0, tid, NT, src, ph1, ph2, sync_all);
                    else
                        lw_phase<T, false, true>(p, sPhi, sPi, sSt, sTh, r0, nr, g0, tid, NT, src, ph1, ph2, sync_all);
                    return;
                }
            }
            if (interior)
                lw_phase<T, true>(p, sPhi, sPi, sSt, sTh, r0, nr, g0, tid, NT, src, ph1, ph2, sync_all);
            else
                lw_phase<T, false>(p, sPhi, sPi, sSt, sTh, r0, nr, g0, tid, NT, src, ph1, ph2, sync_all);
        };
        // copy of the extraction row (warp 0)
        auto copy_row = [&]() {
            if (tid < 32)
                for (int j = tid; j < N; j += 32) {
                    xPhi[j] = sPhi[lx * P + j];
                    xPi[j] = sPi[lx * P + j];
                }
        };
        // physical sample u = C_{dt/2} s of the copy (warp 0, after copy_row)
        auto sample_copy = [&](long long slot) {
            if (tid < 32) {
                __syncwarp();
                const bool mine = tid < G;
                const bool active = mine && p.i_ext >= 1 && p.i_ext <= Nr - 2;
                implicit_row_fwd<T, S>(p.half, xPhi, xPi, p.half.piv + (size_t)p.i_ext * N, sSt + 2 * lx * NSF, sTh,
                                       N, active, mine, tid % G, G, vec, p.half.plan[p.i_ext]);
                __syncwarp();
                extract_warp<T>(p, xPhi, slot);
            }
        };

        // ---- step 1: implicit on all R rows, then Lax-Wendroff on rows 1 .. R-2
        implicit_rows(0, R, true);
        if (ok)
            for (int c = 0; c < nch; ++c) ok &= (int)mbar_wait(&s_full[b][c], par, wait_lim);
        if (!__syncthreads_and(ok)) {
            // a copy did not land: report, wait (bounded) for every copy this CTA issued, leave
            if (tid == 0) {
                atomicOr(&p.ctl->flags, FLAG_TIMEOUT);
                drain(b, par);   // tile k+1's copies are not issued before this point
                bulk_wait_read();
            }
            return;
        }
        lw(0, 1, R - 2);
        if (tid == 0 && tn < ntiles) {
            // the other buffer held tile k-1, whose store has long been read
            // out by now (the wait returns at once): refill it with tile k+1
            bulk_wait_read();
            issue(tn, b ^ 1);
        }
        __syncthreads();
        if (ext) {
            // the row goes on into step 2; its sample comes from a copy
            copy_row();
            __syncthreads();
            sample_copy(s_n + 1);
        }
        // ---- step 2: implicit on rows 1 .. R-2, Lax-Wendroff on rows 2 .. R-3
        implicit_rows(1, R - 1, false);
        __syncthreads();
        lw(1, 2, R - 4);
        // ---- store the output rows (tile rows 2 .. TR+1); the sample of
        // step n+2 comes from a copy, so the store need not be waited for
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            const int nout = (Nr - i0) < TR ? (Nr - i0) : TR;
            const unsigned bytes = (unsigned)nout * (unsigned)N * (unsigned)sizeof(c2);
            bulk_s2g(p.uout + (size_t)i0 * N, sPhi + KS * P, bytes);
            bulk_s2g(p.uout + ((size_t)Nr + i0) * N, sPi + KS * P, bytes);
            bulk_commit();
        }
        if (ext) {
            copy_row();   // reads the rows the store reads too
            sample_copy(s_n + KS);
        }
        // every thread is done with buffer b before thread 0 refills it
        __syncthreads();
    }
    if (tid == 0) bulk_wait_read();   // the last stores have read their rows before the CTA exits
}

// Materialised coefficients (MatPlanes): thread (e, j) of the grid covers
// step-table position e (node 2i or half node 2i+1) and theta j, forming
// exactly what the kernels would form in place (imp_row, imp_sg, imp_elem
// for the full step at nodes; lw_coef at every position), and where asked
// their spin derivatives (lw_coef_da, imp_da) for the adjoint.
template <typename T>
__global__ void __launch_bounds__(256) k_mat_coef(const StepParams<T> p, const MatOut<T> o)
{
    typedef typename V2<T>::t c2;
    const int N = p.Nth, Nr = p.Nr;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)(2 * Nr - 1) * N) return;
    const int e = (int)(idx / N), j = (int)(idx - (long long)e * N);
    const T *f = p.stab + (size_t)e * NSF;
    const T S2 = p.thtab[TF_S2 * N + j], C = p.thtab[TF_C * N + j];
    T beta, sg;
    c2 kap;
    lw_coef<T>(f, S2, C, beta, kap, &sg);
    T *lo = o.lw + ((size_t)e * N + j) * 4;
    lo[0] = beta;
    lo[1] = kap.x;
    lo[2] = kap.y;
    lo[3] = sg;
    if (o.dlw) {
        const LwDa<T> d = lw_coef_da<T>(f, p.dstab + (size_t)e * NSF, S2, C);
        T *dl = o.dlw + ((size_t)e * N + j) * 4;
        dl[0] = d.dbeta;
        dl[1] = d.dkap.x;
        dl[2] = d.dkap.y;
        dl[3] = d.dsg;
    }
    if (e & 1) return;
    const int i = e >> 1;
    const size_t q = (size_t)i * N + j;
    const c2 zero = cmk<c2>(T(0), T(0));
    if (i < 1 || i > Nr - 2) {
        // boundary rows: the step treats them as inactive and reads nothing here
        o.fk[q] = zero;
        o.dg[q] = zero;
        o.ct[q] = zero;
        o.sub[q] = o.qam[q] = o.qap[q] = T(0);
        if (o.dimp)
            for (int k = 0; k < 8; ++k) o.dimp[q * 8 + k] = T(0);
        return;
    }
    const ImpRow<T> r = imp_row(p.full, f);
    const T am = p.thtab[TF_AM * N + j], a0 = p.thtab[TF_A0 * N + j], ap = p.thtab[TF_AP * N + j];
    c2 vct, vdg, vfk;
    T vqam, vqap, vsub;
    imp_elem(p.full, r, imp_sg(r, S2), C, am, a0, ap, p.full.piv[q], vct, vdg, vqam, vqap, vsub, vfk);
    o.fk[q] = vfk;
    o.dg[q] = vdg;
    o.ct[q] = vct;
    o.sub[q] = vsub;
    o.qam[q] = vqam;
    o.qap[q] = vqap;
    if (o.dimp) {
        T fr[8], dfr[8];
        vload<8>(fr, f);
        vload<8>(dfr, p.dstab + (size_t)e * NSF);
        c2 ddg, dct;
        T dqam, dqap;
        imp_da<T>(r, fr, dfr, S2, C, am, a0, ap, ddg, dct, dqam, dqap);
        T *dq = o.dimp + q * 8;
        dq[0] = ddg.x;
        dq[1] = ddg.y;
        dq[2] = dct.x;
        dq[3] = dct.y;
        dq[4] = dqam;
        dq[5] = dqap;
        dq[6] = T(0);
        dq[7] = T(0);
    }
}

}  // namespace

template <typename T>
size_t pipe_smem_bytes(int tile_rows, int Nth)
{
    return pipe_smem_plan(tile_rows + 4, Nth, (int)sizeof(T)).total;
}

// The pipelined kernel for Ntheta and `threads` per CTA (256 or 512; 512
// only for segments of up to 8 elements), or nullptr.
template <typename T>
static void (*pipe_fn(int Nth, int threads))(const StepParams<T>)
{
    const int seg = implicit_seg(Nth);
    if (threads == 256)
        return seg == kSegNarrow ? k_split_pipe<T, kSegNarrow, 256>
                                 : (seg == kSeg ? k_split_pipe<T, kSeg, 256> : k_split_pipe<T, kSegWide, 256>);
    if (threads == 512)
        return seg == kSegNarrow ? k_split_pipe<T, kSegNarrow, 512> : (seg == kSeg ? k_split_pipe<T, kSeg, 512> : nullptr);
    return nullptr;
}

template <typename T>
int pipe_blocks_per_sm(int Nth, int threads, size_t smem)
{
    auto fn = pipe_fn<T>(Nth, threads);
    if (!fn) return 0;
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
cudaError_t launch_split_pipe(const StepParams<T> &p, int threads, int grid, size_t smem, cudaStream_t st)
{
    if (p.first || p.imp_only || !p.bulk || p.nfix >= 0 || grid < 1) return cudaErrorInvalidValue;
    auto fn = pipe_fn<T>(p.Nth, threads);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = smem_limit_max((const void *)fn);
    if (e != cudaSuccess) return e;
    fn<<<grid, threads, smem, st>>>(p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mat_coef_to(const StepParams<T> &p, const MatOut<T> &o, cudaStream_t st)
{
    const long long n = (long long)(2 * p.Nr - 1) * p.Nth;
    k_mat_coef<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, o);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mat_coef(const StepParams<T> &p, cudaStream_t st)
{
    typedef typename V2<T>::t c2;
    if (!p.mat_on) return cudaSuccess;
    MatOut<T> o;
    o.fk = (c2 *)p.mat.fk;
    o.dg = (c2 *)p.mat.dg;
    o.ct = (c2 *)p.mat.ct;
    o.sub = (T *)p.mat.sub;
    o.qam = (T *)p.mat.qam;
    o.qap = (T *)p.mat.qap;
    o.lw = (T *)p.mat.lw;
    o.dlw = o.dimp = nullptr;
    return launch_mat_coef_to<T>(p, o, st);
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
cudaError_t launch_scan_plans(const StepParams<T> &p, int *plan_full, int *plan_half, typename V2<T>::t *seg_full,
                              typename V2<T>::t *seg_half, cudaStream_t st)
{
    const int seg = implicit_seg(p.Nth);
    auto fn = seg == kSegNarrow ? k_scan_plans<T, kSegNarrow>
                                : (seg == kSeg ? k_scan_plans<T, kSeg> : k_scan_plans<T, kSegWide>);
    const int rows = 256 / p.group;
    fn<<<(p.Nr + rows - 1) / rows, 256, 0, st>>>(p, plan_full, plan_half, seg_full, seg_half);
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
static void (*split3_fn(int Nth))(const StepParams<T>)
{
    const int seg = implicit_seg(Nth);
    return seg == kSegNarrow ? k_split_step3<T, kSegNarrow>
                             : (seg == kSeg ? k_split_step3<T, kSeg> : k_split_step3<T, kSegWide>);
}

template <typename T>
size_t split3_smem_bytes(int tile_rows, int Nth)
{
    return split_smem_plan(tile_rows + 6, Nth, (int)sizeof(T)).total + 2 * (size_t)Nth * sizeof(typename V2<T>::t);
}

template <typename T>
int split3_blocks_per_sm(int Nth, int threads, size_t smem)
{
    auto fn = split3_fn<T>(Nth);
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
cudaError_t launch_split_step3(const StepParams<T> &p, int threads, size_t smem, cudaStream_t st)
{
    if (p.first || p.imp_only) return cudaErrorInvalidValue;   // three full steps only
    auto fn = split3_fn<T>(p.Nth);
    cudaError_t e = smem_limit_max((const void *)fn);
    if (e != cudaSuccess) return e;
    int grid = (p.Nr + p.tile_rows - 1) / p.tile_rows;
    fn<<<grid, threads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace teuk
