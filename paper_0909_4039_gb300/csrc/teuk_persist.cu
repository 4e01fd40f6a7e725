// teuk_persist.cu -- persistent form of the split-scheme step kernel: one CTA
// per SM walks the tiles, a producer warp moves them by TMA bulk copies into
// two shared-memory buffers while the consumer threads compute.
#include "teuk_dev.cuh"

namespace teuk {
namespace {

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
            // phases of Eqs. 13 and 14 times their stage lengths dt/2 and dt
            const double2 e1 = phase_at(p.mOmega, tt), e2 = phase_at(p.mOmega, tt + 0.5 * p.dt64);
            sph[0] = make_double2(0.5 * p.dt64 * e1.x, 0.5 * p.dt64 * e1.y);
            sph[1] = make_double2(p.dt64 * e2.x, p.dt64 * e2.y);
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
            const unsigned br = (unsigned)q.npos * NSF * (unsigned)sizeof(T);
            mbar_expect_tx(&s_full[b], 3 * bs + br);
            bulk_g2s(bphi(b) + q.la * P, p.uin + (size_t)q.ga * N, bs, &s_full[b]);
            bulk_g2s(bpi(b) + q.la * P, p.uin + ((size_t)Nr + q.ga) * N, bs, &s_full[b]);
            bulk_g2s(bpiv(b) + q.la * P, K.piv + (size_t)q.ga * N, bs, &s_full[b]);
            bulk_g2s(brt(b) + q.lp * NSF, p.stab + (size_t)q.pos0 * NSF, br, &s_full[b]);
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
        T *sSt = brt(b);   // step-table entries of the tile
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
            for (int idx = tid; idx < (2 * R - 1) * NSF; idx += NC) {
                int e = idx / NSF;
                if (e < q.lp || e >= q.lp + q.npos) sSt[idx] = T(0);
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
            implicit_row_fwd<T, S>(K, sPhi + lrc * P, sPi + lrc * P, sPiv + lrc * P, sSt + 2 * lrc * NSF, sTh, N,
                                     active, in_tile, g, G, vec, active ? K.plan[gi] : 0);
        }
        bar();
        // The extraction row (its r-table entry and, after the Lax-Wendroff
        // phase, its state) is copied out for the sample below: the buffer
        // is refilled once it is handed back.
        const bool ext = p.i_ext >= i0 && p.i_ext < i0 + TR && p.i_ext < Nr;
        const int lx = p.i_ext - i0 + 1;
        if (ext && tid < NSF) xF[tid] = sSt[2 * lx * NSF + tid];
        const bool src = p.patch_np > 0 && i0 + TR >= p.patch_p0 && i0 - 1 <= p.patch_p0 + p.patch_np;
        lw_phase<T, false>(p, sPhi, sPi, sSt, sTh, 1, TR, i0 - 1, tid, NC, src, ph1, ph2, bar);
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
            implicit_row_fwd<T, S>(p.half, xPhi, xPi, p.half.piv + (size_t)p.i_ext * N, xF, sTh, N, active, mine,
                                     tid % G, G, vec, p.half.plan[p.i_ext]);
            __syncwarp();
            extract_warp<T>(p, xPhi, s_n + 1);
        }
    }
}

}  // namespace

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

}  // namespace teuk
