// teuk_api.cu -- host implementation of the C ABI declared in include/teuk.h.
//
// Validation, workspace layout, the stability guards, the ping-pong of the
// two state levels, CUDA-graph replay of long runs, state and waveform I/O.
// All arithmetic of the method runs in the kernels of teuk_coef.cu and
// teuk_step.cu; the host computes only grid constants and bounds.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <algorithm>
#include <vector>

#include "teuk_internal.cuh"

using namespace teuk;

namespace {

constexpr int kGraphChunk = 64;          // steps per captured graph (even)
constexpr size_t kStagingElems = 1u << 20;  // complex doubles in the staging area

thread_local char g_init_err[512] = "";

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct teuk_ctx {
    teuk_grid_desc d;
    double drs, dt;
    int i_ext;
    char *state;
    char *coef;
    double2 *wave;
    int64_t cap;
    Layout L;
    size_t level_bytes;     // one time level
    int cur;                // level holding the current state
    int shifted;            // split scheme: the level holds s_n (u_n = C_{dt/2} s_n)
    int64_t step;           // host mirror of the device step counter
    int64_t rec_lo;         // oldest recorded waveform step
    // source: patch rows of the forward source (patch_np = 0: off) and of
    // the unit-amplitude patch, which exists whenever the orbit is valid
    // (derivatives with respect to the amplitude and the orbit radius)
    int patch_p0, patch_np, unit_p0, unit_np;
    double mOmega;
    double amp_re, amp_im, rs0, sig_r, drs0_dr0, m_dOmega;
    double m_dOmega_da;     // m dOmega/da (Kepler frequency; 0 for a given Omega)
    // launch configuration: tiled kernel (tile_rows, threads, smem) or the
    // persistent kernel (persist = 1: nc consumer threads, grid CTAs,
    // persist_smem); the tiled kernel at the same tile height also serves
    // the state output (C_{dt/2} only)
    int tile_rows, threads;
    size_t smem;
    int persist, nc, grid;
    int pipe;                // the pipelined two-step kernel (grid persistent CTAs)
    size_t persist_smem;
    int ks;                  // time steps per launch of the tiled kernel (1, 2 or 3)
    int wait0;               // teuk_set_wait_limit (< 0: default bound)
    size_t smem2;            // shared memory of the two- or three-step kernel
    const void *adj_ws;      // adjoint workspace whose coefficient planes teuk_adjoint_prepare filled
    // graphs, one per starting level
    cudaGraphExec_t graph[2];
    cudaStream_t graph_stream[2];
    char err[512];
};

namespace teuk {

Layout make_layout(const teuk_grid_desc &d)
{
    Layout L;
    size_t Nr = (size_t)d.Nr, N = (size_t)d.Ntheta;
    size_t rs = sizeof(double) * (2 * Nr - 1) * NRF;
    size_t ts = sizeof(double) * NTF * N;
    bool f32 = d.precision == TEUK_FP32;
    size_t c2 = f32 ? sizeof(float2) : sizeof(double2);
    size_t patch_rows = Nr < (size_t)TEUK_MAX_PATCH_ROWS ? Nr : (size_t)TEUK_MAX_PATCH_ROWS;
    size_t off = 0;
    L.rtab64 = off; off = align256(off + rs);
    L.rtabT = f32 ? off : L.rtab64; if (f32) off = align256(off + rs / 2);
    L.stab = off; off = align256(off + (f32 ? sizeof(float) : sizeof(double)) * (2 * Nr - 1) * NSF);
    L.dstab = off; off = align256(off + (f32 ? sizeof(float) : sizeof(double)) * (2 * Nr - 1) * NSF);
    L.th64 = off; off = align256(off + ts);
    L.thT = f32 ? off : L.th64; if (f32) off = align256(off + ts / 2);
    L.piv = off; off = align256(off + c2 * N * Nr);
    L.pivh = off; off = align256(off + c2 * N * Nr);
    L.plan = off; off = align256(off + sizeof(int) * Nr);
    L.planh = off; off = align256(off + sizeof(int) * Nr);
    {
        const size_t lanes = (size_t)implicit_group((int)N);
        L.seg = off; off = align256(off + c2 * 2 * lanes * Nr);
        L.segh = off; off = align256(off + c2 * 2 * lanes * Nr);
    }
    L.patch = off; off = align256(off + c2 * 2 * N * patch_rows);
    L.patchu = off; off = align256(off + c2 * 2 * N * patch_rows);
    L.w = off; off = align256(off + sizeof(double) * N);
    L.ctl = off; off = align256(off + sizeof(Ctl));
    L.staging_elems = 0;
    L.staging = off;
    if (f32) {
        size_t want = 2 * Nr * N;
        L.staging_elems = want < kStagingElems ? want : kStagingElems;
        off = align256(off + sizeof(double2) * L.staging_elems);
    }
    L.scratch = off;
    if (d.scheme == TEUK_SCHEME_LITERAL) off = align256(off + c2 * 2 * (Nr - 1) * N);
    // FP64 split scheme: materialised coefficients (MatPlanes), three complex
    // and three real planes [Nr][N], then the Lax-Wendroff planes [2Nr-1][N][4]
    L.mat = off;
    L.mat_bytes = 0;
    if (!f32 && d.scheme == TEUK_SCHEME_SPLIT) {
        L.mat_bytes = align256(sizeof(double) * Nr * N * 9) + sizeof(double) * 4 * (2 * Nr - 1) * N;
        off = align256(off + L.mat_bytes);
    }
    L.total = off;
    return L;
}

}  // namespace teuk

namespace {

__attribute__((format(printf, 3, 4))) int set_err(teuk_ctx *c, int code, const char *fmt, ...)
{
    char *buf = c ? c->err : g_init_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_err(teuk_ctx *c, cudaError_t e, const char *where)
{
    char *buf = c ? c->err : g_init_err;
    snprintf(buf, 512, "%s: %s", where, cudaGetErrorString(e));
    return TEUK_E_CUDA;
}

#define CK(call, where)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_err(c, e_, where); \
    } while (0)

int validate(const teuk_grid_desc *d, char *msg)
{
    if (!d) { snprintf(msg, 512, "descriptor is NULL"); return TEUK_E_INVAL; }
    if (d->Nr < 3 || d->Nr > (1LL << 28)) { snprintf(msg, 512, "Nr=%lld out of range [3, 2^28]", (long long)d->Nr); return TEUK_E_INVAL; }
    if (d->Ntheta < 1 || d->Ntheta > TEUK_MAX_NTHETA) { snprintf(msg, 512, "Ntheta=%lld out of range [1, %d]", (long long)d->Ntheta, TEUK_MAX_NTHETA); return TEUK_E_INVAL; }
    if (d->Nr * d->Ntheta > (1LL << 31)) { snprintf(msg, 512, "Nr*Ntheta exceeds 2^31"); return TEUK_E_INVAL; }
    if (!(d->M > 0.0) || !isfinite(d->M)) { snprintf(msg, 512, "M must be positive"); return TEUK_E_INVAL; }
    if (!(fabs(d->a) < d->M)) { snprintf(msg, 512, "need |a| < M"); return TEUK_E_INVAL; }
    if (d->s < -2 || d->s > 2) { snprintf(msg, 512, "spin weight s=%d not in [-2, 2]", d->s); return TEUK_E_INVAL; }
    if (!isfinite(d->rstar_min) || !isfinite(d->rstar_max) || !(d->rstar_max > d->rstar_min)) { snprintf(msg, 512, "need rstar_max > rstar_min"); return TEUK_E_INVAL; }
    if (!isfinite(d->dt) || !isfinite(d->rstar_extract)) { snprintf(msg, 512, "dt and rstar_extract must be finite"); return TEUK_E_INVAL; }
    if (d->precision != TEUK_FP64 && d->precision != TEUK_FP32) { snprintf(msg, 512, "precision must be TEUK_FP64 or TEUK_FP32"); return TEUK_E_INVAL; }
    if (d->scheme != TEUK_SCHEME_SPLIT && d->scheme != TEUK_SCHEME_LITERAL) { snprintf(msg, 512, "unknown scheme"); return TEUK_E_INVAL; }
    if (d->reserved != 0) { snprintf(msg, 512, "reserved field must be 0"); return TEUK_E_INVAL; }
    return TEUK_OK;
}

// Eq. 2 integrated, host copy for the orbit radius: r*(r).
double host_rstar(double M, double a, double r)
{
    double d = sqrt(M * M - a * a), rp = M + d, rm = M - d;
    return r + (M * rp / d) * log((r - rp) / (2.0 * M)) - (M * rm / d) * log((r - rm) / (2.0 * M));
}

// Bounds over the whole exterior (sampled on a log grid in r - r_+):
// b_max = max b (radial characteristic speed), q_max = max Delta/Sigma^2,
// ct_max = max |c_t|.
void host_bounds(const teuk_grid_desc &d, double *b_max, double *q_max, double *ct_max)
{
    double M = d.M, a = d.a, s = d.s, m = d.m;
    double dd = sqrt(M * M - a * a), rp = M + dd, rm = M - dd;
    double bm = 1.0, qm = 0.0, cm = 0.0;
    for (int k = 0; k <= 4000; ++k) {
        double x = exp(log(1e-10) + (log(1e8) - log(1e-10)) * k / 4000.0);
        double r = rp + x, D = x * (x + rp - rm), R = r * r + a * a;
        for (int e = 0; e <= 1; ++e) {
            double s2 = (double)e;   // sin^2 = 0 or 1 bracket Sigma^2
            double sig2 = R * R - a * a * D * s2;
            double b = R / sqrt(sig2), q = D / sig2;
            double ctr = 2.0 * s * (r * D - M * (r * r - a * a)) / sig2;
            double cti = (fabs(4.0 * M * a * m * r) + fabs(2.0 * s * a * D)) / sig2;
            bm = fmax(bm, b);
            qm = fmax(qm, q);
            cm = fmax(cm, sqrt(ctr * ctr + cti * cti));
        }
    }
    *b_max = bm;
    *q_max = qm;
    *ct_max = cm;
}

// Gershgorin bound of the discrete angular operator (folded ghost rows).
double host_atheta_bound(const teuk_grid_desc &d)
{
    int N = (int)d.Ntheta;
    double dth = kPi / N, lam = 0.0;
    double par = (abs(d.m) % 2 == 0) ? 1.0 : -1.0;
    for (int j = 0; j < N; ++j) {
        double th = (j + 0.5) * dth, sn = sin(th), cs = cos(th), cot = cs / sn;
        double am = -(1.0 - 0.5 * cot * dth) / (dth * dth), ap = -(1.0 + 0.5 * cot * dth) / (dth * dth);
        double mc = d.m + d.s * cs;
        double a0 = 2.0 / (dth * dth) + mc * mc / (sn * sn) - d.s;
        if (j == 0) { a0 += par * am; am = 0.0; }
        if (j == N - 1) { a0 += par * ap; ap = 0.0; }
        lam = fmax(lam, fabs(am) + fabs(a0) + fabs(ap));
    }
    return lam;
}

// Launch configurations of the split step and their model cost.
//
// Tiled kernel (256 threads, one tile per CTA): a tile of R = TR + 2 rows
// costs about 0.6 Rpad + 0.4 R + 4 row-times, where Rpad rounds R up to
// whole passes of the implicit phase (256 threads / G rows per pass) and the
// 4 stands for load latency and barriers; k CTAs share an SM, so one wave
// costs k times that and the grid needs ceil(tiles / (k SMs)) waves, with a
// 20 % penalty for k = 1 (no second CTA to overlap memory with compute).
//
// Persistent kernel (nc consumer threads + a producer warp, one CTA per SM,
// tiles double-buffered): a CTA computes ceil(tiles / grid) tiles of
// (0.6 Rpad + 0.4 R) (256 / nc) + 2 row-times each (Rpad in passes of
// nc / G rows; the 2 for its barriers), plus the first tile's load.  Its
// consumers move in lockstep between barriers, which costs about a factor
// of two per row-time against the tiled kernel's two independent CTAs per
// SM (measured on 16384 x 128 at equal tile height).
struct TileCand {
    double cost;             // model cost per time step
    int R;                   // tile_rows + 2
    int persist, nc, grid;
    int ks;                  // time steps per launch (tiled kernel: 1, 2 or 3)
    int pipe;                // 1: the pipelined two-step kernel (grid persistent CTAs)
    size_t smem;
};

static int sm_count()
{
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    return nsm;
}

// A tiled-kernel candidate of height TR (false if it does not fit).
static bool tiled_cand(const teuk_ctx *c, int TR, int nsm, TileCand *out)
{
    const int N = (int)c->d.Ntheta;
    const bool f32 = c->d.precision == TEUK_FP32;
    const int threads = 256, R = TR + 2;
    size_t sm = f32 ? split_smem_bytes<float>(TR, N) : split_smem_bytes<double>(TR, N);
    if (sm > 227 * 1024) return false;
    int k = f32 ? split_blocks_per_sm<float>(N, threads, sm) : split_blocks_per_sm<double>(N, threads, sm);
    if (k < 1) return false;
    const long long Nr = c->d.Nr;
    long long tiles = (Nr + TR - 1) / TR;
    long long waves = (tiles + (long long)k * nsm - 1) / ((long long)k * nsm);
    int rpp = threads / implicit_group(N);
    int rpad = ((R + rpp - 1) / rpp) * rpp;
    double rows = 0.6 * rpad + 0.4 * R + 4.0;
    out->cost = (double)waves * k * rows * (k == 1 ? 1.2 : 1.0);
    out->R = R;
    out->persist = 0;
    out->nc = 0;
    out->grid = (int)tiles;
    out->ks = 1;
    out->pipe = 0;
    out->smem = sm;
    return true;
}

// A two-steps-per-launch candidate of height TR: per step, half of a tile
// whose first step covers TR + 4 rows (implicit) and TR + 2 (LW) and whose
// second covers TR + 2 and TR, with one load latency per two steps.
static bool tiled2_cand(const teuk_ctx *c, int TR, int nsm, TileCand *out)
{
    const int N = (int)c->d.Ntheta;
    const bool f32 = c->d.precision == TEUK_FP32;
    const int threads = 256;
    size_t sm = f32 ? split2_smem_bytes<float>(TR, N) : split2_smem_bytes<double>(TR, N);
    if (sm > 227 * 1024) return false;
    int k = f32 ? split2_blocks_per_sm<float>(N, threads, sm) : split2_blocks_per_sm<double>(N, threads, sm);
    if (k < 1) return false;
    const long long Nr = c->d.Nr;
    long long tiles = (Nr + TR - 1) / TR;
    long long waves = (tiles + (long long)k * nsm - 1) / ((long long)k * nsm);
    int rpp = threads / implicit_group(N);
    auto rpad = [&](int r) { return ((r + rpp - 1) / rpp) * rpp; };
    double rows = 0.6 * (rpad(TR + 4) + rpad(TR + 2)) + 0.4 * (2.0 * TR + 6.0) + 4.0;
    out->cost = 0.5 * (double)waves * k * rows * (k == 1 ? 1.2 : 1.0);
    out->R = TR + 2;
    out->persist = 0;
    out->nc = 0;
    out->grid = (int)tiles;
    out->ks = 2;
    out->pipe = 0;
    out->smem = sm;
    return true;
}

// A three-steps-per-launch candidate of height TR: per step, a third of a
// tile whose steps cover TR + 6, TR + 4 and TR + 2 rows (implicit) and
// TR + 4, TR + 2 and TR (LW).  The model leaves it out of the default
// choice (tile_candidates); the autotuners time it at the heights of the
// model-best two-step candidates.
static bool tiled3_cand(const teuk_ctx *c, int TR, int nsm, TileCand *out)
{
    const int N = (int)c->d.Ntheta;
    const bool f32 = c->d.precision == TEUK_FP32;
    const int threads = 256;
    if (TR > kMaxTileRows - 6) return false;
    size_t sm = f32 ? split3_smem_bytes<float>(TR, N) : split3_smem_bytes<double>(TR, N);
    if (sm > 227 * 1024) return false;
    int k = f32 ? split3_blocks_per_sm<float>(N, threads, sm) : split3_blocks_per_sm<double>(N, threads, sm);
    if (k < 1) return false;
    const long long Nr = c->d.Nr;
    long long tiles = (Nr + TR - 1) / TR;
    long long waves = (tiles + (long long)k * nsm - 1) / ((long long)k * nsm);
    int rpp = threads / implicit_group(N);
    auto rpad = [&](int r) { return ((r + rpp - 1) / rpp) * rpp; };
    double rows = 0.6 * (rpad(TR + 6) + rpad(TR + 4) + rpad(TR + 2)) + 0.4 * (3.0 * TR + 9.0) + 4.0;
    out->cost = (double)waves * k * rows * (k == 1 ? 1.2 : 1.0) / 3.0;
    out->R = TR + 2;
    out->persist = 0;
    out->nc = 0;
    out->grid = (int)tiles;
    out->ks = 3;
    out->pipe = 0;
    out->smem = sm;
    return true;
}

// A pipelined two-step candidate of height TR with `threads` per CTA: grid =
// resident CTAs (or fewer tiles), each walking ceil(tiles / grid) tiles of
// the same per-tile work as tiled2_cand with the loads of all but its first
// tile overlapped.
static bool pipe_cand(const teuk_ctx *c, int TR, int threads, int nsm, TileCand *out)
{
    const int N = (int)c->d.Ntheta;
    const bool f32 = c->d.precision == TEUK_FP32;
    if (((size_t)N * (f32 ? sizeof(float2) : sizeof(double2))) % 16 != 0) return false;   // rows move by TMA
    size_t sm = f32 ? pipe_smem_bytes<float>(TR, N) : pipe_smem_bytes<double>(TR, N);
    if (sm > 227 * 1024) return false;
    int k = f32 ? pipe_blocks_per_sm<float>(N, threads, sm) : pipe_blocks_per_sm<double>(N, threads, sm);
    if (k < 1) return false;
    const long long Nr = c->d.Nr;
    long long tiles = (Nr + TR - 1) / TR;
    long long grid = tiles < (long long)k * nsm ? tiles : (long long)k * nsm;
    long long per = (tiles + grid - 1) / grid;
    int rpp = threads / implicit_group(N);
    auto rpad = [&](int r) { return ((r + rpp - 1) / rpp) * rpp; };
    double rows = (0.6 * (rpad(TR + 4) + rpad(TR + 2)) + 0.4 * (2.0 * TR + 6.0)) * 256.0 / threads + 1.0;
    const int warps = k * threads / 32;
    out->cost = 0.5 * (double)per * k * rows * (warps < 16 ? 1.2 : 1.0) + 2.0;
    out->R = TR + 2;
    out->persist = 0;
    out->nc = threads;
    out->grid = (int)grid;
    out->ks = 2;
    out->pipe = 1;
    out->smem = sm;
    return true;
}

// A persistent-kernel candidate of height TR with nc consumer threads.
static bool persist_cand(const teuk_ctx *c, int TR, int nc, int nsm, TileCand *out)
{
    const int N = (int)c->d.Ntheta;
    const bool f32 = c->d.precision == TEUK_FP32;
    const bool ok = f32 ? persist_available<float>(N, nc) : persist_available<double>(N, nc);
    if (!ok) return false;
    if (((size_t)N * (f32 ? sizeof(float2) : sizeof(double2))) % 16 != 0) return false;   // rows move by TMA
    const int R = TR + 2;
    size_t sm = f32 ? persist_smem_bytes<float>(TR, N) : persist_smem_bytes<double>(TR, N);
    if (sm > 227 * 1024) return false;
    int k = f32 ? persist_blocks_per_sm<float>(N, nc, sm) : persist_blocks_per_sm<double>(N, nc, sm);
    if (k < 1) return false;
    const long long Nr = c->d.Nr;
    long long tiles = (Nr + TR - 1) / TR;
    long long grid = tiles < (long long)k * nsm ? tiles : (long long)k * nsm;
    long long per = (tiles + grid - 1) / grid;
    int rpp = nc / implicit_group(N);
    int rpad = ((R + rpp - 1) / rpp) * rpp;
    double rows = (0.6 * rpad + 0.4 * R) * 256.0 / nc + 2.0;
    out->cost = 2.0 * (double)per * k * rows + 4.0;
    out->R = R;
    out->persist = 1;
    out->nc = nc;
    out->grid = (int)grid;
    out->ks = 1;
    out->pipe = 0;
    out->smem = sm;
    return true;
}

// All launch configurations that fit, best model cost first.
int tile_candidates(teuk_ctx *c, TileCand *out, int maxn)
{
    const int nsm = sm_count();
    const long long Nr = c->d.Nr;
    int n = 0;
    // one-row tiles are the only ones that fit for the widest FP64 rows
    for (int TR = 1; TR <= kMaxTileRows && n < maxn; ++TR) {
        if (tiled_cand(c, TR, nsm, &out[n])) ++n;
        if (n < maxn && c->d.scheme == TEUK_SCHEME_SPLIT && tiled2_cand(c, TR, nsm, &out[n])) ++n;
        for (int th : {256, 512})
            if (n < maxn && c->d.scheme == TEUK_SCHEME_SPLIT && pipe_cand(c, TR, th, nsm, &out[n])) ++n;
        for (int nc : {384, 480})
            if (n < maxn && persist_cand(c, TR, nc, nsm, &out[n])) ++n;
        if (TR >= Nr) break;
    }
    // insertion sort by cost
    for (int a = 1; a < n; ++a)
        for (int b = a; b > 0 && out[b].cost < out[b - 1].cost; --b) {
            TileCand t = out[b];
            out[b] = out[b - 1];
            out[b - 1] = t;
        }
    return n;
}

// Make candidate k the launch configuration.  The tiled kernel at the same
// height must fit too: it applies C_{dt/2} for the state output.
static bool apply_cand(teuk_ctx *c, const TileCand &k)
{
    const int TR = k.R - 2;
    TileCand t;
    if (!tiled_cand(c, TR, sm_count(), &t)) return false;
    c->tile_rows = TR;
    c->threads = 256;
    c->smem = t.smem;
    c->persist = k.persist;
    c->pipe = k.pipe;
    c->nc = (k.persist || k.pipe) ? k.nc : 0;
    c->grid = (k.persist || k.pipe) ? k.grid : 0;
    c->persist_smem = k.persist ? k.smem : 0;
    c->ks = k.persist ? 1 : k.ks;
    c->smem2 = (!k.persist && k.ks >= 2) ? k.smem : 0;
    return true;
}

int choose_tiles(teuk_ctx *c)
{
    std::vector<TileCand> cand(1024);
    int n = tile_candidates(c, cand.data(), (int)cand.size());
    for (int k = 0; k < n; ++k)
        if (apply_cand(c, cand[k])) return TEUK_OK;
    return set_err(c, TEUK_E_CUDA, "no tile of the split kernel fits on this device");
}

template <typename T>
StepParams<T> make_params(const teuk_ctx *c, int in_level)
{
    typedef typename V2<T>::t c2;
    StepParams<T> p;
    const teuk_grid_desc &d = c->d;
    p.Nr = (int)d.Nr;
    p.Nth = (int)d.Ntheta;
    p.tile_rows = c->tile_rows;
    p.pitch = (int)d.Ntheta;
    p.bulk = ((size_t)d.Ntheta * sizeof(c2)) % 16 == 0 ? 1 : 0;
    p.group = implicit_group((int)d.Ntheta);
    {
        const int seg = implicit_seg((int)d.Ntheta);
        p.vec = (d.Ntheta % seg == 0 && d.Ntheta % 4 == 0) ? 1 : 0;
    }
    p.first = c->shifted ? 0 : 1;
    p.imp_only = 0;
    p.i_ext = c->i_ext;
    p.wave_cap = (int)c->cap;
    p.patch_p0 = c->patch_p0;
    p.patch_np = c->patch_np;
    p.wait0 = c->wait0;
    p.dt = (T)c->dt;
    p.half_dt = (T)(0.5 * c->dt);
    p.drs_inv = (T)(1.0 / c->drs);
    for (int k = 0; k < 2; ++k) {
        double h = k ? 0.5 * c->dt : c->dt, gh = kGamma * h;
        ImpConst<T> &K = k ? p.half : p.full;
        K.gh = (T)gh;
        K.gh2 = (T)(gh * gh);
        K.h1g = (T)((1.0 - kGamma) * h);
        K.h12g = (T)((1.0 - 2.0 * kGamma) * h);
        K.h = (T)h;
        K.g2h1 = (T)(2.0 * gh * (1.0 - kGamma) * h);
        K.piv = (const c2 *)(c->coef + (k ? c->L.pivh : c->L.piv));
        K.plan = (const int *)(c->coef + (k ? c->L.planh : c->L.plan));
        K.seg = (const c2 *)(c->coef + (k ? c->L.segh : c->L.seg));
    }
    p.dt64 = c->dt;
    p.mOmega = c->mOmega;
    p.rtab = (const T *)(c->coef + c->L.rtabT);
    p.stab = (const T *)(c->coef + c->L.stab);
    p.dstab = (const T *)(c->coef + c->L.dstab);
    p.m_dOmega_da = c->m_dOmega_da;
    p.mat_on = c->L.mat_bytes > 0 ? 1 : 0;
    {
        const size_t pl = (size_t)d.Nr * (size_t)d.Ntheta;   // elements per plane
        const char *m = c->coef + c->L.mat;
        p.mat.fk = (const c2 *)m;
        p.mat.dg = (const c2 *)(m + 2 * pl * sizeof(T));
        p.mat.ct = (const c2 *)(m + 4 * pl * sizeof(T));
        p.mat.sub = (const T *)(m + 6 * pl * sizeof(T));
        p.mat.qam = (const T *)(m + 7 * pl * sizeof(T));
        p.mat.qap = (const T *)(m + 8 * pl * sizeof(T));
        p.mat.lw = (const T *)(m + ((9 * pl * sizeof(T) + 255) & ~(size_t)255));
    }
    p.thtab = (const T *)(c->coef + c->L.thT);
    p.patch = (const c2 *)(c->coef + c->L.patch);
    p.nfix = -1;
    p.h_out = nullptr;
    p.tape = nullptr;
    p.patchu = (const c2 *)(c->coef + c->L.patchu);
    p.unit_p0 = c->unit_p0;
    p.unit_np = c->unit_np;
    p.amp_re = c->amp_re;
    p.amp_im = c->amp_im;
    p.rs_min64 = d.rstar_min;
    p.drs64 = c->drs;
    p.rs0 = c->rs0;
    p.inv_sig_r2 = c->sig_r > 0.0 ? 1.0 / (c->sig_r * c->sig_r) : 0.0;
    p.drs0_dr0 = c->drs0_dr0;
    p.m_dOmega = c->m_dOmega;
    p.w = (const double *)(c->coef + c->L.w);
    p.uin = (const c2 *)(c->state + (size_t)in_level * c->level_bytes);
    p.uout = (c2 *)(c->state + (size_t)(1 - in_level) * c->level_bytes);
    p.mid = (c2 *)(c->coef + c->L.scratch);
    p.wave = c->wave;
    p.ctl = (Ctl *)(c->coef + c->L.ctl);
    return p;
}

template <typename T>
cudaError_t launch_split(const teuk_ctx *c, const StepParams<T> &p, cudaStream_t st)
{
    if (c->persist) return launch_split_persist<T>(p, c->nc, c->grid, c->persist_smem, st);
    return launch_split_step<T>(p, c->threads, c->smem, st);
}

// Scan levels of the implicit solves of every row, for the steps dt and
// dt/2 (split scheme): computed once from the coefficients and pivots, read
// by every step kernel.
cudaError_t compute_plans(teuk_ctx *c, cudaStream_t st)
{
    if (c->d.scheme != TEUK_SCHEME_SPLIT) return cudaSuccess;
    int *pf = (int *)(c->coef + c->L.plan), *ph = (int *)(c->coef + c->L.planh);
    char *sf = c->coef + c->L.seg, *sh = c->coef + c->L.segh;
    if (c->d.precision == TEUK_FP32)
        return launch_scan_plans<float>(make_params<float>(c, 0), pf, ph, (float2 *)sf, (float2 *)sh, st);
    const StepParams<double> p = make_params<double>(c, 0);
    cudaError_t e = launch_scan_plans<double>(p, pf, ph, (double2 *)sf, (double2 *)sh, st);
    if (e != cudaSuccess) return e;
    // the FP64 path's materialised coefficients come from the same tables
    return launch_mat_coef<double>(p, st);
}

cudaError_t launch_one(teuk_ctx *c, int in_level, cudaStream_t st)
{
    if (c->d.precision == TEUK_FP32) {
        StepParams<float> p = make_params<float>(c, in_level);
        return c->d.scheme == TEUK_SCHEME_SPLIT ? launch_split<float>(c, p, st) : launch_literal_step<float>(p, st);
    }
    StepParams<double> p = make_params<double>(c, in_level);
    return c->d.scheme == TEUK_SCHEME_SPLIT ? launch_split<double>(c, p, st) : launch_literal_step<double>(p, st);
}

// One launch of the configured kernel from level in_level: two or three
// steps when the tiled kernel takes that many per launch and the state is
// shifted (full steps follow), else one; *steps receives the count.
cudaError_t launch_unit(teuk_ctx *c, int in_level, cudaStream_t st, int *steps)
{
    if (c->d.scheme == TEUK_SCHEME_SPLIT && c->ks == 3 && c->shifted) {
        *steps = 3;
        if (c->d.precision == TEUK_FP32)
            return launch_split_step3<float>(make_params<float>(c, in_level), c->threads, c->smem2, st);
        return launch_split_step3<double>(make_params<double>(c, in_level), c->threads, c->smem2, st);
    }
    if (c->d.scheme == TEUK_SCHEME_SPLIT && c->ks == 2 && c->shifted) {
        *steps = 2;
        if (c->d.precision == TEUK_FP32) {
            StepParams<float> p = make_params<float>(c, in_level);
            return c->pipe ? launch_split_pipe<float>(p, c->nc, c->grid, c->smem2, st)
                           : launch_split_step2<float>(p, c->threads, c->smem2, st);
        }
        StepParams<double> p = make_params<double>(c, in_level);
        return c->pipe ? launch_split_pipe<double>(p, c->nc, c->grid, c->smem2, st)
                       : launch_split_step2<double>(p, c->threads, c->smem2, st);
    }
    *steps = 1;
    return launch_one(c, in_level, st);
}

// Physical state u_n = C_{dt/2} s_n of a shifted split-scheme state, written
// to the other level (which the next step overwrites anyway).
cudaError_t physical_to_other(teuk_ctx *c, cudaStream_t st)
{
    if (c->d.precision == TEUK_FP32) {
        StepParams<float> p = make_params<float>(c, c->cur);
        p.imp_only = 1;
        return launch_split_step<float>(p, c->threads, c->smem, st);
    }
    StepParams<double> p = make_params<double>(c, c->cur);
    p.imp_only = 1;
    return launch_split_step<double>(p, c->threads, c->smem, st);
}

cudaError_t extract_current(teuk_ctx *c, cudaStream_t st)
{
    if (c->d.precision == TEUK_FP32) {
        StepParams<float> p = make_params<float>(c, c->cur);
        return launch_extract<float>(p, p.uin, c->step, st);
    }
    StepParams<double> p = make_params<double>(c, c->cur);
    return launch_extract<double>(p, p.uin, c->step, st);
}

void drop_graphs(teuk_ctx *c)
{
    for (int k = 0; k < 2; ++k) {
        if (c->graph[k]) cudaGraphExecDestroy(c->graph[k]);
        c->graph[k] = nullptr;
        c->graph_stream[k] = nullptr;
    }
}

// Back to a clean state: zero field at step 0, empty ring buffer, cleared
// flags (the source and weights are kept).
int reset_state(teuk_ctx *c, cudaStream_t st)
{
    CK(cudaMemsetAsync(c->state, 0, 2 * c->level_bytes, st), "zero state");
    CK(cudaMemsetAsync(c->wave, 0, sizeof(double2) * (size_t)(c->d.Ntheta + 1) * (size_t)c->cap, st), "zero wave");
    CK(launch_set_ctl(c->coef, c->L, 0, 1, st), "control block");
    c->cur = 0;
    c->shifted = 0;
    c->step = 0;
    c->rec_lo = 0;
    CK(extract_current(c, st), "extract");
    return TEUK_OK;
}

}  // namespace

extern "C" {

const char *teuk_status_string(int s)
{
    switch (s) {
    case TEUK_OK: return "TEUK_OK";
    case TEUK_E_INVAL: return "TEUK_E_INVAL";
    case TEUK_E_CUDA: return "TEUK_E_CUDA";
    case TEUK_E_NONFINITE: return "TEUK_E_NONFINITE";
    case TEUK_E_UNSTABLE: return "TEUK_E_UNSTABLE";
    case TEUK_E_TIMEOUT: return "TEUK_E_TIMEOUT";
    case TEUK_E_STATE: return "TEUK_E_STATE";
    case TEUK_E_RANGE: return "TEUK_E_RANGE";
    default: return "unknown status";
    }
}

const char *teuk_last_error(const teuk_ctx *c) { return c ? c->err : g_init_err; }

int64_t teuk_current_step(const teuk_ctx *c) { return c ? c->step : -1; }

int teuk_workspace_bytes(const teuk_grid_desc *d, size_t *state_bytes, size_t *coef_bytes,
                         size_t *wave_bytes_per_step)
{
    int rc = validate(d, g_init_err);
    if (rc) return rc;
    size_t c2 = d->precision == TEUK_FP32 ? sizeof(float2) : sizeof(double2);
    if (state_bytes) *state_bytes = 2 * align256(c2 * 2 * (size_t)d->Nr * (size_t)d->Ntheta);
    if (coef_bytes) *coef_bytes = make_layout(*d).total;
    if (wave_bytes_per_step) *wave_bytes_per_step = sizeof(double2) * (size_t)(d->Ntheta + 1);
    return TEUK_OK;
}

int teuk_init_grid(const teuk_grid_desc *desc, void *d_state, void *d_coef, void *d_wave,
                   int64_t wave_capacity, void *stream, teuk_ctx **out)
{
    teuk_ctx *c = nullptr;
    if (!out) return set_err(c, TEUK_E_INVAL, "out is NULL");
    *out = nullptr;
    int rc = validate(desc, g_init_err);
    if (rc) return rc;
    if (!d_state || !d_coef || !d_wave) return set_err(c, TEUK_E_INVAL, "device buffers must not be NULL");
    if (((uintptr_t)d_state | (uintptr_t)d_coef | (uintptr_t)d_wave) & 255)
        return set_err(c, TEUK_E_INVAL, "device buffers must be 256-byte aligned");
    if (wave_capacity < 1 || wave_capacity > (1LL << 31)) return set_err(c, TEUK_E_INVAL, "wave_capacity out of range");

    teuk_grid_desc d = *desc;
    double drs = (d.rstar_max - d.rstar_min) / (double)(d.Nr - 1);
    double dt = d.dt > 0.0 ? d.dt : 0.5 * drs;
    d.dt = dt;

    // stability guards
    double bmax, qmax, ctmax;
    host_bounds(d, &bmax, &qmax, &ctmax);
    if (bmax * dt / drs > 1.0)
        return set_err(c, TEUK_E_UNSTABLE, "radial Courant number %.4f > 1", bmax * dt / drs);
    if (d.scheme == TEUK_SCHEME_LITERAL && !d.allow_unstable) {
        double z = fmax(sqrt(qmax * host_atheta_bound(d)) * dt, ctmax * dt);
        if (z > 0.05)
            return set_err(c, TEUK_E_UNSTABLE,
                           "literal scheme: explicit S has |lambda dt| = %.3g > 0.05 (grows each step); "
                           "use TEUK_SCHEME_SPLIT or set allow_unstable", z);
    }

    c = new (std::nothrow) teuk_ctx();
    if (!c) return set_err(nullptr, TEUK_E_INVAL, "out of host memory");
    memset(c, 0, sizeof(*c));
    c->wait0 = -1;   // default bound of the tile-copy waits
    c->d = d;
    c->drs = drs;
    c->dt = dt;
    long long ie = llround((d.rstar_extract - d.rstar_min) / drs);
    if (ie < 0) ie = 0;
    if (ie > d.Nr - 1) ie = d.Nr - 1;
    c->i_ext = (int)ie;
    c->state = (char *)d_state;
    c->coef = (char *)d_coef;
    c->wave = (double2 *)d_wave;
    c->cap = wave_capacity;
    c->L = make_layout(d);
    size_t c2 = d.precision == TEUK_FP32 ? sizeof(float2) : sizeof(double2);
    c->level_bytes = align256(c2 * 2 * (size_t)d.Nr * (size_t)d.Ntheta);
    c->cur = 0;
    c->step = 0;
    c->rec_lo = 0;
    c->patch_p0 = 0;
    c->patch_np = 0;
    c->mOmega = 0.0;
    if (d.scheme == TEUK_SCHEME_SPLIT) {
        int rt = choose_tiles(c);
        if (rt != TEUK_OK) {
            memcpy(g_init_err, c->err, sizeof(g_init_err));
            delete c;
            return rt;
        }
    } else {
        c->tile_rows = 1;
        c->threads = 256;
        c->smem = 0;
    }

    cudaStream_t st = (cudaStream_t)stream;
    int r2 = TEUK_OK;
    do {
        cudaError_t e;
        if ((e = cudaMemsetAsync(c->state, 0, 2 * c->level_bytes, st)) != cudaSuccess) { r2 = cuda_err(c, e, "zero state"); break; }
        if ((e = cudaMemsetAsync(c->coef, 0, c->L.total, st)) != cudaSuccess) { r2 = cuda_err(c, e, "zero coef"); break; }
        if ((e = cudaMemsetAsync(c->wave, 0, sizeof(double2) * (size_t)(d.Ntheta + 1) * (size_t)wave_capacity, st)) != cudaSuccess) { r2 = cuda_err(c, e, "zero wave"); break; }
        if ((e = launch_coef_tables(d, drs, dt, c->coef, c->L, st)) != cudaSuccess) { r2 = cuda_err(c, e, "coefficient kernels"); break; }
        if ((e = compute_plans(c, st)) != cudaSuccess) { r2 = cuda_err(c, e, "scan plans"); break; }
        if ((e = launch_set_ctl(c->coef, c->L, 0, 1, st)) != cudaSuccess) { r2 = cuda_err(c, e, "control block"); break; }
        if ((e = extract_current(c, st)) != cudaSuccess) { r2 = cuda_err(c, e, "extract"); break; }
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { r2 = cuda_err(c, e, "init sync"); break; }
    } while (0);
    if (r2 != TEUK_OK) {
        memcpy(g_init_err, c->err, sizeof(g_init_err));
        delete c;
        return r2;
    }
    *out = c;
    return TEUK_OK;
}

int teuk_set_source(teuk_ctx *c, double amp_re, double amp_im, double r0, double sigma_rstar,
                    double sigma_theta, double Omega)
{
    if (!c) return TEUK_E_STATE;
    const teuk_grid_desc &d = c->d;
    if (!isfinite(amp_re) || !isfinite(amp_im)) return set_err(c, TEUK_E_INVAL, "amplitude must be finite");
    drop_graphs(c);
    // steps still in flight on any stream read the source tables
    CK(cudaDeviceSynchronize(), "source sync");
    const bool off = amp_re == 0.0 && amp_im == 0.0;
    double rp = d.M + sqrt(d.M * d.M - d.a * d.a);
    const bool orbit_ok = r0 > rp && isfinite(r0) && sigma_rstar > 0.0 && sigma_theta > 0.0;
    if (off && !orbit_ok) {
        CK(launch_src_fields(d, c->drs, c->coef, c->L, 0, 0, 0.0, 0.0, 0.0, 1.0, 1.0, 0.0, 0), "source factors");
        CK(cudaStreamSynchronize(0), "source sync");
        c->patch_np = 0;
        c->unit_np = 0;
        c->mOmega = 0.0;
        c->amp_re = c->amp_im = 0.0;
        return TEUK_OK;
    }
    if (!(r0 > rp) || !isfinite(r0)) return set_err(c, TEUK_E_INVAL, "orbit radius must exceed r_+");
    if (!(sigma_rstar > 0.0) || !(sigma_theta > 0.0)) return set_err(c, TEUK_E_INVAL, "source widths must be positive");
    const bool kepler = isnan(Omega);
    double Om = kepler ? sqrt(d.M) / (pow(r0, 1.5) + d.a * sqrt(d.M)) : Omega;
    if (!isfinite(Om)) return set_err(c, TEUK_E_INVAL, "Omega must be finite or NaN");
    double rs0 = host_rstar(d.M, d.a, r0);
    double lo = (rs0 - 9.0 * sigma_rstar - d.rstar_min) / c->drs;
    double hi = (rs0 + 9.0 * sigma_rstar - d.rstar_min) / c->drs;
    long long p0 = (long long)floor(lo) - 1, p1 = (long long)ceil(hi) + 1;
    if (p0 < 0) p0 = 0;
    if (p1 > d.Nr - 1) p1 = d.Nr - 1;
    int np = (int)(p1 - p0 + 1);
    if (p1 < p0) np = 0;
    long long cap_rows = d.Nr < TEUK_MAX_PATCH_ROWS ? d.Nr : TEUK_MAX_PATCH_ROWS;
    if (np > cap_rows) return set_err(c, TEUK_E_INVAL, "source patch needs more rows than TEUK_MAX_PATCH_ROWS");
    cudaStream_t st = 0;
    if (np > 0)
        CK(launch_patch(d, c->drs, c->coef, c->L, (int)p0, np, amp_re, amp_im, rs0, sigma_rstar, sigma_theta, st), "source patch");
    // the factored form the forward step kernels use (zero when the amplitude is)
    // r0* moves with the spin: d r0*/d a at fixed r0 (Eq. 2)
    const double drs0_da = host_drstar_da(d.M, d.a, r0 - rp);
    CK(launch_src_fields(d, c->drs, c->coef, c->L, (int)p0, off ? 0 : np, amp_re, amp_im, rs0, sigma_rstar,
                         sigma_theta, drs0_da, st), "source factors");
    CK(cudaStreamSynchronize(st), "source sync");
    c->patch_p0 = (int)p0;
    c->patch_np = off ? 0 : np;
    c->unit_p0 = (int)p0;
    c->unit_np = np;
    c->mOmega = (double)d.m * Om;
    c->amp_re = amp_re;
    c->amp_im = amp_im;
    c->rs0 = rs0;
    c->sig_r = sigma_rstar;
    // d r0*/d r0 = (r0^2 + a^2)/Delta(r0); with the Kepler frequency
    // Omega = M^(1/2)/(r0^(3/2) + a M^(1/2)), dOmega/dr0 = -(3/2) r0^(1/2) Omega^2 / M^(1/2)
    const double Delta0 = r0 * r0 - 2.0 * d.M * r0 + d.a * d.a;
    c->drs0_dr0 = (r0 * r0 + d.a * d.a) / Delta0;
    c->m_dOmega = kepler ? (double)d.m * (-1.5 * sqrt(r0) * Om * Om / sqrt(d.M)) : 0.0;
    // and dOmega/da = -M / (r0^(3/2) + a M^(1/2))^2 = -Omega^2 for the Kepler frequency
    c->m_dOmega_da = kepler ? (double)d.m * (-Om * Om) : 0.0;
    return TEUK_OK;
}

int teuk_set_weights(teuk_ctx *c, const double *w)
{
    if (!c) return TEUK_E_STATE;
    double *dw = (double *)(c->coef + c->L.w);
    if (w)
        for (int64_t j = 0; j < c->d.Ntheta; ++j)
            if (!isfinite(w[j])) return set_err(c, TEUK_E_INVAL, "weights must be finite");
    // steps still in flight on any stream read the weights (fused extraction):
    // let them finish before the weights change
    CK(cudaDeviceSynchronize(), "weights sync");
    if (w) {
        CK(cudaMemcpy(dw, w, sizeof(double) * (size_t)c->d.Ntheta, cudaMemcpyHostToDevice), "weights copy");
    } else {
        CK(launch_coef_tables(c->d, c->drs, c->dt, c->coef, c->L, 0), "default weights");
        CK(compute_plans(c, 0), "scan plans");
        CK(cudaDeviceSynchronize(), "weights sync");
    }
    return TEUK_OK;
}

int teuk_set_state(teuk_ctx *c, const void *src, int64_t step, void *stream)
{
    if (!c) return TEUK_E_STATE;
    if (!src || step < 0) return set_err(c, TEUK_E_INVAL, "src must not be NULL and step >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    size_t n = 2 * (size_t)c->d.Nr * (size_t)c->d.Ntheta;   // complex elements
    char *dst = c->state + (size_t)c->cur * c->level_bytes;
    cudaPointerAttributes at;
    bool dev = cudaPointerGetAttributes(&at, src) == cudaSuccess &&
               (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (c->d.precision == TEUK_FP64) {
        CK(cudaMemcpyAsync(dst, src, n * sizeof(double2), cudaMemcpyDefault, st), "state copy");
    } else if (dev) {
        CK(launch_convert_to(TEUK_FP32, (const double2 *)src, dst, n, st), "state convert");
    } else {
        double2 *stg = (double2 *)(c->coef + c->L.staging);
        for (size_t o = 0; o < n; o += c->L.staging_elems) {
            size_t k = n - o < c->L.staging_elems ? n - o : c->L.staging_elems;
            CK(cudaMemcpyAsync(stg, (const double2 *)src + o, k * sizeof(double2), cudaMemcpyHostToDevice, st), "state upload");
            CK(launch_convert_to(TEUK_FP32, stg, (float2 *)dst + o, k, st), "state convert");
        }
    }
    CK(launch_set_ctl(c->coef, c->L, step, 1, st), "control block");
    c->step = step;
    c->rec_lo = step;
    c->shifted = 0;
    CK(extract_current(c, st), "extract");
    if (!dev) CK(cudaStreamSynchronize(st), "state sync");
    return TEUK_OK;
}

int teuk_get_state(teuk_ctx *c, void *dst, int64_t *step, void *stream)
{
    if (!c) return TEUK_E_STATE;
    if (!dst) return set_err(c, TEUK_E_INVAL, "dst must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    size_t n = 2 * (size_t)c->d.Nr * (size_t)c->d.Ntheta;
    const char *src = c->state + (size_t)c->cur * c->level_bytes;
    if (c->d.scheme == TEUK_SCHEME_SPLIT && c->shifted) {
        CK(physical_to_other(c, st), "physical state");
        src = c->state + (size_t)(1 - c->cur) * c->level_bytes;
    }
    cudaPointerAttributes at;
    bool dev = cudaPointerGetAttributes(&at, dst) == cudaSuccess &&
               (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (c->d.precision == TEUK_FP64) {
        CK(cudaMemcpyAsync(dst, src, n * sizeof(double2), cudaMemcpyDefault, st), "state copy");
    } else if (dev) {
        CK(launch_convert_from(TEUK_FP32, src, (double2 *)dst, n, st), "state convert");
    } else {
        double2 *stg = (double2 *)(c->coef + c->L.staging);
        for (size_t o = 0; o < n; o += c->L.staging_elems) {
            size_t k = n - o < c->L.staging_elems ? n - o : c->L.staging_elems;
            CK(launch_convert_from(TEUK_FP32, (const float2 *)src + o, stg, k, st), "state convert");
            CK(cudaMemcpyAsync((double2 *)dst + o, stg, k * sizeof(double2), cudaMemcpyDeviceToHost, st), "state download");
        }
    }
    CK(cudaStreamSynchronize(st), "state sync");
    if (step) *step = c->step;
    return TEUK_OK;
}

int teuk_state_level(const teuk_ctx *c, int64_t *offset_bytes, size_t *level_bytes, int *shifted)
{
    if (!c) return TEUK_E_STATE;
    if (offset_bytes) *offset_bytes = (int64_t)c->cur * (int64_t)c->level_bytes;
    if (level_bytes) *level_bytes = c->level_bytes;
    if (shifted) *shifted = (c->d.scheme == TEUK_SCHEME_SPLIT && c->shifted) ? 1 : 0;
    return TEUK_OK;
}

int teuk_step(teuk_ctx *c, int64_t nsteps, void *stream)
{
    if (!c) return TEUK_E_STATE;
    if (nsteps < 0) return set_err(c, TEUK_E_INVAL, "nsteps must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    int64_t left = nsteps;
    if (left > 0 && c->d.scheme == TEUK_SCHEME_SPLIT && !c->shifted) {
        // first step from a physical state: s_{n+1} = LW C_{dt/2} u_n
        CK(launch_one(c, c->cur, st), "first step launch");
        c->cur ^= 1;
        c->shifted = 1;
        left -= 1;
    }
    // steps per launch from here on (the state is shifted)
    const int ks = (c->d.scheme == TEUK_SCHEME_SPLIT && c->ks >= 2) ? c->ks : 1;
    // steps per captured graph: a multiple of ks over an even number of launches
    const int chunk = ks == 3 ? 3 * kGraphChunk / 2 : kGraphChunk;
    bool use_graph = st != nullptr && c->d.scheme == TEUK_SCHEME_SPLIT && left >= 2 * chunk;
    if (use_graph) {
        int g = c->cur;
        if (c->graph[g] && c->graph_stream[g] != st) {
            cudaGraphExecDestroy(c->graph[g]);
            c->graph[g] = nullptr;
        }
        if (!c->graph[g]) {
            cudaGraph_t graph;
            CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
            int lev = g, done = 0;
            cudaError_t le = cudaSuccess;
            while (done < chunk && le == cudaSuccess) {
                int k = 0;
                le = launch_unit(c, lev, st, &k);
                done += k;
                lev ^= 1;
            }
            cudaError_t ee = cudaStreamEndCapture(st, &graph);
            if (le != cudaSuccess) return cuda_err(c, le, "captured launch");
            if (ee != cudaSuccess) return cuda_err(c, ee, "end capture");
            cudaError_t ie = cudaGraphInstantiate(&c->graph[g], graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) {
                c->graph[g] = nullptr;
                return cuda_err(c, ie, "graph instantiate");
            }
            c->graph_stream[g] = st;
        }
        while (left >= chunk) {
            CK(cudaGraphLaunch(c->graph[g], st), "graph launch");
            left -= chunk;
        }
    }
    while (left >= ks) {
        int k = 0;
        CK(launch_unit(c, c->cur, st, &k), "step launch");
        c->cur ^= 1;
        left -= k;
    }
    while (left > 0) {
        CK(launch_one(c, c->cur, st), "step launch");
        c->cur ^= 1;
        left -= 1;
    }
    c->step += nsteps;
    return TEUK_OK;
}

int teuk_extract_waveform(teuk_ctx *c, int64_t first, int64_t count, double *h_out, double *row_out,
                          void *stream)
{
    if (!c) return TEUK_E_STATE;
    if (count < 0 || (count > 0 && !h_out)) return set_err(c, TEUK_E_INVAL, "need count >= 0 and h_out");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaStreamSynchronize(st), "sync");
    int64_t lo = c->rec_lo > c->step - c->cap + 1 ? c->rec_lo : c->step - c->cap + 1;
    if (count > 0 && (first < lo || first + count - 1 > c->step))
        return set_err(c, TEUK_E_RANGE, "steps not in the ring buffer");
    size_t slot_bytes = sizeof(double2) * (size_t)(c->d.Ntheta + 1);
    int64_t done = 0;
    while (done < count) {
        int64_t s = first + done;
        int64_t slot = s % c->cap;
        int64_t run = c->cap - slot;
        if (run > count - done) run = count - done;
        const char *base = (const char *)c->wave + (size_t)slot * slot_bytes;
        CK(cudaMemcpy2D(h_out + 2 * done, sizeof(double2), base, slot_bytes, sizeof(double2), (size_t)run,
                        cudaMemcpyDeviceToHost), "waveform copy");
        if (row_out)
            CK(cudaMemcpy2D(row_out + 2 * c->d.Ntheta * done, sizeof(double2) * (size_t)c->d.Ntheta,
                            base + sizeof(double2), slot_bytes, sizeof(double2) * (size_t)c->d.Ntheta,
                            (size_t)run, cudaMemcpyDeviceToHost), "row copy");
        done += run;
    }
    Ctl h;
    CK(cudaMemcpy(&h, c->coef + c->L.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost), "control read");
    if (h.flags & FLAG_TIMEOUT) return set_err(c, TEUK_E_TIMEOUT, "a bulk copy of a state tile did not complete");
    if (h.flags & FLAG_NONFINITE) return set_err(c, TEUK_E_NONFINITE, "a non-finite waveform sample was produced");
    return TEUK_OK;
}

int teuk_destroy(teuk_ctx *c)
{
    if (!c) return TEUK_OK;
    drop_graphs(c);
    delete c;
    return TEUK_OK;
}

int teuk_tiling(const teuk_ctx *c, int *tile_rows, int *threads, size_t *smem_bytes, int *group)
{
    if (!c) return TEUK_E_STATE;
    if (tile_rows) *tile_rows = c->tile_rows;
    if (threads) *threads = c->persist ? c->nc + 32 : c->threads;
    if (smem_bytes) *smem_bytes = c->persist ? c->persist_smem : c->smem;
    if (group) *group = implicit_group((int)c->d.Ntheta);
    return TEUK_OK;
}

int teuk_kernel_config(const teuk_ctx *c, int *persistent, int *consumer_threads, int *grid, int *steps_per_launch)
{
    if (!c) return TEUK_E_STATE;
    if (persistent) *persistent = c->persist ? 1 : (c->pipe ? 2 : 0);
    if (consumer_threads) *consumer_threads = (c->persist || c->pipe) ? c->nc : c->threads;
    if (grid) *grid = (c->persist || c->pipe) ? c->grid : (int)((c->d.Nr + c->tile_rows - 1) / c->tile_rows);
    if (steps_per_launch) *steps_per_launch = c->d.scheme == TEUK_SCHEME_SPLIT ? c->ks : 1;
    return TEUK_OK;
}

// Times the best few launch configurations of each kernel and keeps the
// fastest.  With a flush buffer every timed step starts from a cold L2 (the
// buffer is overwritten between steps, outside the timed interval).
static int autotune_impl(teuk_ctx *c, int trial_steps, void *flush, size_t flush_bytes, cudaStream_t st,
                         int *tile_rows_out)
{
    if (trial_steps < 1 || trial_steps > 100000) return set_err(c, TEUK_E_INVAL, "trial_steps out of range");
    if (c->d.scheme != TEUK_SCHEME_SPLIT) {
        if (tile_rows_out) *tile_rows_out = c->tile_rows;
        return TEUK_OK;
    }
    std::vector<TileCand> all(1024);
    int n = tile_candidates(c, all.data(), (int)all.size());
    // the best few of each kernel by the model
    std::vector<TileCand> cand;
    for (int kind = 0; kind < 4; ++kind) {   // tiled, tiled two steps per launch, persistent, pipelined
        int taken = 0;
        for (int k = 0; k < n && taken < 4; ++k) {
            const int kk = all[k].pipe ? 3 : (all[k].persist ? 2 : (all[k].ks == 2 ? 1 : 0));
            if (kk == kind) {
                cand.push_back(all[k]);
                ++taken;
            }
        }
    }
    // three steps per launch at the heights of the two-step candidates
    {
        const size_t n2 = cand.size();
        for (size_t k = 0; k < n2; ++k) {
            TileCand t3;
            if (cand[k].ks == 2 && !cand[k].pipe && tiled3_cand(c, cand[k].R - 2, sm_count(), &t3)) cand.push_back(t3);
        }
    }
    if (cand.empty()) return set_err(c, TEUK_E_CUDA, "no tile of the split kernel fits on this device");
    drop_graphs(c);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    // Two interleaved rounds over the candidates; a candidate's score is its
    // better round, each round the median time per step over L2-flushed
    // single launches (cold) or the mean over back-to-back launches.
    std::vector<float> score(cand.size(), 3.4e38f), per;
    cudaError_t e = cudaSuccess;
    for (int round = 0; round < 2 && e == cudaSuccess; ++round)
        for (size_t k = 0; k < cand.size() && e == cudaSuccess; ++k) {
            if (!apply_cand(c, cand[k])) continue;
            c->shifted = 1;
            int lev = c->cur, ku = 0, steps = 0;
            for (int w = 0; w < 3 && e == cudaSuccess; ++w, lev ^= 1) e = launch_unit(c, lev, st, &ku);
            float t = 0.0f;
            if (flush) {
                per.clear();
                for (int w = 0; w < trial_steps && e == cudaSuccess; ++w, lev ^= 1) {
                    float ms = 0.0f;
                    e = cudaMemsetAsync(flush, w & 0xff, flush_bytes, st);
                    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
                    if (e == cudaSuccess) e = launch_unit(c, lev, st, &ku);
                    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                    if (e == cudaSuccess && ku > 0) per.push_back(ms / (float)ku);
                }
                if (per.empty()) continue;
                std::nth_element(per.begin(), per.begin() + per.size() / 2, per.end());
                t = per[per.size() / 2];
            } else {
                if (e == cudaSuccess) e = cudaEventRecord(e0, st);
                for (int w = 0; w < trial_steps && e == cudaSuccess; ++w, lev ^= 1) {
                    e = launch_unit(c, lev, st, &ku);
                    steps += ku;
                }
                if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
                if (steps < 1) continue;
                t /= (float)steps;   // time per step
            }
            if (e == cudaSuccess && t < score[k]) score[k] = t;
        }
    int bestk = -1;
    for (size_t k = 0; k < cand.size(); ++k)
        if (score[k] < 3.4e38f && (bestk < 0 || score[k] < score[bestk])) bestk = (int)k;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_err(c, e, "autotune trial");
    if (bestk < 0) return set_err(c, TEUK_E_CUDA, "no tile of the split kernel fits on this device");
    apply_cand(c, cand[bestk]);
    int rr = reset_state(c, st);
    if (rr != TEUK_OK) return rr;
    CK(cudaStreamSynchronize(st), "autotune sync");
    if (tile_rows_out) *tile_rows_out = c->tile_rows;
    return TEUK_OK;
}

int teuk_autotune(teuk_ctx *c, int trial_steps, void *stream, int *tile_rows_out)
{
    if (!c) return TEUK_E_STATE;
    return autotune_impl(c, trial_steps, nullptr, 0, (cudaStream_t)stream, tile_rows_out);
}

int teuk_autotune_cold(teuk_ctx *c, int trial_steps, void *d_flush, size_t flush_bytes, void *stream,
                       int *tile_rows_out)
{
    if (!c) return TEUK_E_STATE;
    if (!d_flush || flush_bytes == 0) return set_err(c, TEUK_E_INVAL, "need a device flush buffer");
    return autotune_impl(c, trial_steps, d_flush, flush_bytes, (cudaStream_t)stream, tile_rows_out);
}

int teuk_set_tiling(teuk_ctx *c, int tile_rows)
{
    if (!c) return TEUK_E_STATE;
    if (c->d.scheme != TEUK_SCHEME_SPLIT) return TEUK_OK;
    if (tile_rows < 1 || tile_rows > 254) return set_err(c, TEUK_E_INVAL, "tile_rows out of range [1, 254]");
    TileCand t;
    if (!tiled_cand(c, tile_rows, sm_count(), &t)) return set_err(c, TEUK_E_INVAL, "tile does not fit in shared memory");
    drop_graphs(c);
    apply_cand(c, t);
    return TEUK_OK;
}

int teuk_set_tiling_steps(teuk_ctx *c, int tile_rows, int steps_per_launch)
{
    if (!c) return TEUK_E_STATE;
    if (steps_per_launch == 1) return teuk_set_tiling(c, tile_rows);
    if (steps_per_launch != 2 && steps_per_launch != 3)
        return set_err(c, TEUK_E_INVAL, "steps_per_launch must be 1, 2 or 3");
    if (c->d.scheme != TEUK_SCHEME_SPLIT)
        return set_err(c, TEUK_E_INVAL, "several steps per launch need the split scheme");
    const int trmax = kMaxTileRows - 2 * steps_per_launch;
    if (tile_rows < 1 || tile_rows > trmax) return set_err(c, TEUK_E_INVAL, "tile_rows out of range [1, %d]", trmax);
    TileCand t;
    if (!(steps_per_launch == 3 ? tiled3_cand(c, tile_rows, sm_count(), &t) : tiled2_cand(c, tile_rows, sm_count(), &t)))
        return set_err(c, TEUK_E_INVAL, "tile does not fit in shared memory");
    TileCand tt;
    if (!tiled_cand(c, tile_rows, sm_count(), &tt)) return set_err(c, TEUK_E_INVAL, "tile does not fit in shared memory");
    drop_graphs(c);
    apply_cand(c, t);
    return TEUK_OK;
}

int teuk_set_pipelined(teuk_ctx *c, int tile_rows, int threads)
{
    if (!c) return TEUK_E_STATE;
    if (c->d.scheme != TEUK_SCHEME_SPLIT) return set_err(c, TEUK_E_INVAL, "the pipelined kernel is a split-scheme kernel");
    if (tile_rows < 1 || tile_rows > 250) return set_err(c, TEUK_E_INVAL, "tile_rows out of range [1, 250]");
    if (threads != 256 && threads != 512) return set_err(c, TEUK_E_INVAL, "threads must be 256 or 512");
    TileCand t;
    if (!pipe_cand(c, tile_rows, threads, sm_count(), &t))
        return set_err(c, TEUK_E_INVAL, "pipelined kernel unavailable: rows must be 16-byte multiples and two tile "
                                        "buffers must fit in shared memory");
    TileCand tt;
    if (!tiled_cand(c, tile_rows, sm_count(), &tt)) return set_err(c, TEUK_E_INVAL, "tile does not fit in shared memory");
    drop_graphs(c);
    apply_cand(c, t);
    return TEUK_OK;
}

int teuk_set_persistent(teuk_ctx *c, int tile_rows, int consumer_threads)
{
    if (!c) return TEUK_E_STATE;
    if (c->d.scheme != TEUK_SCHEME_SPLIT) return set_err(c, TEUK_E_INVAL, "the persistent kernel is a split-scheme kernel");
    if (tile_rows < 1 || tile_rows > 254) return set_err(c, TEUK_E_INVAL, "tile_rows out of range [1, 254]");
    TileCand t;
    if (!persist_cand(c, tile_rows, consumer_threads, sm_count(), &t)) {
        const int N = (int)c->d.Ntheta;
        const bool f32 = c->d.precision == TEUK_FP32;
        size_t sm = f32 ? persist_smem_bytes<float>(tile_rows, N) : persist_smem_bytes<double>(tile_rows, N);
        char why[320];
        if (f32) persist_explain<float>(N, consumer_threads, sm, why, sizeof(why));
        else persist_explain<double>(N, consumer_threads, sm, why, sizeof(why));
        return set_err(c, TEUK_E_INVAL, "persistent kernel unavailable for this grid: %s", why);
    }
    TileCand tt;
    if (!tiled_cand(c, tile_rows, sm_count(), &tt)) return set_err(c, TEUK_E_INVAL, "tile does not fit in shared memory");
    drop_graphs(c);
    apply_cand(c, t);
    return TEUK_OK;
}

int teuk_set_wait_limit(teuk_ctx *c, int rounds)
{
    if (!c) return TEUK_E_STATE;
    drop_graphs(c);   // captured launches carry the old bound
    c->wait0 = rounds < 0 ? -1 : rounds;
    return TEUK_OK;
}

int teuk_literal_step_static(const teuk_ctx *c, const void *d_in, void *d_out, int64_t n, void *stream)
{
    teuk_ctx *cm = const_cast<teuk_ctx *>(c);
    if (!c) return TEUK_E_STATE;
    if (c->d.scheme != TEUK_SCHEME_LITERAL)
        return set_err(cm, TEUK_E_INVAL, "teuk_literal_step_static needs a context of the literal scheme");
    if (!d_in || !d_out || n < 0) return set_err(cm, TEUK_E_INVAL, "need non-NULL device buffers and n >= 0");
    size_t c2 = c->d.precision == TEUK_FP32 ? sizeof(float2) : sizeof(double2);
    {
        // the node kernel writes d_out while other threads still read d_in: no byte may be shared
        const size_t bytes = c2 * 2 * (size_t)c->d.Nr * (size_t)c->d.Ntheta;
        const uintptr_t a0 = (uintptr_t)d_in, b0 = (uintptr_t)d_out;
        if (a0 < b0 + bytes && b0 < a0 + bytes)
            return set_err(cm, TEUK_E_INVAL, "d_in and d_out overlap (each spans %zu bytes)", bytes);
    }
    size_t need = c2 * 2 * (size_t)(c->d.Nr - 1) * (size_t)c->d.Ntheta;
    if (need > literal_static_scratch_bytes())
        return set_err(cm, TEUK_E_INVAL, "grid needs %.0f bytes of midpoint scratch, above the static limit of 8 MiB",
                       (double)need);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (c->d.precision == TEUK_FP32) {
        StepParams<float> p = make_params<float>(c, 0);
        p.uin = (const float2 *)d_in;
        p.uout = (float2 *)d_out;
        e = launch_literal_step_static<float>(p, (long long)n, st);
    } else {
        StepParams<double> p = make_params<double>(c, 0);
        p.uin = (const double2 *)d_in;
        p.uout = (double2 *)d_out;
        e = launch_literal_step_static<double>(p, (long long)n, st);
    }
    if (e != cudaSuccess) return cuda_err(cm, e, "literal step (static scratch)");
    return TEUK_OK;
}


}  // extern "C"


// ------------------------------------------------------ operator and adjoint

namespace {

// Tile height of the adjoint kernel (one CTA per SM): enough tiles for two
// waves over the SMs where the grid allows, at most 30 rows and about 100 KB
// of shared memory (four state planes) per tile.
int adjoint_tile_rows(const teuk_ctx *c)
{
    const int N = (int)c->d.Ntheta;
    const bool f32 = c->d.precision == TEUK_FP32;
    const long long want = (c->d.Nr + 2LL * sm_count() - 1) / (2LL * sm_count());
    int best = 1;
    for (int tr = 1; tr <= 30; ++tr) {
        size_t sm = f32 ? adjoint_smem_bytes<float>(tr, N) : adjoint_smem_bytes<double>(tr, N);
        if (sm <= 100 * 1024) best = tr;
    }
    if (want >= 4 && want < best) best = (int)want;
    return best;
}

// Tile height of the adjoint step with the spin derivative: twice the
// shared memory per row (eight state planes), at most about 200 KB per tile.
int adjoint_spin_tile_rows(const teuk_ctx *c)
{
    const int N = (int)c->d.Ntheta;
    const bool f32 = c->d.precision == TEUK_FP32;
    const long long want = (c->d.Nr + 2LL * sm_count() - 1) / (2LL * sm_count());
    int best = 1;
    for (int tr = 1; tr <= 30; ++tr) {
        size_t sm = f32 ? adjoint_spin_smem_bytes<float>(tr, N) : adjoint_spin_smem_bytes<double>(tr, N);
        if (sm <= 200 * 1024) best = tr;
    }
    if (want >= 4 && want < best) best = (int)want;
    return best;
}

// The adjoint workspace: accumulators (8 doubles), per-CTA parts, the
// dot product's parts (512 doubles), then the coefficient planes of the
// spin adjoint from a 256-byte boundary.
size_t adjoint_small_doubles(const teuk_ctx *c)
{
    const int tr = adjoint_tile_rows(c), trs = adjoint_spin_tile_rows(c);
    const int grid = (int)((c->d.Nr + tr - 1) / tr), grids = (int)((c->d.Nr + trs - 1) / trs);
    const int gmax = grid > grids ? grid : grids;
    return 8 + 6 * (size_t)gmax + 2 * 256;
}
size_t adjoint_planes_offset(const teuk_ctx *c) { return (sizeof(double) * adjoint_small_doubles(c) + 255) & ~(size_t)255; }
// FP64 only: the FP32 adjoint forms its coefficients in place, which costs
// it less than reading them (the FP64 step is bound by the FP64 pipe, the
// FP32 step is not)
AdjPlaneLayout adjoint_planes_layout(const teuk_ctx *c)
{
    if (c->d.precision == TEUK_FP32) {
        AdjPlaneLayout L = {};
        return L;
    }
    return adj_plane_layout(c->d.Nr, c->d.Ntheta, sizeof(double));
}
size_t adjoint_ws_bytes(const teuk_ctx *c) { return adjoint_planes_offset(c) + adjoint_planes_layout(c).total; }

template <typename T>
AdjPlanes<T> adjoint_planes(const teuk_ctx *c, const void *ws)
{
    typedef typename V2<T>::t c2;
    const char *b = (const char *)ws + adjoint_planes_offset(c);
    const AdjPlaneLayout L = adjoint_planes_layout(c);
    AdjPlanes<T> A;
    A.m.fk = (const c2 *)(b + L.off[0]);
    A.m.dg = (const c2 *)(b + L.off[1]);
    A.m.ct = (const c2 *)(b + L.off[2]);
    A.m.sub = (const T *)(b + L.off[3]);
    A.m.qam = (const T *)(b + L.off[4]);
    A.m.qap = (const T *)(b + L.off[5]);
    A.m.lw = (const T *)(b + L.off[6]);
    A.dlw = (const T *)(b + L.off[7]);
    A.dimp = (const T *)(b + L.off[8]);
    return A;
}

template <typename T>
cudaError_t fill_adjoint_planes(const teuk_ctx *c, void *ws, cudaStream_t st)
{
    typedef typename V2<T>::t c2;
    const AdjPlanes<T> A = adjoint_planes<T>(c, ws);
    MatOut<T> o;
    o.fk = (c2 *)A.m.fk;
    o.dg = (c2 *)A.m.dg;
    o.ct = (c2 *)A.m.ct;
    o.sub = (T *)A.m.sub;
    o.qam = (T *)A.m.qam;
    o.qap = (T *)A.m.qap;
    o.lw = (T *)A.m.lw;
    o.dlw = (T *)A.dlw;
    o.dimp = (T *)A.dimp;
    return launch_mat_coef_to<T>(make_params<T>(c, 0), o, st);
}

}  // namespace

extern "C" {

static int apply_step(teuk_ctx *c, const void *d_in, void *d_out, int64_t n, int first, void *d_h, void *stream)
{
    if (!c) return TEUK_E_STATE;
    if (c->d.scheme != TEUK_SCHEME_SPLIT) return set_err(c, TEUK_E_INVAL, "teuk_apply_step needs the split scheme");
    if (!d_in || !d_out || d_in == d_out || n < 0)
        return set_err(c, TEUK_E_INVAL, "need distinct non-NULL device buffers and n >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (c->d.precision == TEUK_FP32) {
        StepParams<float> p = make_params<float>(c, 0);
        p.uin = (const float2 *)d_in;
        p.uout = (float2 *)d_out;
        p.first = first ? 1 : 0;
        p.nfix = n;
        p.h_out = (double2 *)d_h;
        e = launch_apply_step<float>(p, c->threads, c->smem, st);
    } else {
        StepParams<double> p = make_params<double>(c, 0);
        p.uin = (const double2 *)d_in;
        p.uout = (double2 *)d_out;
        p.first = first ? 1 : 0;
        p.nfix = n;
        p.h_out = (double2 *)d_h;
        e = launch_apply_step<double>(p, c->threads, c->smem, st);
    }
    if (e != cudaSuccess) return cuda_err(c, e, "apply step");
    return TEUK_OK;
}

int teuk_apply_step(teuk_ctx *c, const void *d_in, void *d_out, int64_t n, int first, void *stream)
{
    return apply_step(c, d_in, d_out, n, first, nullptr, stream);
}

int teuk_apply_step_sample(teuk_ctx *c, const void *d_in, void *d_out, int64_t n, int first, void *d_h,
                           void *stream)
{
    if (c && !d_h) return set_err(c, TEUK_E_INVAL, "need a device address for the sample");
    return apply_step(c, d_in, d_out, n, first, d_h, stream);
}

int teuk_apply_sample(teuk_ctx *c, const void *d_s, int physical, void *d_h, void *stream)
{
    if (!c) return TEUK_E_STATE;
    if (!d_s || !d_h) return set_err(c, TEUK_E_INVAL, "need non-NULL device buffers");
    if (c->d.scheme != TEUK_SCHEME_SPLIT && !physical)
        return set_err(c, TEUK_E_INVAL, "the literal scheme has no internal state: pass physical = 1");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (c->d.precision == TEUK_FP32)
        e = launch_sample<float>(make_params<float>(c, 0), (const float2 *)d_s, physical, (double2 *)d_h, st);
    else
        e = launch_sample<double>(make_params<double>(c, 0), (const double2 *)d_s, physical, (double2 *)d_h, st);
    if (e != cudaSuccess) return cuda_err(c, e, "sample");
    return TEUK_OK;
}

int teuk_adjoint_workspace_bytes(const teuk_ctx *c, size_t *bytes)
{
    if (!c || !bytes) return TEUK_E_STATE;
    *bytes = adjoint_ws_bytes(c);
    return TEUK_OK;
}

int teuk_adjoint_prepare(teuk_ctx *c, void *d_ws, void *stream)
{
    if (!c) return TEUK_E_STATE;
    if (c->d.scheme != TEUK_SCHEME_SPLIT) return set_err(c, TEUK_E_INVAL, "the adjoint needs the split scheme");
    if (!d_ws || ((uintptr_t)d_ws & 255)) return set_err(c, TEUK_E_INVAL, "need a 256-byte aligned workspace");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = c->d.precision == TEUK_FP32 ? cudaSuccess : fill_adjoint_planes<double>(c, d_ws, st);
    if (e != cudaSuccess) return cuda_err(c, e, "adjoint planes");
    c->adj_ws = d_ws;
    return TEUK_OK;
}

int teuk_adjoint_step(teuk_ctx *c, const void *d_lam_in, void *d_lam_out, int64_t n, int first, const void *d_gseed,
                      void *d_ws, void *stream)
{
    if (!c) return TEUK_E_STATE;
    if (c->d.scheme != TEUK_SCHEME_SPLIT) return set_err(c, TEUK_E_INVAL, "the adjoint needs the split scheme");
    if (!d_lam_in || !d_lam_out || d_lam_in == d_lam_out || !d_ws || n < 0)
        return set_err(c, TEUK_E_INVAL, "need distinct non-NULL device buffers, a workspace and n >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    const int tr = adjoint_tile_rows(c);
    double *acc = (double *)d_ws, *part = acc + 8;
    cudaError_t e;
    if (c->d.precision == TEUK_FP32) {
        StepParams<float> p = make_params<float>(c, 0);
        p.uin = (const float2 *)d_lam_in;
        p.uout = (float2 *)d_lam_out;
        p.first = first ? 1 : 0;
        p.nfix = n;
        e = launch_adjoint_step<float>(p, tr, (const double2 *)d_gseed, part, acc, st);
    } else {
        StepParams<double> p = make_params<double>(c, 0);
        p.uin = (const double2 *)d_lam_in;
        p.uout = (double2 *)d_lam_out;
        p.first = first ? 1 : 0;
        p.nfix = n;
        // full steps with a prepared workspace read the coefficient planes
        // (the FP64 pipe bounds this step)
        if (!first && d_ws == c->adj_ws)
            e = launch_adjoint_planes<double>(p, adjoint_spin_tile_rows(c), (const double2 *)d_gseed,
                                              adjoint_planes<double>(c, d_ws), part, acc, st);
        else
            e = launch_adjoint_step<double>(p, tr, (const double2 *)d_gseed, part, acc, st);
    }
    if (e != cudaSuccess) return cuda_err(c, e, "adjoint step");
    return TEUK_OK;
}

static int adjoint_spin(teuk_ctx *c, const void *d_lam_in, void *d_lam_out, const void *d_s, const void *d_tape,
                        int64_t n, int first, const void *d_gseed, void *d_ws, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    if (d_ws != c->adj_ws)
        return set_err(c, TEUK_E_STATE, "call teuk_adjoint_prepare with this workspace first");
    const int tr = adjoint_spin_tile_rows(c);
    double *acc = (double *)d_ws, *part = acc + 8;
    cudaError_t e;
    if (c->d.precision == TEUK_FP32) {
        StepParams<float> p = make_params<float>(c, 0);
        p.uin = (const float2 *)d_lam_in;
        p.uout = (float2 *)d_lam_out;
        p.first = first ? 1 : 0;
        p.nfix = n;
        e = launch_adjoint_spin<float>(p, tr, (const float2 *)d_s, (const float2 *)d_tape, (const double2 *)d_gseed,
                                       adjoint_planes<float>(c, d_ws), part, acc, st);
    } else {
        StepParams<double> p = make_params<double>(c, 0);
        p.uin = (const double2 *)d_lam_in;
        p.uout = (double2 *)d_lam_out;
        p.first = first ? 1 : 0;
        p.nfix = n;
        e = launch_adjoint_spin<double>(p, tr, (const double2 *)d_s, (const double2 *)d_tape,
                                        (const double2 *)d_gseed, adjoint_planes<double>(c, d_ws), part, acc, st);
    }
    if (e != cudaSuccess) return cuda_err(c, e, "adjoint step (spin)");
    return TEUK_OK;
}

int teuk_adjoint_step_spin(teuk_ctx *c, const void *d_lam_in, void *d_lam_out, const void *d_s, int64_t n, int first,
                           const void *d_gseed, void *d_ws, void *stream)
{
    if (!c) return TEUK_E_STATE;
    if (c->d.scheme != TEUK_SCHEME_SPLIT) return set_err(c, TEUK_E_INVAL, "the adjoint needs the split scheme");
    if (!d_lam_in || !d_lam_out || !d_s || d_lam_in == d_lam_out || d_s == d_lam_out || !d_ws || n < 0)
        return set_err(c, TEUK_E_INVAL, "need distinct non-NULL device buffers, a workspace and n >= 0");
    return adjoint_spin(c, d_lam_in, d_lam_out, d_s, nullptr, n, first, d_gseed, d_ws, stream);
}

int teuk_tape_bytes(const teuk_ctx *c, size_t *bytes)
{
    if (!c || !bytes) return TEUK_E_STATE;
    const size_t c2 = c->d.precision == TEUK_FP32 ? sizeof(float2) : sizeof(double2);
    *bytes = (tape_elems(c->d.Nr, c->d.Ntheta) * c2 + 255) & ~(size_t)255;
    return TEUK_OK;
}

int teuk_apply_step_tape(teuk_ctx *c, const void *d_in, void *d_out, int64_t n, int first, void *d_h, void *d_tape,
                         void *stream)
{
    if (!c) return TEUK_E_STATE;
    if (c->d.scheme != TEUK_SCHEME_SPLIT) return set_err(c, TEUK_E_INVAL, "teuk_apply_step needs the split scheme");
    if (!d_in || !d_out || !d_h || !d_tape || d_in == d_out || n < 0 || ((uintptr_t)d_tape & 255))
        return set_err(c, TEUK_E_INVAL, "need distinct non-NULL device buffers, a 256-byte aligned tape and n >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (c->d.precision == TEUK_FP32) {
        StepParams<float> p = make_params<float>(c, 0);
        p.uin = (const float2 *)d_in;
        p.uout = (float2 *)d_out;
        p.first = first ? 1 : 0;
        p.nfix = n;
        p.h_out = (double2 *)d_h;
        p.tape = (float2 *)d_tape;
        e = launch_apply_step<float>(p, c->threads, c->smem, st);
    } else {
        StepParams<double> p = make_params<double>(c, 0);
        p.uin = (const double2 *)d_in;
        p.uout = (double2 *)d_out;
        p.first = first ? 1 : 0;
        p.nfix = n;
        p.h_out = (double2 *)d_h;
        p.tape = (double2 *)d_tape;
        e = launch_apply_step<double>(p, c->threads, c->smem, st);
    }
    if (e != cudaSuccess) return cuda_err(c, e, "apply step (tape)");
    return TEUK_OK;
}

int teuk_adjoint_step_tape(teuk_ctx *c, const void *d_lam_in, void *d_lam_out, const void *d_tape, int64_t n,
                           int first, const void *d_gseed, void *d_ws, void *stream)
{
    if (!c) return TEUK_E_STATE;
    if (c->d.scheme != TEUK_SCHEME_SPLIT) return set_err(c, TEUK_E_INVAL, "the adjoint needs the split scheme");
    if (!d_lam_in || !d_lam_out || !d_tape || d_lam_in == d_lam_out || !d_ws || n < 0 ||
        ((uintptr_t)d_tape & 255))
        return set_err(c, TEUK_E_INVAL, "need distinct non-NULL device buffers, an aligned tape, a workspace and n >= 0");
    return adjoint_spin(c, d_lam_in, d_lam_out, nullptr, d_tape, n, first, d_gseed, d_ws, stream);
}

int teuk_dot(teuk_ctx *c, const void *d_x, const void *d_y, const void *d_z, void *d_ws, void *d_out, void *stream)
{
    if (!c) return TEUK_E_STATE;
    if (!d_x || !d_y || !d_ws || !d_out) return set_err(c, TEUK_E_INVAL, "need non-NULL device buffers");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = 2 * (size_t)c->d.Nr * (size_t)c->d.Ntheta;
    double *part = (double *)d_ws + adjoint_small_doubles(c) - 2 * 256;
    cudaError_t e;
    if (c->d.precision == TEUK_FP32)
        e = launch_dot<float>((const float2 *)d_x, (const float2 *)d_y, (const float2 *)d_z, n, part,
                              (double2 *)d_out, st);
    else
        e = launch_dot<double>((const double2 *)d_x, (const double2 *)d_y, (const double2 *)d_z, n, part,
                               (double2 *)d_out, st);
    if (e != cudaSuccess) return cuda_err(c, e, "dot");
    return TEUK_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches

struct teuk_batch {
    std::vector<teuk_ctx *> c;
    std::vector<int> tr;             // tile height per instance
    int prec, seg;
    char *ws;                        // caller-owned device workspace
    size_t ws_bytes, par_bytes;      // par_bytes: one parameter table
    size_t off_par[3], off_tiles;    // tables: in = cur, in = cur ^ 1, first step; tile list
    int ntot;
    int ks;                          // time steps per launch (1, or 2 once every instance is shifted)
    size_t smem;
    cudaGraphExec_t graph;
    cudaStream_t graph_stream;
    std::vector<unsigned char> hpar;
    std::vector<int2> htiles;
    char err[512];
};

namespace {

__attribute__((format(printf, 3, 4))) int bset_err(teuk_batch *b, int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b ? b->err : g_init_err, 512, fmt, ap);
    va_end(ap);
    return code;
}

int bcuda_err(teuk_batch *b, cudaError_t e, const char *where)
{
    snprintf(b ? b->err : g_init_err, 512, "%s: %s", where, cudaGetErrorString(e));
    return TEUK_E_CUDA;
}

#define BCK(call, where)                                      \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return bcuda_err(b, e_, where); \
    } while (0)

size_t params_size(int prec) { return prec == TEUK_FP32 ? sizeof(StepParams<float>) : sizeof(StepParams<double>); }

size_t batch_ws_bytes(teuk_ctx *const *ctxs, int count, size_t *par_bytes, size_t *tiles_off)
{
    const size_t pb = align256(params_size(ctxs[0]->d.precision) * (size_t)count);
    size_t rows = 0;
    for (int i = 0; i < count; ++i) rows += (size_t)ctxs[i]->d.Nr;
    if (par_bytes) *par_bytes = pb;
    if (tiles_off) *tiles_off = 3 * pb;
    return 3 * pb + align256(sizeof(int2) * rows);
}

// Rows of one implicit pass for Ntheta (256 threads / G).
int batch_rpp(int N) { return 256 / implicit_group(N); }

// Shared memory of a batch tile of height tr with ks steps per launch.
size_t batch_tile_smem(int prec, int tr, int N, int ks)
{
    if (ks == 2) return prec == TEUK_FP32 ? split2_smem_bytes<float>(tr, N) : split2_smem_bytes<double>(tr, N);
    return prec == TEUK_FP32 ? split_smem_bytes<float>(tr, N) : split_smem_bytes<double>(tr, N);
}

// Default tile height: the largest whole number of implicit passes (tile
// rows plus halos) whose tile leaves room for as many CTAs per SM as the
// kernel's registers allow: two for FP32 rows of up to 128 theta points,
// one otherwise (wider segments and FP64 take over 128 registers a thread).
int batch_default_tr(const teuk_ctx *c, int ks)
{
    const int N = (int)c->d.Ntheta, rpp = batch_rpp(N);
    const size_t budget =
        (c->d.precision == TEUK_FP32 && implicit_seg(N) <= kSegNarrow) ? 112 * 1024 : 220 * 1024;
    int best = 1;
    for (int R = rpp; R - 2 * ks <= 254; R += rpp) {
        const int tr = R - 2 * ks;
        if (tr < 1) continue;
        if (batch_tile_smem(c->d.precision, tr, N, ks) > budget && best > 1) break;
        best = tr;
        if (tr >= c->d.Nr) break;
    }
    return best;
}

// Tile list (instances interleaved tile by tile) and shared memory for the
// current tile heights; drops the captured graph.
int batch_layout(teuk_batch *b)
{
    const int n = (int)b->c.size();
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_stream = nullptr;
    std::vector<int> nt(n);
    int maxt = 0;
    size_t smem = 0;
    for (int i = 0; i < n; ++i) {
        const teuk_ctx *c = b->c[i];
        nt[i] = (int)((c->d.Nr + b->tr[i] - 1) / b->tr[i]);
        maxt = nt[i] > maxt ? nt[i] : maxt;
        const int N = (int)c->d.Ntheta;
        size_t sm = batch_tile_smem(b->prec, b->tr[i], N, b->ks);
        smem = sm > smem ? sm : smem;
    }
    if (smem > 227 * 1024) return bset_err(b, TEUK_E_INVAL, "a tile of the batch does not fit in shared memory");
    int k = b->prec == TEUK_FP32 ? split_batch_blocks_per_sm<float>(b->seg, smem, b->ks)
                                 : split_batch_blocks_per_sm<double>(b->seg, smem, b->ks);
    // the first step of a two-step batch runs the one-step kernel with this shared memory
    if (k >= 1 && b->ks == 2)
        k = b->prec == TEUK_FP32 ? split_batch_blocks_per_sm<float>(b->seg, smem, 1)
                                 : split_batch_blocks_per_sm<double>(b->seg, smem, 1);
    if (k < 1) return bset_err(b, TEUK_E_INVAL, "the batched kernel does not fit on this device with these tiles");
    b->htiles.clear();
    for (int t = 0; t < maxt; ++t)
        for (int i = 0; i < n; ++i)
            if (t < nt[i]) b->htiles.push_back(make_int2(i, t));
    b->ntot = (int)b->htiles.size();
    b->smem = smem;
    if ((size_t)b->ntot * sizeof(int2) > b->ws_bytes - b->off_tiles)
        return bset_err(b, TEUK_E_INVAL, "workspace too small for the tile list");
    // launches in flight on any stream may still read the old list
    BCK(cudaDeviceSynchronize(), "wait before the tile list changes");
    BCK(cudaMemcpy(b->ws + b->off_tiles, b->htiles.data(), sizeof(int2) * b->htiles.size(), cudaMemcpyHostToDevice),
        "tile list upload");
    return TEUK_OK;
}

template <typename T>
void batch_fill(teuk_batch *b)
{
    const int n = (int)b->c.size();
    b->hpar.assign(3 * b->par_bytes, 0);
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < n; ++i) {
            teuk_ctx *c = b->c[i];
            StepParams<T> p = make_params<T>(c, k == 1 ? c->cur ^ 1 : c->cur);
            p.tile_rows = b->tr[i];
            p.first = k == 2 ? (c->shifted ? 0 : 1) : 0;
            memcpy(b->hpar.data() + k * b->par_bytes + i * sizeof(StepParams<T>), &p, sizeof(p));
        }
}

// Parameter tables for the instances' current levels, uploaded on `st`.
int batch_tables(teuk_batch *b, cudaStream_t st)
{
    if (b->prec == TEUK_FP32) batch_fill<float>(b);
    else batch_fill<double>(b);
    BCK(cudaMemcpyAsync(b->ws, b->hpar.data(), b->hpar.size(), cudaMemcpyHostToDevice, st), "parameter upload");
    return TEUK_OK;
}

// One launch from parameter table `table` with ks steps (the first-step
// table always takes one).
cudaError_t batch_launch(teuk_batch *b, int table, int ks, cudaStream_t st)
{
    const int2 *tiles = (const int2 *)(b->ws + b->off_tiles);
    if (table == 2) ks = 1;
    if (b->prec == TEUK_FP32)
        return launch_split_batch<float>((const StepParams<float> *)(b->ws + b->off_par[table]), tiles, b->ntot, b->seg,
                                         b->smem, ks, st);
    return launch_split_batch<double>((const StepParams<double> *)(b->ws + b->off_par[table]), tiles, b->ntot, b->seg,
                                      b->smem, ks, st);
}

int batch_step_impl(teuk_batch *b, int64_t nsteps, cudaStream_t st)
{
    int64_t left = nsteps;
    if (left <= 0) return TEUK_OK;
    int r = batch_tables(b, st);
    if (r != TEUK_OK) return r;
    bool any_first = false;
    for (teuk_ctx *c : b->c) any_first = any_first || !c->shifted;
    if (any_first) {
        // first step from physical states: s_{n+1} = LW C_{dt/2} u_n where needed
        BCK(batch_launch(b, 2, 1, st), "batched first step");
        for (teuk_ctx *c : b->c) {
            c->cur ^= 1;
            c->shifted = 1;
        }
        left -= 1;
        r = batch_tables(b, st);
        if (r != TEUK_OK) return r;
    }
    if (st != nullptr && left >= 2 * kGraphChunk) {
        if (b->graph && b->graph_stream != st) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        if (!b->graph) {
            cudaGraph_t graph;
            BCK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
            cudaError_t le = cudaSuccess;
            // kGraphChunk / ks launches: an even count, so the level parity is unchanged
            for (int k = 0; k < kGraphChunk / b->ks && le == cudaSuccess; ++k) le = batch_launch(b, k & 1, b->ks, st);
            cudaError_t ee = cudaStreamEndCapture(st, &graph);
            if (le != cudaSuccess) return bcuda_err(b, le, "captured batched launch");
            if (ee != cudaSuccess) return bcuda_err(b, ee, "end capture");
            cudaError_t ie = cudaGraphInstantiate(&b->graph, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) {
                b->graph = nullptr;
                return bcuda_err(b, ie, "graph instantiate");
            }
            b->graph_stream = st;
        }
        while (left >= kGraphChunk) {
            BCK(cudaGraphLaunch(b->graph, st), "graph launch");
            left -= kGraphChunk;
        }
    }
    // each launch (one or two steps) flips every instance's level once
    int64_t launches = 0;
    for (; left >= b->ks; left -= b->ks, ++launches) BCK(batch_launch(b, (int)(launches & 1), b->ks, st), "batched step");
    for (; left > 0; --left, ++launches) BCK(batch_launch(b, (int)(launches & 1), 1, st), "batched step");
    for (teuk_ctx *c : b->c) {
        c->cur ^= (int)(launches & 1);
        c->step += nsteps;
    }
    return TEUK_OK;
}

}  // namespace

extern "C" {

int teuk_batch_workspace_bytes(teuk_ctx *const *ctxs, int count, size_t *bytes)
{
    if (!ctxs || count < 1 || !bytes) {
        snprintf(g_init_err, sizeof(g_init_err), "need count >= 1 contexts and an output pointer");
        return TEUK_E_INVAL;
    }
    for (int i = 0; i < count; ++i)
        if (!ctxs[i]) {
            snprintf(g_init_err, sizeof(g_init_err), "context %d is NULL", i);
            return TEUK_E_INVAL;
        }
    *bytes = batch_ws_bytes(ctxs, count, nullptr, nullptr);
    return TEUK_OK;
}

int teuk_batch_create(teuk_ctx *const *ctxs, int count, void *d_ws, size_t ws_bytes, teuk_batch **out)
{
    if (!out) return TEUK_E_INVAL;
    *out = nullptr;
    size_t need = 0;
    int r = teuk_batch_workspace_bytes(ctxs, count, &need);
    if (r != TEUK_OK) return r;
    if (!d_ws || ws_bytes < need || ((uintptr_t)d_ws & 255u)) {
        snprintf(g_init_err, sizeof(g_init_err), "workspace must be 256-byte aligned and at least %zu bytes", need);
        return TEUK_E_INVAL;
    }
    const int prec = ctxs[0]->d.precision;
    const int seg = implicit_seg((int)ctxs[0]->d.Ntheta);
    for (int i = 0; i < count; ++i) {
        const teuk_ctx *c = ctxs[i];
        const char *why = nullptr;
        if (c->d.scheme != TEUK_SCHEME_SPLIT) why = "is not a split-scheme context";
        else if (c->d.precision != prec) why = "has another state precision than context 0";
        else if (implicit_seg((int)c->d.Ntheta) != seg) why = "has an Ntheta of another theta-segment class";
        for (int j = 0; j < i && !why; ++j)
            if (ctxs[j] == c) why = "appears twice";
        if (why) {
            snprintf(g_init_err, sizeof(g_init_err), "context %d %s", i, why);
            return TEUK_E_INVAL;
        }
    }
    teuk_batch *b = new (std::nothrow) teuk_batch();
    if (!b) return TEUK_E_INVAL;
    b->c.assign(ctxs, ctxs + count);
    b->prec = prec;
    b->seg = seg;
    b->ws = (char *)d_ws;
    b->ws_bytes = ws_bytes;
    batch_ws_bytes(ctxs, count, &b->par_bytes, &b->off_tiles);
    for (int k = 0; k < 3; ++k) b->off_par[k] = (size_t)k * b->par_bytes;
    b->ks = split_batch_available(seg, 2) ? 2 : 1;
    b->tr.resize(count);
    for (int i = 0; i < count; ++i) b->tr[i] = batch_default_tr(ctxs[i], b->ks);
    r = batch_layout(b);
    if (r != TEUK_OK) {
        memcpy(g_init_err, b->err, sizeof(g_init_err));
        delete b;
        return r;
    }
    // the workspace holds valid parameter tables from the start
    r = batch_tables(b, nullptr);
    if (r == TEUK_OK && cudaStreamSynchronize(nullptr) != cudaSuccess) r = bcuda_err(b, cudaGetLastError(), "table upload");
    if (r != TEUK_OK) {
        memcpy(g_init_err, b->err, sizeof(g_init_err));
        delete b;
        return r;
    }
    for (teuk_ctx *c : b->c) drop_graphs(c);
    *out = b;
    return TEUK_OK;
}

int teuk_batch_step(teuk_batch *b, int64_t nsteps, void *stream)
{
    if (!b) return TEUK_E_STATE;
    if (nsteps < 0) return bset_err(b, TEUK_E_INVAL, "nsteps must be >= 0");
    return batch_step_impl(b, nsteps, (cudaStream_t)stream);
}

int teuk_batch_tiling(const teuk_batch *b, int *tile_rows, int *total_tiles, size_t *smem_bytes)
{
    if (!b) return TEUK_E_STATE;
    if (tile_rows)
        for (size_t i = 0; i < b->tr.size(); ++i) tile_rows[i] = b->tr[i];
    if (total_tiles) *total_tiles = b->ntot;
    if (smem_bytes) *smem_bytes = b->smem;
    return TEUK_OK;
}

int teuk_batch_set_tiling(teuk_batch *b, const int *tile_rows)
{
    if (!b) return TEUK_E_STATE;
    if (!tile_rows) return bset_err(b, TEUK_E_INVAL, "tile_rows is NULL");
    std::vector<int> old = b->tr;
    for (size_t i = 0; i < b->tr.size(); ++i) {
        if (tile_rows[i] < 1 || tile_rows[i] > 254) return bset_err(b, TEUK_E_INVAL, "tile_rows out of range [1, 254]");
        b->tr[i] = tile_rows[i];
    }
    int r = batch_layout(b);
    if (r != TEUK_OK) {
        b->tr = old;
        char keep[512];
        memcpy(keep, b->err, sizeof(keep));
        batch_layout(b);
        memcpy(b->err, keep, sizeof(keep));
    }
    return r;
}

int teuk_batch_autotune(teuk_batch *b, int trial_steps, void *stream)
{
    if (!b) return TEUK_E_STATE;
    if (trial_steps < 1 || trial_steps > 100000) return bset_err(b, TEUK_E_INVAL, "trial_steps out of range");
    cudaStream_t st = (cudaStream_t)stream;
    // For each number of steps per launch the kernel offers, a coordinate
    // descent over the Ntheta classes of the batch: for each class, every
    // whole number of implicit passes per tile that fits is timed with the
    // other classes fixed, and the fastest is kept.  The faster of the
    // descents' results (time per step) is the configuration.
    std::vector<int> classes;
    for (teuk_ctx *c : b->c) {
        int N = (int)c->d.Ntheta;
        bool seen = false;
        for (int v : classes) seen = seen || v == N;
        if (!seen) classes.push_back(N);
    }
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0), "event");
    BCK(cudaEventCreate(&e1), "event");
    int rc = TEUK_OK;
    // ms per step of the current tile list and steps per launch (negative: does not fit)
    auto trial = [&](float &ms_step) -> int {
        ms_step = -1.0f;
        if (batch_layout(b) != TEUK_OK) return TEUK_OK;
        for (teuk_ctx *c : b->c) c->shifted = 1;
        int r = batch_tables(b, st);   // parameters for these tile heights
        if (r != TEUK_OK) return r;
        cudaError_t e = cudaSuccess;
        for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = batch_launch(b, w & 1, b->ks, st);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int w = 0; w < trial_steps && e == cudaSuccess; ++w) e = batch_launch(b, w & 1, b->ks, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) return bcuda_err(b, e, "batch autotune trial");
        ms_step = ms / (float)(trial_steps * b->ks);
        return TEUK_OK;
    };
    float best_all = 3.4e38f;
    int best_ks = b->ks;
    std::vector<int> best_tr = b->tr;
    for (int ks = 1; ks <= 2 && rc == TEUK_OK; ++ks) {
        if (!split_batch_available(b->seg, ks)) continue;
        b->ks = ks;
        for (size_t i = 0; i < b->c.size(); ++i) b->tr[i] = batch_default_tr(b->c[i], ks);
        for (int N : classes) {
            const int rpp = batch_rpp(N);
            std::vector<int> keep = b->tr;
            float best = 3.4e38f;
            int best_h = -1;
            for (int R = rpp; R - 2 * ks <= 254 && rc == TEUK_OK; R += rpp) {
                if (R - 2 * ks < 1) continue;
                b->tr = keep;
                for (size_t i = 0; i < b->c.size(); ++i)
                    if ((int)b->c[i]->d.Ntheta == N) b->tr[i] = R - 2 * ks;
                float ms = -1.0f;
                rc = trial(ms);
                if (rc != TEUK_OK || ms < 0.0f) break;   // larger tiles do not fit either
                if (ms < best) {
                    best = ms;
                    best_h = R - 2 * ks;
                }
            }
            b->tr = keep;
            if (best_h > 0)
                for (size_t i = 0; i < b->c.size(); ++i)
                    if ((int)b->c[i]->d.Ntheta == N) b->tr[i] = best_h;
            if (rc != TEUK_OK) break;
        }
        if (rc != TEUK_OK) break;
        float ms = -1.0f;
        rc = trial(ms);
        if (rc == TEUK_OK && ms >= 0.0f && ms < best_all) {
            best_all = ms;
            best_ks = ks;
            best_tr = b->tr;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->ks = best_ks;
    b->tr = best_tr;
    if (rc != TEUK_OK) {
        batch_layout(b);
        return rc;
    }
    int r = batch_layout(b);
    if (r != TEUK_OK) return r;
    for (teuk_ctx *c : b->c) {
        r = reset_state(c, st);
        if (r != TEUK_OK) {
            snprintf(b->err, sizeof(b->err), "reset after autotune: %.400s", c->err);
            return r;
        }
    }
    BCK(cudaStreamSynchronize(st), "autotune sync");
    return TEUK_OK;
}

int teuk_batch_steps_per_launch(const teuk_batch *b, int *steps_per_launch)
{
    if (!b) return TEUK_E_STATE;
    if (steps_per_launch) *steps_per_launch = b->ks;
    return TEUK_OK;
}

int teuk_batch_set_steps_per_launch(teuk_batch *b, int steps_per_launch)
{
    if (!b) return TEUK_E_STATE;
    if (steps_per_launch != 1 && steps_per_launch != 2)
        return bset_err(b, TEUK_E_INVAL, "steps_per_launch must be 1 or 2");
    if (!split_batch_available(b->seg, steps_per_launch))
        return bset_err(b, TEUK_E_INVAL, "two steps per launch need Ntheta <= 256");
    const int old = b->ks;
    b->ks = steps_per_launch;
    int r = batch_layout(b);
    if (r != TEUK_OK) {
        b->ks = old;
        char keep[512];
        memcpy(keep, b->err, sizeof(keep));
        batch_layout(b);
        memcpy(b->err, keep, sizeof(keep));
    }
    return r;
}

const char *teuk_batch_last_error(const teuk_batch *b) { return b ? b->err : g_init_err; }

int teuk_batch_destroy(teuk_batch *b)
{
    if (!b) return TEUK_OK;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    delete b;
    return TEUK_OK;
}

}  // extern "C"
