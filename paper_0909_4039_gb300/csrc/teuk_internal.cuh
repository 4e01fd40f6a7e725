// teuk_internal.cuh -- definitions shared by the translation units of libteuk
// (host API, FP64 coefficient generation, step kernels).  Not installed.
//
// Data layout in device memory (all caller-owned, 256-byte aligned blocks):
//   state  : 2 time levels x [2 planes][Nr][Ntheta] complex T (T = float or
//            double), plane 0 = Phi, plane 1 = Pi, theta fastest.
//   coef   : r tables   [2Nr-1][NRF] FP64 and [2Nr-1][NRF] T
//                        (position p = 2i: node i; p = 2i+1: r*_{i+1/2})
//            step table [2Nr-1][NSF] T (see SField) and its spin
//                        derivative d/da at fixed r* (split scheme)
//            theta tables [NTF][Ntheta] FP64 and T
//            pivots     two tables [Nr][Ntheta] complex T, for implicit
//                        steps of length dt and dt/2 (row-major, so the
//                        lanes that solve one theta row read it with
//                        contiguous vector loads)
//            patch      [patch_rows][2][Ntheta] complex T (node, half node)
//            weights    [Ntheta] FP64
//            ctl        step counter, CTA ticket, error flags
//            staging    host <-> device conversion chunk (FP32 state only)
//            scratch    literal scheme only: midpoints [2][Nr-1][Ntheta] T
//   wave   : ring buffer [capacity][1 + Ntheta] complex double (h_n, row).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "teuk.h"

namespace teuk {

// Fields of one r-table entry.  With Sigma^2 = R2 - aD sin^2(theta) and
// sg = 1/Sigma^2 the coefficients of the first-order system are
//   b      = R sqrt(sg)
//   c_t    = sg (CTR + i (CTI + CTC cos theta))
//   c_*    = -sg (CSR + i CSI)
//   b b_*  = sg (E1 - sg (E2 - E3 sin^2 theta))
//   K      = b c_t - c_* - b b_*
//   c0rad  = -sg (C0R + i C0I)
//   q      = DELTA sg
enum RField {
    RF_R = 0, RF_R2, RF_AD, RF_DELTA, RF_CTR, RF_CTI, RF_CTC, RF_CSR, RF_CSI,
    RF_E1, RF_E2, RF_E3, RF_C0R, RF_C0I, RF_RR, RF_X, NRF
};

// Fields of the step table: one entry of NSF values per r* position (node
// i at 2i, half node at 2i+1), in the state precision, read by the forward
// step kernels.  The first block is the implicit stage's (unscaled r-table
// values); the second is the Lax-Wendroff stages', with c_p = dt/dr* at
// nodes (Eq. 14) and dt/(2 dr*) at half nodes (Eq. 13) folded in, so that
// with rs = 1/Sigma, sg = rs^2
//   c_p b   = rs RB
//   c_p K   = sg (sg (E2 - E3 sin^2) + rs RCTR + CSE) + i sg (rs (RCTC cos + RCTI) + CSI)
// (K = b c_t - c_* - b b_* as for RField).  The last block holds the
// radial factors of the source (set by teuk_set_source, zero outside its
// patch rows): the source term of Eq. 1 after the division that gives
// Eq. 9 is separable,
//   F = A 4 pi (r^2 + a^2 cos^2) Delta/(Sigma^2 r^3) G_r(r*) G_th(theta)
//     = SRC sg (SR2 GTH + GA2),   SRC = A 4 pi Delta G_r / r^3,  SR2 = r^2,
// with GTH = G_th and GA2 = a^2 cos^2 G_th in the theta table.
enum SField {
    SF_R2 = 0, SF_AD, SF_DELTA, SF_CTR, SF_CTI, SF_CTC, SF_C0R, SF_C0I,
    SF_RB, SF_E2, SF_E3, SF_RCTR, SF_CSE, SF_RCTC, SF_RCTI, SF_CSI,
    SF_SRE, SF_SIM, SF_SR2, SF_SPAD, NSF
};

// Fields of the theta table.  AM, A0, AP are row j of the angular operator
// A_th = -(d_thth + cot d_th) + (m + s cos)^2/sin^2 - s, centred differences,
// parity ghosts folded into A0 at j = 0 and j = Ntheta-1.
// GTH, GA2: the angular factors of the source (see SField), set by
// teuk_set_source.
// DGA2 = d GA2 / d a (the spin derivative of the adjoint).
enum TField { TF_S2 = 0, TF_C, TF_AM, TF_A0, TF_AP, TF_GTH, TF_GA2, TF_DGA2, NTF };

// Error flags in Ctl::flags.
enum : unsigned { FLAG_NONFINITE = 1u, FLAG_TIMEOUT = 2u };

struct Ctl {
    long long step;      // index n of the state the next step reads
    unsigned ticket;     // CTAs of the current step that have finished
    unsigned flags;      // FLAG_*
    long long pad[6];
};

template <typename T> struct V2;
template <> struct V2<float> { typedef float2 t; };
template <> struct V2<double> { typedef double2 t; };

// Constants of one implicit SDIRK2 step of length h.
template <typename T> struct ImpConst {
    typedef typename V2<T>::t c2;
    T gh, gh2, h1g, h12g;    // gamma h, (gamma h)^2, (1-gamma) h, (1-2 gamma) h
    T h, g2h1;               // h, 2 gamma (1-gamma) h^2
    const c2 *piv;           // Thomas pivots of the stage matrix, [Nr][Nth]
    const int *plan;         // scan levels of each row's solves, [Nr]: forward | backward << 8
    // each lane segment's products of the solve's multipliers, [Nr][G][2]:
    // prod(-e_j sub_j) (forward) and prod(-fk_j) (backward), as
    // scan_plan_lu forms them; read when the row's scan uses a level
    const c2 *seg;
};

// Materialised coefficients of the FP64 path: the implicit step of length
// dt ([Nr][Nth] per element, as imp_elem forms them) and the Lax-Wendroff
// stages ([2Nr-1][Nth][4]: c_p b, c_p K, 1/Sigma^2 per position and theta).
// The FP64 pipe is the bound of the FP64 step, so what the step can read
// instead of recompute it reads.
template <typename T> struct MatPlanes {
    typedef typename V2<T>::t c2;
    const c2 *fk, *dg, *ct;
    const T *sub, *qam, *qap;
    const T *lw;
};

// The coefficient planes of the adjoint step with the spin derivative, in
// its workspace (either precision): the full step's MatPlanes, the spin
// derivatives of the Lax-Wendroff coefficients (dlw, [2Nr-1][Nth][4]:
// d(c_p b), d(c_p K), d(1/Sigma^2)) and of the implicit operator (dimp,
// [Nr][Nth][8]: dW's diagonal (2), dc_t (2), dW's off-diagonals, 0, 0).
template <typename T> struct AdjPlanes {
    MatPlanes<T> m;
    const T *dlw, *dimp;
};

// One applied step's tape record, in elements of the state's complex type:
// the first stage value U1 and the implicit stage's output U2 = C_h s_n of
// every row ([2][Nr][Nth] each), then the input's extraction row ([2][Nth]).
__host__ __device__ inline size_t tape_u2_off(long long Nr, long long Nth) { return 2 * (size_t)Nr * (size_t)Nth; }
__host__ __device__ inline size_t tape_x_off(long long Nr, long long Nth) { return 4 * (size_t)Nr * (size_t)Nth; }
__host__ __device__ inline size_t tape_elems(long long Nr, long long Nth) { return 4 * (size_t)Nr * (size_t)Nth + 2 * (size_t)Nth; }

// Where the generator of k_mat_coef writes (dlw, dimp NULL: no derivatives).
template <typename T> struct MatOut {
    typedef typename V2<T>::t c2;
    c2 *fk, *dg, *ct;
    T *sub, *qam, *qap, *lw, *dlw, *dimp;
};

// Byte layout of those planes from offset 0 of their region: plane offsets
// (fk, dg, ct, sub, qam, qap, lw, dlw, dimp) and the total.
struct AdjPlaneLayout {
    size_t off[9];
    size_t total;
};
inline AdjPlaneLayout adj_plane_layout(long long Nr, long long Nth, size_t tsize)
{
    const size_t pl = (size_t)Nr * (size_t)Nth, pos = (size_t)(2 * Nr - 1) * (size_t)Nth;
    const size_t sz[9] = {2 * pl * tsize, 2 * pl * tsize, 2 * pl * tsize, pl * tsize, pl * tsize, pl * tsize,
                          4 * pos * tsize, 4 * pos * tsize, 8 * pl * tsize};
    AdjPlaneLayout L;
    size_t o = 0;
    for (int k = 0; k < 9; ++k) {
        L.off[k] = o;
        o = (o + sz[k] + 255) & ~(size_t)255;
    }
    L.total = o;
    return L;
}

// Everything a step kernel needs, passed by value.
template <typename T> struct StepParams {
    typedef typename V2<T>::t c2;
    int Nr, Nth;
    int tile_rows;           // output rows per CTA (split kernel)
    int pitch;               // shared-memory row pitch in complex elements
    int group;               // threads per theta row in the implicit phase
    int first;               // 1: implicit step dt/2 (input is a physical state)
    int imp_only;            // 1: only C_{dt/2} on the tile rows (state output)
    int bulk;                // 1: tile rows move by TMA bulk copies (rows are 16-byte multiples)
    int vec;                 // 1: theta segments are whole and 16-byte aligned (vector loads)
    int i_ext;               // extraction node
    int wave_cap;            // ring-buffer slots
    int patch_p0, patch_np;  // source patch rows [p0, p0+np); np = 0: no source
    int wait0;               // try_wait rounds of a tile's waits on its state copy (< 0: kWaitLimit)
    T dt, half_dt, drs_inv;  // step, dt/2, 1/dr*
    ImpConst<T> full, half;  // implicit steps of length dt and dt/2
    double dt64;             // dt in FP64 (time and phase)
    double mOmega;           // m * Omega (FP64)
    const T *rtab;           // [2Nr-1][NRF]
    const T *stab;           // step table [2Nr-1][NSF]
    const T *dstab;          // its derivative with respect to the spin a at fixed r* and theta
    MatPlanes<T> mat;        // materialised coefficients (mat_on)
    int mat_on;              // 1: full steps read them (FP64 state)
    const T *thtab;          // [NTF][Nth]
    const c2 *patch;         // [np][2][Nth]
    const double *w;         // [Nth]
    const c2 *uin;           // [2][Nr][Nth]
    c2 *uout;                // [2][Nr][Nth]
    c2 *mid;                 // literal scheme scratch [2][Nr-1][Nth]
    double2 *wave;           // [cap][1 + Nth]
    Ctl *ctl;
    // Applying one step to caller buffers (nfix >= 0): the step index is
    // nfix, the step counter is not touched and the ring buffer is not
    // written; with h_out set, the sample E C_{dt/2} of the output state goes
    // to *h_out (FP64) instead.
    long long nfix;
    double2 *h_out;
    // Forward tape of an applied step (nfix >= 0, one step per launch):
    // the record tape_* describes, or NULL.
    c2 *tape;
    // Source-parameter derivatives (adjoint step): the unit-amplitude patch
    // [np][2][Nth] (same rows as patch), the amplitude, the r* grid and the
    // orbit's r0*, 1/sigma_r^2, d r0*/d r0 and m dOmega/d r0.
    const c2 *patchu;
    int unit_p0, unit_np;    // rows of the unit-amplitude patch (np = 0: none)
    double amp_re, amp_im, rs_min64, drs64, rs0, inv_sig_r2, drs0_dr0, m_dOmega;
    double m_dOmega_da;      // m dOmega/da of the orbit (spin derivative of the source phase)
};

// SDIRK2 constant gamma = 1 - 1/sqrt(2) (Alexander 1977).
constexpr double kGamma = 0.29289321881345247559915563789515;
constexpr double kPi = 3.14159265358979323846264338327950;

// Shared-memory carve-up of the split kernel for R = tile_rows + 2 KS rows
// of N theta points; every section starts on a 16-byte boundary.  piv holds
// the tile rows' Thomas pivots; rt holds the step-table entries (SField) of
// the tile's positions, nodes and half nodes interleaved as in the global
// table.
struct SplitSmem {
    unsigned phi, pi, piv, rt, th, total;
};
__host__ __device__ inline unsigned smem_align16(unsigned x) { return (x + 15u) & ~15u; }
__host__ __device__ inline SplitSmem split_smem_plan(int R, int N, int tsize)
{
    SplitSmem s;
    const unsigned plane = (unsigned)R * (unsigned)N * 2u * (unsigned)tsize;
    s.phi = 0;
    s.pi = smem_align16(plane);
    s.piv = smem_align16(s.pi + plane);
    s.rt = s.piv;   // no pivot plane: the row solves read the pivots from global memory (L2)
    s.th = smem_align16(s.rt + (unsigned)(2 * R - 1) * NSF * (unsigned)tsize);
    s.total = smem_align16(s.th + (unsigned)NTF * (unsigned)N * (unsigned)tsize);
    return s;
}

// Shared-memory carve-up of the persistent split kernel: theta tables, a
// copy of the extraction row (state and step-table entry) and two tile
// buffers, each with the two state planes [R][N], the pivots [R][N] and the
// interleaved step-table entries [2R-1][NSF].
struct PersistSmem {
    unsigned th, xphi, xpi, xf, buf, bpi, bpiv, brt, bsize, total;
};
__host__ __device__ inline PersistSmem persist_smem_plan(int R, int N, int tsize)
{
    PersistSmem s;
    const unsigned c2 = 2u * (unsigned)tsize, plane = (unsigned)R * (unsigned)N * c2;
    s.th = 0;
    s.xphi = smem_align16((unsigned)NTF * (unsigned)N * (unsigned)tsize);
    s.xpi = smem_align16(s.xphi + (unsigned)N * c2);
    s.xf = smem_align16(s.xpi + (unsigned)N * c2);
    s.buf = smem_align16(s.xf + NSF * (unsigned)tsize);
    s.bpi = smem_align16(plane);
    s.bpiv = smem_align16(s.bpi + plane);
    s.brt = smem_align16(s.bpiv + plane);
    s.bsize = smem_align16(s.brt + (unsigned)(2 * R - 1) * NSF * (unsigned)tsize);
    s.total = s.buf + 2u * s.bsize;
    return s;
}

// Shared-memory carve-up of the pipelined split kernel (two steps per
// launch, persistent CTAs): theta tables, a copy of the extraction row, then
// two tile buffers of R = tile_rows + 4 rows, each with the state planes
// and pivots [R][N], the step-table entries of the tile's positions
// [2R][NSF] and the scan plans of its rows (R + 8 ints, the copy starts on
// a 16-byte boundary of the global plan array).
struct PipeSmem {
    unsigned th, xphi, xpi, buf, pi, piv, st, plan, bsize, total;
};
__host__ __device__ inline PipeSmem pipe_smem_plan(int R, int N, int tsize)
{
    PipeSmem s;
    const unsigned c2 = 2u * (unsigned)tsize, plane = (unsigned)R * (unsigned)N * c2;
    s.th = 0;
    s.xphi = smem_align16((unsigned)NTF * (unsigned)N * (unsigned)tsize);
    s.xpi = smem_align16(s.xphi + (unsigned)N * c2);
    s.buf = smem_align16(s.xpi + (unsigned)N * c2);
    s.pi = smem_align16(plane);
    s.piv = smem_align16(s.pi + plane);
    s.st = s.piv;   // no pivot plane: the row solves read the pivots from global memory (L2)
    s.plan = smem_align16(s.st + 2u * (unsigned)R * NSF * (unsigned)tsize);
    s.bsize = smem_align16(s.plan + ((unsigned)R + 8u) * 4u);
    s.total = s.buf + 2u * s.bsize;
    return s;
}

// ---------------------------------------------------------------- host side
struct Layout {
    size_t rtab64, rtabT, stab, dstab, th64, thT, piv, pivh, plan, planh, seg, segh, patch, patchu, w, ctl, staging,
        scratch;
    size_t mat, mat_bytes;   // materialised coefficients (FP64 split scheme; 0 bytes otherwise)
    size_t total;
    size_t staging_elems;    // complex doubles that fit in the staging area
};

Layout make_layout(const teuk_grid_desc &d);

// Launchers (defined in teuk_coef.cu and teuk_step.cu).
cudaError_t launch_coef_tables(const teuk_grid_desc &d, double drs, double dt, void *coef,
                               const Layout &L, cudaStream_t st);
cudaError_t launch_patch(const teuk_grid_desc &d, double drs, void *coef, const Layout &L,
                         int p0, int np, double amp_re, double amp_im, double rs0,
                         double sig_r, double sig_th, cudaStream_t st);
cudaError_t launch_set_ctl(void *coef, const Layout &L, long long step, int clear_flags,
                           cudaStream_t st);
// Source factors in the step and theta tables (SField, TField): positions
// 2 p0 .. 2 (p0 + np) - 1 get the radial factor, every other position zero.
cudaError_t launch_src_fields(const teuk_grid_desc &d, double drs, void *coef, const Layout &L, int p0, int np,
                              double amp_re, double amp_im, double rs0, double sig_r, double sig_th,
                              double drs0_da, cudaStream_t st);
// d r*/d a at fixed Boyer-Lindquist r (Eq. 2 with the usual constant), x = r - r_+.
double host_drstar_da(double M, double a, double x);

// Adjoint and operator entry points (teuk_step.cu).
template <typename T>
cudaError_t launch_apply_step(const StepParams<T> &p, int threads, size_t smem, cudaStream_t st);
template <typename T>
cudaError_t launch_sample(const StepParams<T> &p, const typename V2<T>::t *s, int physical, double2 *h_out,
                          cudaStream_t st);
template <typename T>
cudaError_t launch_adjoint_step(const StepParams<T> &p, int tile_rows, const double2 *gseed, double *part,
                                double *acc, cudaStream_t st);
template <typename T>
size_t adjoint_smem_bytes(int tile_rows, int Nth);
// The adjoint step with the spin derivative (k_adjoint_spin): sin = s_n,
// per-CTA parts of six sums, acc[0 .. 5] += their totals (acc[4]: the spin
// term).
template <typename T>
size_t adjoint_spin_smem_bytes(int tile_rows, int Nth);
// A: the context's adjoint planes (read for the full steps; a first step,
// of length dt/2, forms its coefficients from the tables).  tape: the
// forward step's record (tape_* above) whose stage values replace their
// recomputation from sin (NULL: recompute).
template <typename T>
cudaError_t launch_adjoint_spin(const StepParams<T> &p, int tile_rows, const typename V2<T>::t *sin,
                                const typename V2<T>::t *tape, const double2 *gseed, const AdjPlanes<T> &A,
                                double *part, double *acc, cudaStream_t st);
// The adjoint step without the spin term through the FP64 coefficient
// planes (the same lam_n and source sums as launch_adjoint_step up to
// rounding; full steps of FP64 contexts only).
template <typename T>
cudaError_t launch_adjoint_planes(const StepParams<T> &p, int tile_rows, const double2 *gseed, const AdjPlanes<T> &A,
                                  double *part, double *acc, cudaStream_t st);
template <typename T>
int adjoint_grid(int Nr, int tile_rows);
template <typename T>
cudaError_t launch_dot(const typename V2<T>::t *x, const typename V2<T>::t *y, const typename V2<T>::t *z,
                       size_t n, double *part, double2 *out, cudaStream_t st);

template <typename T>
cudaError_t launch_split_step(const StepParams<T> &p, int threads, size_t smem, cudaStream_t st);
template <typename T>
cudaError_t launch_literal_step(const StepParams<T> &p, cudaStream_t st);
template <typename T>
cudaError_t launch_literal_step_static(const StepParams<T> &p, long long n, cudaStream_t st);
size_t literal_static_scratch_bytes();
template <typename T>
cudaError_t launch_extract(const StepParams<T> &p, const typename V2<T>::t *u, long long step,
                           cudaStream_t st);
template <typename T>
size_t split_smem_bytes(int tile_rows, int Nth);
// Persistent split kernel (one producer warp moves tiles by TMA into two
// buffers while nc consumer threads compute): available for the FP32 state
// with Ntheta <= 128 and nc in {384, 480}.
template <typename T>
bool persist_available(int Nth, int nc);
template <typename T>
size_t persist_smem_bytes(int tile_rows, int Nth);
template <typename T>
int persist_blocks_per_sm(int Nth, int nc, size_t smem);   // 0 if the launch cannot fit
template <typename T>
void persist_explain(int Nth, int nc, size_t smem, char *buf, size_t len);   // why it cannot
template <typename T>
cudaError_t launch_split_persist(const StepParams<T> &p, int nc, int grid, size_t smem, cudaStream_t st);
template <typename T>
int split_blocks_per_sm(int Nth, int threads, size_t smem);   // 0 if the launch cannot fit
// Two time steps per launch (k_split_step2): tile of tile_rows output rows
// with two halo rows on either side.  Full steps only (not the first step
// from a physical state, not the state output).
template <typename T>
size_t split2_smem_bytes(int tile_rows, int Nth);
template <typename T>
int split2_blocks_per_sm(int Nth, int threads, size_t smem);
template <typename T>
cudaError_t launch_split_step2(const StepParams<T> &p, int threads, size_t smem, cudaStream_t st);
// The same with three time steps per launch (tiles of tile_rows + 6 rows).
template <typename T>
size_t split3_smem_bytes(int tile_rows, int Nth);
template <typename T>
int split3_blocks_per_sm(int Nth, int threads, size_t smem);
template <typename T>
cudaError_t launch_split_step3(const StepParams<T> &p, int threads, size_t smem, cudaStream_t st);
// Scan levels of every row's implicit solves for the steps dt (p.full) and
// dt/2 (p.half), written to plan_full / plan_half ([Nr] ints each).
template <typename T>
cudaError_t launch_scan_plans(const StepParams<T> &p, int *plan_full, int *plan_half, typename V2<T>::t *seg_full,
                              typename V2<T>::t *seg_half, cudaStream_t st);
// Pipelined split kernel: two time steps per launch, `grid` persistent CTAs
// of `threads` (256, or 512 for Ntheta <= 256) walk the tiles, each
// double-buffering them in shared memory (the next tile's copies land while
// the current one computes).  Full steps only, bulk-copyable rows (p.bulk).
template <typename T>
size_t pipe_smem_bytes(int tile_rows, int Nth);
template <typename T>
int pipe_blocks_per_sm(int Nth, int threads, size_t smem);
template <typename T>
cudaError_t launch_split_pipe(const StepParams<T> &p, int threads, int grid, size_t smem, cudaStream_t st);
// Materialised coefficients of the FP64 path into p.mat (no-op unless p.mat_on).
template <typename T>
cudaError_t launch_mat_coef(const StepParams<T> &p, cudaStream_t st);
// The same planes, plus the spin derivatives where o.dlw / o.dimp are set,
// into o (either precision).
template <typename T>
cudaError_t launch_mat_coef_to(const StepParams<T> &p, const MatOut<T> &o, cudaStream_t st);
// Largest tile height of the split kernels (rows of the per-tile plan copy).
constexpr int kMaxTileRows = 254;
// Batched split step: one CTA of 256 threads per entry of the tile list
// (instance, tile); params[instance] describes the instance's step.  Every
// instance must use the theta segment `seg` (implicit_seg of its Ntheta).
// ks = 2 advances every instance by two steps per launch (no first steps);
// it exists for segments of up to 8 elements only (split_batch_available).
template <typename T>
int split_batch_blocks_per_sm(int seg, size_t smem, int ks);
template <typename T>
cudaError_t launch_split_batch(const StepParams<T> *d_params, const int2 *d_tiles, int ntiles, int seg, size_t smem,
                               int ks, cudaStream_t st);
constexpr int kSegNarrow = 4;           // theta elements per thread (Ntheta <= 128)
constexpr int kSeg = 8;                 // theta elements per thread (Ntheta <= 256)
constexpr int kSegWide = 32;            // theta elements per thread (Ntheta <= 1024)
// theta elements per thread of the implicit row solves
inline int implicit_seg(int Nth) { return Nth <= 128 ? kSegNarrow : (Nth <= 256 ? kSeg : kSegWide); }
// threads per theta row (a power of two, at most a warp)
inline int implicit_group(int Nth)
{
    int seg = implicit_seg(Nth);
    int need = (Nth + seg - 1) / seg;
    int G = 1;
    while (G < need) G <<= 1;
    return G;
}
inline bool split_batch_available(int seg, int ks) { return ks == 1 || (ks == 2 && seg != kSegWide); }

cudaError_t launch_convert_to(int prec, const double2 *src, void *dst, size_t n, cudaStream_t st);
cudaError_t launch_convert_from(int prec, const void *src, double2 *dst, size_t n, cudaStream_t st);

}  // namespace teuk
