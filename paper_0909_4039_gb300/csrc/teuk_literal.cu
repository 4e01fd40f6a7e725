// teuk_literal.cu -- the literal scheme (all of S inside the Lax-Wendroff
// stages of Eqs. 12-14), its allocation-free variant with a static scratch
// array, the one-row extraction kernel and the FP64 <-> FP32 state
// conversions.
#include "teuk_dev.cuh"

namespace teuk {
namespace {

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


template cudaError_t launch_literal_step_static<float>(const StepParams<float> &, long long, cudaStream_t);
template cudaError_t launch_literal_step_static<double>(const StepParams<double> &, long long, cudaStream_t);
template cudaError_t launch_literal_step<float>(const StepParams<float> &, cudaStream_t);
template cudaError_t launch_literal_step<double>(const StepParams<double> &, cudaStream_t);
template cudaError_t launch_extract<float>(const StepParams<float> &, const float2 *, long long, cudaStream_t);
template cudaError_t launch_extract<double>(const StepParams<double> &, const double2 *, long long, cudaStream_t);

}  // namespace teuk
