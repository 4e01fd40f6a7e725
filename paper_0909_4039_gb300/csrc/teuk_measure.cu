// teuk_measure.cu -- the FMA throughput of the current GPU in FP64 or FP32,
// the denominator of the ALU roofline of a step kernel.  The FP64 path is
// bound by the FP64 pipe (the paper requires double precision for these
// evolutions, Sec. 4 and the single- versus double-precision remark of
// Sec. 5.2), so its fraction of this measured rate is what says how close
// it runs to its ceiling.
#include <cuda_runtime.h>

#include "teuk_internal.cuh"

namespace teuk {
namespace {

constexpr int kChains = 8;   // independent FMA chains per thread

// Each thread runs kChains independent chains x <- a x + b for `iters`
// rounds; the result is stored only if it equals an impossible value, so the
// loop is kept but no memory traffic is added.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_rate(T *sink, int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (T)(threadIdx.x + k) * T(1e-3);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(a, x[k], b);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == T(-1.2345e30)) *sink = s;
}

template <typename T>
cudaError_t run_rate(T *sink, int iters, cudaStream_t st, double *flops)
{
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int block = 256, grid = nsm * 8;
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    k_fma_rate<T><<<grid, block, 0, st>>>(sink, iters / 8 + 1, T(0.999999), T(1e-7));   // warm-up
    cudaEventRecord(e0, st);
    k_fma_rate<T><<<grid, block, 0, st>>>(sink, iters, T(0.999999), T(1e-7));
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    const double fmas = (double)grid * block * kChains * (double)iters;
    *flops = 2.0 * fmas / ((double)ms * 1e-3);
    return cudaSuccess;
}

}  // namespace
}  // namespace teuk

extern "C" int teuk_fma_rate(int precision, int iters, void *d_sink, void *stream, double *flops_per_s)
{
    using namespace teuk;
    if (!flops_per_s || !d_sink || iters < 1 || (precision != TEUK_FP64 && precision != TEUK_FP32))
        return TEUK_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = precision == TEUK_FP64 ? run_rate<double>((double *)d_sink, iters, st, flops_per_s)
                                           : run_rate<float>((float *)d_sink, iters, st, flops_per_s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return TEUK_E_CUDA;
    }
    return TEUK_OK;
}
