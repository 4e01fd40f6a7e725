// teuk_split_f32.cu -- the split-scheme step kernels and launchers for the FP32 state.
#include "teuk_split.cuh"

namespace teuk {

template cudaError_t launch_apply_step<float>(const StepParams<float> &, int, size_t, cudaStream_t);
template cudaError_t launch_scan_plans<float>(const StepParams<float> &, int *, int *, float2 *, float2 *,
                                               cudaStream_t);
template int split_batch_blocks_per_sm<float>(int, size_t, int);
template cudaError_t launch_split_batch<float>(const StepParams<float> *, const int2 *, int, int, size_t, int,
                                               cudaStream_t);
template size_t split2_smem_bytes<float>(int, int);
template int split2_blocks_per_sm<float>(int, int, size_t);
template cudaError_t launch_split_step2<float>(const StepParams<float> &, int, size_t, cudaStream_t);
template size_t split3_smem_bytes<float>(int, int);
template int split3_blocks_per_sm<float>(int, int, size_t);
template cudaError_t launch_split_step3<float>(const StepParams<float> &, int, size_t, cudaStream_t);
template int split_blocks_per_sm<float>(int, int, size_t);
template size_t split_smem_bytes<float>(int, int);
template cudaError_t launch_split_step<float>(const StepParams<float> &, int, size_t, cudaStream_t);
template cudaError_t launch_mat_coef<float>(const StepParams<float> &, cudaStream_t);
template cudaError_t launch_mat_coef_to<float>(const StepParams<float> &, const MatOut<float> &, cudaStream_t);
template size_t pipe_smem_bytes<float>(int, int);
template int pipe_blocks_per_sm<float>(int, int, size_t);
template cudaError_t launch_split_pipe<float>(const StepParams<float> &, int, int, size_t, cudaStream_t);

}  // namespace teuk
