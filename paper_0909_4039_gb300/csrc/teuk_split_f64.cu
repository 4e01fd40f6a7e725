// teuk_split_f64.cu -- the split-scheme step kernels and launchers for the FP64 state.
#include "teuk_split.cuh"

namespace teuk {

template cudaError_t launch_apply_step<double>(const StepParams<double> &, int, size_t, cudaStream_t);
template cudaError_t launch_scan_plans<double>(const StepParams<double> &, int *, int *, double2 *, double2 *,
                                               cudaStream_t);
template int split_batch_blocks_per_sm<double>(int, size_t, int);
template cudaError_t launch_split_batch<double>(const StepParams<double> *, const int2 *, int, int, size_t, int,
                                                cudaStream_t);
template size_t split2_smem_bytes<double>(int, int);
template int split2_blocks_per_sm<double>(int, int, size_t);
template cudaError_t launch_split_step2<double>(const StepParams<double> &, int, size_t, cudaStream_t);
template size_t split3_smem_bytes<double>(int, int);
template int split3_blocks_per_sm<double>(int, int, size_t);
template cudaError_t launch_split_step3<double>(const StepParams<double> &, int, size_t, cudaStream_t);
template int split_blocks_per_sm<double>(int, int, size_t);
template size_t split_smem_bytes<double>(int, int);
template cudaError_t launch_split_step<double>(const StepParams<double> &, int, size_t, cudaStream_t);
template cudaError_t launch_mat_coef<double>(const StepParams<double> &, cudaStream_t);
template cudaError_t launch_mat_coef_to<double>(const StepParams<double> &, const MatOut<double> &, cudaStream_t);
template size_t pipe_smem_bytes<double>(int, int);
template int pipe_blocks_per_sm<double>(int, int, size_t);
template cudaError_t launch_split_pipe<double>(const StepParams<double> &, int, int, size_t, cudaStream_t);

}  // namespace teuk
