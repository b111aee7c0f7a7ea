// Order-6 instantiations of the FP32 tensor-core stage kernel with 3xTF32
// products: uniform medium, per-element permittivity (each with its
// alternative element-block size where there is one), and the order's
// kernels of the concurrent batched launch.
#include "kernels_tc.cuh"

namespace dgw {
template cudaError_t launch_stage_tc<6, kTcTf32x3>(const StageArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_stage_tc_media<6>(const StageArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_batch_order<6, kModeFirstStage>(const StageArgs<float>&, int, cudaStream_t);
template cudaError_t launch_batch_order<6, kModeStage>(const StageArgs<float>&, int, cudaStream_t);
template cudaError_t launch_batch_order<6, kModeFirstStage, true>(const StageArgs<float>&, int,
                                                                   cudaStream_t);
template cudaError_t launch_batch_order<6, kModeStage, true>(const StageArgs<float>&, int,
                                                              cudaStream_t);
}  // namespace dgw
