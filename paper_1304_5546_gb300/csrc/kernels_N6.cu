// Order-6 instantiations of the fused CUDA-core stage kernel (FP32 and
// FP64; uniform medium and per-element permittivity).
#include "kernels.cuh"

namespace dgw {
template cudaError_t launch_stage<float, 6>(const StageArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_stage<double, 6>(const StageArgs<double>&, int, int, cudaStream_t);
template cudaError_t launch_stage_media<float, 6>(const StageArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_stage_media<double, 6>(const StageArgs<double>&, int, int, cudaStream_t);
}  // namespace dgw
