// Order-3 instantiation of the fused stage kernel (FP32 and FP64).
#include "kernels.cuh"

namespace dgw {
template cudaError_t launch_stage<float, 3>(const StageArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_stage<double, 3>(const StageArgs<double>&, int, int, cudaStream_t);
}  // namespace dgw
