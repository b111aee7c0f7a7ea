// Order-7 instantiation of the FP32 tensor-core stage kernel, 3xTF32 products.
#include "kernels_tc.cuh"

namespace dgw {
template cudaError_t launch_stage_tc<7, kTcTf32x3>(const StageArgs<float>&, int, int, cudaStream_t);
}  // namespace dgw
