// Order-2 instantiations of the tensor-core stage kernel's other product
// variants: one TF32 product, one BF16 product, three BF16 products.
#include "kernels_tc.cuh"

namespace dgw {
template cudaError_t launch_stage_tc<2, kTcTf32>(const StageArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_stage_tc<2, kTcBf16>(const StageArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_stage_tc<2, kTcBf16x3>(const StageArgs<float>&, int, int, cudaStream_t);
}  // namespace dgw
