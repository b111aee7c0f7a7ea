// Order-2 instantiation of the FP32 element-thread stage kernel.
#include "kernels_ept.cuh"

namespace dgw {
template cudaError_t launch_stage_ept<2>(const StageArgs<float>&, const float*, int, int,
                                        cudaStream_t);
}  // namespace dgw
