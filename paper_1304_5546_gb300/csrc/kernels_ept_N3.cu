// Order-3 instantiations of the FP32 element-thread stage kernel (uniform
// medium and per-element permittivity).
#include "kernels_ept.cuh"

namespace dgw {
template cudaError_t launch_stage_ept<3>(const StageArgs<float>&, const float*, int, int,
                                        cudaStream_t);
template cudaError_t launch_stage_ept_media<3>(const StageArgs<float>&, const float*, int, int,
                                              cudaStream_t);
}  // namespace dgw
