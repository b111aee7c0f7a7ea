// Batched multi-order tensor-core launch, LSRK stages 2..5.
#include "kernels_tc.cuh"

namespace dgw {
template cudaError_t launch_batch_tc<kModeStage>(const BatchArgs&, int, size_t, cudaStream_t);
}  // namespace dgw
