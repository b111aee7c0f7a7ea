// Batched multi-order tensor-core launch, first LSRK stage (a_1 = 0: the
// residual is not read), and the shared-memory size and elements per block
// of each order's CTA.
#include "kernels_tc.cuh"

namespace dgw {

size_t batch_tc_smem_bytes(int N, bool alt) {
#define DG_SMEM_CASE(NN_)                                                           \
  case NN_:                                                                         \
    return alt ? TcLayout<NN_, kTcTf32x3, true, true>::SMEM_BYTES                   \
               : TcLayout<NN_, kTcTf32x3, true>::SMEM_BYTES;
  switch (N) {
    DG_SMEM_CASE(1)
    DG_SMEM_CASE(2)
    DG_SMEM_CASE(3)
    DG_SMEM_CASE(4)
    DG_SMEM_CASE(5)
    DG_SMEM_CASE(6)
    DG_SMEM_CASE(7)
    default: return 0;
  }
#undef DG_SMEM_CASE
}

// elements per block; alt: the alternative size (the default where an order
// has none)
int batch_tc_block_elems(int N, bool alt) {
#define DG_ELEMS_CASE(NN_)                                                          \
  case NN_:                                                                         \
    return alt ? TcLayout<NN_, kTcTf32x3, true, true>::E : TcLayout<NN_, kTcTf32x3, true>::E;
  switch (N) {
    DG_ELEMS_CASE(1)
    DG_ELEMS_CASE(2)
    DG_ELEMS_CASE(3)
    DG_ELEMS_CASE(4)
    DG_ELEMS_CASE(5)
    DG_ELEMS_CASE(6)
    DG_ELEMS_CASE(7)
    default: return 0;
  }
#undef DG_ELEMS_CASE
}

template cudaError_t launch_batch_tc<kModeFirstStage>(const BatchArgs&, int, size_t, cudaStream_t);

}  // namespace dgw
