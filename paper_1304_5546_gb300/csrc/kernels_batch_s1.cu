// Batched multi-order tensor-core launch, first LSRK stage (a_1 = 0: the
// residual is not read), and the shared-memory size and elements per block
// of each order's CTA.
#include "kernels_tc.cuh"

namespace dgw {

size_t batch_tc_smem_bytes(int N) {
  switch (N) {
    case 1: return TcLayout<1, kTcTf32x3, true>::SMEM_BYTES;
    case 2: return TcLayout<2, kTcTf32x3, true>::SMEM_BYTES;
    case 3: return TcLayout<3, kTcTf32x3, true>::SMEM_BYTES;
    case 4: return TcLayout<4, kTcTf32x3, true>::SMEM_BYTES;
    case 5: return TcLayout<5, kTcTf32x3, true>::SMEM_BYTES;
    case 6: return TcLayout<6, kTcTf32x3, true>::SMEM_BYTES;
    case 7: return TcLayout<7, kTcTf32x3, true>::SMEM_BYTES;
    default: return 0;
  }
}

int batch_tc_block_elems(int N) {
  switch (N) {
    case 1: return TcLayout<1, kTcTf32x3, true>::E;
    case 2: return TcLayout<2, kTcTf32x3, true>::E;
    case 3: return TcLayout<3, kTcTf32x3, true>::E;
    case 4: return TcLayout<4, kTcTf32x3, true>::E;
    case 5: return TcLayout<5, kTcTf32x3, true>::E;
    case 6: return TcLayout<6, kTcTf32x3, true>::E;
    case 7: return TcLayout<7, kTcTf32x3, true>::E;
    default: return 0;
  }
}

template cudaError_t launch_batch_tc<kModeFirstStage>(const BatchArgs&, int, size_t, cudaStream_t);

}  // namespace dgw
