// Launch interface between the C ABI (api.cu) and the per-order kernel
// translation units (kernels_N*.cu).  Private to the library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace dgw {

// geometry record per element: rx ry sx sy, then per face nx ny Fscale/2
constexpr int kGeo = 13;

template <typename T>
struct StageArgs {
  int64_t K = 0;
  int64_t fstride = 0;  // elements of T between fields
  const T* qin = nullptr;
  T* qout = nullptr;
  T* res = nullptr;
  T* rhs = nullptr;
  const T* geo = nullptr;         // K x kGeo
  const int32_t* conn = nullptr;  // K x 3 face connection codes
  const T* Dr = nullptr;          // Np x Np
  const T* Ds = nullptr;          // Np x Np
  const T* LIFT = nullptr;        // Np x Nafp
  T a = 0, b = 0, dt = 0;
  int* status = nullptr;  // set to 1 by a CTA whose bounded wait expired
};

enum StageMode : int { kModeRhs = 0, kModeFirstStage = 1, kModeStage = 2 };

// One fused stage launch for order N in precision T (see kernels.cuh).
template <typename T, int N>
cudaError_t launch_stage(const StageArgs<T>& args, int mode, int num_sms, cudaStream_t stream);

}  // namespace dgw
