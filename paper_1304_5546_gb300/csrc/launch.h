// Launch interface between the C ABI (api.cu) and the per-order kernel
// translation units (kernels_N*.cu).  Private to the library.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

namespace dgw {

// Per-device, per-kernel configuration: kernel attributes such as the
// dynamic shared-memory limit are set in each device's context, so each
// launcher keeps one bit per device (ids 0..63; larger ids configure on
// every launch).  Returns cudaSuccess once configure() has succeeded on the
// current device.
template <class F>
cudaError_t configure_once_per_device(std::atomic<uint64_t>& done, F configure) {
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const uint64_t bit = dev < 64 ? (uint64_t(1) << dev) : 0;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  err = configure();
  if (err == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return err;
}

// Bits of a launch's status word (dg_sync_check): a bounded wait expired;
// a checked build (DGW_DEVICE_CHECKS) found an index it read from device
// memory out of range and skipped the access instead of making it.
constexpr int kStatusTimeout = 1, kStatusIndex = 2;

// Checked builds: a face connection code (-1, or neighbour * 8 + face * 2 +
// reversed) names a face 0..2 of an element whose Np values lie inside a
// field of fstride values.
__host__ __device__ constexpr bool nbr_code_ok(int32_t code, int64_t fstride, int Np) {
  return code < 0 || (((code >> 1) & 3) < 3 &&
                      (static_cast<int64_t>(code >> 3) + 1) * Np <= fstride);
}

// Checked builds: a block-table entry (first element k0, count n) of a
// launch with blocks of at most E elements lies inside a field of fstride
// values.
__host__ __device__ constexpr bool block_ok(int k0, int n, int E, int64_t fstride, int Np) {
  return k0 >= 0 && n >= 1 && n <= E && (static_cast<int64_t>(k0) + n) * Np <= fstride;
}

// Elements per block of the CUDA-core stage kernel (kernels.cuh): a multiple
// of 4, so every per-block chunk (E Np values, E geometry records, E
// face-code triples) is a whole number of 16-byte units as TMA requires;
// E Np <= 512 from N = 4 on, because ptxas budgets registers for the CTA
// rounded up to 4 warps and each thread needs 2 Np + Nafp registers for its
// matrix rows.
__host__ __device__ constexpr int simt_block_elems(int N, bool fp64) {
  return fp64 ? (N == 1 ? 32 : N <= 4 ? 16 : N == 5 ? 12 : 8)
              : (N == 1 ? 64 : N <= 4 ? 32 : N == 5 ? 24 : N == 6 ? 16 : 12);
}

// geometry record per element: rx ry sx sy, then per face nx ny Fscale/2
constexpr int kGeo = 13;

// Geometry record per element of an operator with a piecewise-constant
// permittivity eps_k (mu = 1; Eq. tm-maxwells with variable eps), 20 values:
//   [0, 4)          rx ry sx sy
//   [4 + 4f, 8 + 4f) face f: nx, ny, cH = Fscale Z+ / (Z- + Z+),
//                   cE = Fscale / (Z- + Z+)   (Z = 1 / sqrt(eps), '+' the
//                   neighbour, Z+ = Z- at a PEC face)
//   16              Z- of the element
//   17, 18          row scales sH (Hx, Hy rows) and sE (Ez row): the
//                   update multiplies the right-hand side by dt * s, so
//                   sH = 1, sE = 1 / eps_k for a single operator, and a
//                   batch folds each problem's own time step in
//                   (sH = dt_p, sE = dt_p / eps_k, launch dt = 1)
//   19              point source of the batched launch: source index + 1
//                   (0: none; the single-operator launches never read it)
// With these the upwind flux at a face node is, for the jumps
// [u] = u- - u+ and [Ht] = ny [Hx] - nx [Hy],
//   fz = cH [Ht] - cE [Ez];  lifted terms (-Z- ny fz, Z- nx fz, fz)
// which is Fscale n.(F - F*) of the exact interface Riemann solution, and
// for eps = 1 everywhere the eps = 1 upwind flux times Fscale / 2.
constexpr int kGeoMedia = 20;
constexpr int kSrcStride = 36;  // Np at N = 7

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
  const T* lam = nullptr;         // [2][Np]: (1 + r_n) / 2, (1 + s_n) / 2 per node
  T a = 0, b = 0, dt = 0;
  T alpha = 1;  // flux parameter of Eq. max2d-numflux (uniform medium only)
  // tensor-core kernel: compute the flux of a face whose two elements lie in
  // the same block once, for both sides (0: every face node per side)
  int face_pairs = 0;
  // tensor-core kernel with 3xTF32 products: the alternative element-block
  // size (tc_tiles(N, prec, true)) instead of the default; chosen on the host
  int tc_alt = 0;
  int* status = nullptr;  // set to 1 by a CTA whose bounded wait expired
  // timeout test only (tensor-core kernel): the memory warp first waits,
  // bounded by kGateLimitNs, for *stall_gate to become non-zero; NULL
  // otherwise
  const int* stall_gate = nullptr;
  // block table of the batched launch: block i of the launch covers
  // elements [blocks[i].x, blocks[i].x + blocks[i].y), 1 <= y <= E, x a
  // multiple of 4; the count is read from device memory (*nblocks) so that a
  // captured graph replays with a changed table.  Unused by the
  // single-operator launches (blocks of E consecutive elements over [0, K)).
  const int2* blocks = nullptr;
  const int* nblocks = nullptr;
  // point sources of the batched launch (record value 19 = index + 1):
  // the Ez right-hand side of the source element gains s(t) w, with w the
  // projected point load times the problem's dt (src_w[index][kSrcStride])
  // and s the Ricker wavelet A (1 - 2 a^2) exp(-a^2), a = pi f (t - t0),
  // from src_meta[index] = {dt, t0, pi f, A}; the stage time is
  // t = (step_ctr - src_step[index] + c_stage) dt.
  const float* src_w = nullptr;
  const double* src_meta = nullptr;
  const int* src_step = nullptr;
  const int* step_ctr = nullptr;
  double c_stage = 0.0;
  // tensor-core path only: [Dr | Ds | LIFT | 1] as the operator tiles of the
  // launch's product variant (tc_nsplit tiles of tc_nn(N) x tc_kpp(N, prec)
  // elements, TF32 or BF16, in the core-matrix layout of tc_canon /
  // tc_canon16)
  const void* tc_op = nullptr;
};

enum StageMode : int { kModeRhs = 0, kModeFirstStage = 1, kModeStage = 2 };

// One fused stage launch for order N in precision T on the CUDA cores (see
// kernels.cuh).
template <typename T, int N>
cudaError_t launch_stage(const StageArgs<T>& args, int mode, int num_sms, cudaStream_t stream);

// Tensor-core path (FP32 fields, FP32 accumulation; see kernels_tc.cuh).  The
// element-local products of a block of elements form one GEMM
//   D[3E x Np] = X[3E x KD] [Dr | Ds | LIFT | 1]^T
// whose K columns are laid out part by part, each part starting on a
// 16-byte boundary: Dr columns at [0, NPAD), Ds at [NPAD, 2 NPAD), LIFT at
// [2 NPAD, 2 NPAD + Nafp) with NPAD = Np rounded up to 4, then one column
// (2 NPAD + Nafp) whose operator entries are 1 for every node and whose X
// entry is the row's linear-part term; K is padded to tc_kpp(N, prec) (one
// MMA step: 8 TF32 or 16 BF16 elements) and N to tc_nn(N) (multiple of 16).
__host__ __device__ constexpr int tc_np(int N) { return (N + 1) * (N + 2) / 2; }
__host__ __device__ constexpr int tc_npad(int N) { return (tc_np(N) + 3) / 4 * 4; }
__host__ __device__ constexpr int tc_kd(int N) { return 2 * tc_npad(N) + 3 * (N + 1) + 1; }
__host__ __device__ constexpr int tc_kp(int N) { return (tc_kd(N) + 7) / 8 * 8; }
__host__ __device__ constexpr int tc_nn(int N) { return (tc_np(N) + 15) / 16 * 16; }
// Float index of element (row n, column k) of a K-major operand tile with kp
// columns in the no-swizzle canonical layout: 8-row x 16-byte core matrices
// of 128 contiguous bytes, K-adjacent core matrices 128 bytes apart, 8-row
// groups kp/4 * 128 bytes apart.
__host__ __device__ constexpr int tc_canon(int n, int k, int kp) {
  return ((n / 8) * (kp / 4) + k / 4) * 32 + (n % 8) * 4 + (k % 4);
}
// The same for 16-bit elements (8 per 16-byte core-matrix row); index in
// 16-bit units.
__host__ __device__ constexpr int tc_canon16(int n, int k, int kp) {
  return ((n / 8) * (kp / 8) + k / 8) * 64 + (n % 8) * 8 + (k % 8);
}

// Product variants of the tensor-core path.  FP32 fields and accumulation
// in every variant; they differ in the operand types and the number of
// products per term:
//   kTcTf32x3  X_hi Op_hi + X_hi Op_lo + X_lo Op_hi in TF32 (FP32 accuracy)
//   kTcTf32    X Op with both operands rounded to TF32
//   kTcBf16    X Op with both operands rounded to BF16
//   kTcBf16x3  X_hi Op_hi + X_hi Op_lo + X_lo Op_hi in BF16
enum TcPrecision : int { kTcTf32x3 = 0, kTcTf32 = 1, kTcBf16 = 2, kTcBf16x3 = 3 };
__host__ __device__ constexpr bool tc_is_bf16(int prec) { return prec == kTcBf16 || prec == kTcBf16x3; }
__host__ __device__ constexpr int tc_nsplit(int prec) {
  return (prec == kTcTf32x3 || prec == kTcBf16x3) ? 2 : 1;
}
// K padded to whole MMA steps: 8 TF32 or 16 BF16 elements
__host__ __device__ constexpr int tc_kpp(int N, int prec) {
  return tc_is_bf16(prec) ? (tc_kd(N) + 15) / 16 * 16 : tc_kp(N);
}
// Two 128-row GEMM tiles per element block fit the 512 tensor-memory
// columns: both tiles' double-buffered accumulators (split: two operator
// tiles' columns) and double-buffered operands (the X parts of the variant).
__host__ __device__ constexpr bool tc_two_tiles_fit(int N, int prec) {
  return 2 * 2 * (tc_nsplit(prec) == 2 ? 2 * tc_nn(N) : tc_nn(N)) +
             2 * 2 * tc_nsplit(prec) * (tc_is_bf16(prec) ? tc_kpp(N, prec) / 2 : tc_kpp(N, prec)) <=
         512;
}
// Row tiles of an element block (40 elements per tile).  The default is two
// tiles at N <= 3 where they fit (measured faster there: N = 3 0.86 -> 0.65
// ms/step, N = 2 1.31 -> 0.83) and one above (N = 4, which also fits two,
// measured 0.65 -> 0.68 with two).  alt: the other count where both fit,
// for the autotuner (dg_operator_tune, dg_batch_tune) to try on a live mesh.
__host__ __device__ constexpr int tc_tiles(int N, int prec, bool alt) {
  return (N <= 3 && tc_two_tiles_fit(N, prec)) ? (alt ? 1 : 2)
                                               : ((alt && tc_two_tiles_fit(N, prec)) ? 2 : 1);
}
__host__ __device__ constexpr bool tc_has_alt(int N, int prec) {
  return tc_tiles(N, prec, true) != tc_tiles(N, prec, false);
}

template <int N, int PREC>
cudaError_t launch_stage_tc(const StageArgs<float>& args, int mode, int num_sms,
                            cudaStream_t stream);

// Element-thread path (FP32, CUDA cores, one thread per element; see
// kernels_ept.cuh), orders 1..kEptMaxN; the _media launcher takes
// per-element-permittivity records (kGeoMedia values).  Its reference
// tables travel as a kernel parameter: `ops` points to host memory holding
// ept_ops_floats(N) floats, [Dr (Np x Np, row-major) | Ds | LIFT (Np x
// Nafp) | (1 + r_n) / 2 | (1 + s_n) / 2].
constexpr int kEptMaxN = 5;
__host__ __device__ constexpr int ept_ops_floats(int N) {
  return 2 * tc_np(N) * tc_np(N) + tc_np(N) * 3 * (N + 1) + 2 * tc_np(N);
}
template <int N>
cudaError_t launch_stage_ept(const StageArgs<float>& args, const float* ops, int mode,
                             int num_sms, cudaStream_t stream);
template <int N>
cudaError_t launch_stage_ept_media(const StageArgs<float>& args, const float* ops, int mode,
                                   int num_sms, cudaStream_t stream);

// Operators with a per-element permittivity (geometry records of kGeoMedia
// values): CUDA-core kernel (FP32 / FP64) and tensor-core kernel (3xTF32).
template <typename T, int N>
cudaError_t launch_stage_media(const StageArgs<T>& args, int mode, int num_sms,
                               cudaStream_t stream);
template <int N>
cudaError_t launch_stage_tc_media(const StageArgs<float>& args, int mode, int num_sms,
                                  cudaStream_t stream);

// Batched launch: one persistent launch over the problems of a batch, all
// orders at once.  Group g (order N = g + 1) runs on CTAs
// [cta0[g], cta0[g + 1]) over its own block table; groups without CTAs are
// skipped.  Media records, 3xTF32 products, LSRK stage modes only.
// The CTA ranges are read from device memory (cta0[0..7]) so that a
// captured graph replays with a changed split.
struct BatchArgs {
  StageArgs<float> g[7];
  const int* cta0 = nullptr;
  // tuning launches only: CTA b writes its start and end time (globaltimer,
  // ns) to cta_clock[2b], cta_clock[2b + 1]; NULL otherwise
  unsigned long long* cta_clock = nullptr;
};
// grid: CTAs of the launch (cta0[7]); smem: the largest
// batch_tc_smem_bytes of an order that may have CTAs
template <int MODE>
cudaError_t launch_batch_tc(const BatchArgs& args, int grid, size_t smem, cudaStream_t stream);
// The concurrent mode of the batched launch: order N's share of a stage as a
// kernel of its own, `grid` CTAs (one per SM) over its block table
// (g.blocks, g.nblocks); grid 0 only configures the kernel.
template <int N, int MODE, bool ALT = false>
cudaError_t launch_batch_order(const StageArgs<float>& g, int grid, cudaStream_t stream);
// shared memory and elements per block of order N's CTA in the batched launch
// (alt: the alternative block size of the concurrent mode's kernels)
size_t batch_tc_smem_bytes(int N, bool alt = false);
int batch_tc_block_elems(int N, bool alt = false);

}  // namespace dgw
