// C ABI of the nodal DG wave solver: operator set-up and upload, and the
// hot-path entry points dg_rhs / dg_step / dg_solve / dg_step_host.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "launch.h"

namespace dgw {
const char* last_error_cstr();
std::atomic<int> g_fail_alloc{0};
}

using dgw::fail;

namespace {

// K is padded to whole blocks of <= 64 elements plus at least one spare
// element: the kernels' bulk copies round each block's chunks up to 16 bytes
constexpr int64_t kBlockPad = 64;

dg_status cuda_fail(cudaError_t err, const char* where) {
  return fail(err == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA, "%s: %s (%s)", where,
              cudaGetErrorName(err), cudaGetErrorString(err));
}

void free_device(dg_op* op) {
  void* ptrs[] = {op->d_Dr,   op->d_Ds,     op->d_LIFT, op->d_geo, op->d_conn,    op->d_qtmp,
                  op->d_flag, op->d_status, op->d_tcop, op->d_lam, op->d_src_w};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  op->d_src_w = nullptr;
  op->d_Dr = op->d_Ds = op->d_LIFT = op->d_geo = op->d_conn = op->d_qtmp = nullptr;
  op->d_flag = nullptr;
  op->d_status = nullptr;
  op->d_tcop = nullptr;
  op->d_lam = nullptr;
}

// TF32 value nearest to v (ties away from zero), as a float with its 13 low
// mantissa bits clear.
float tf32_round(double v) {
  float f = static_cast<float>(v);
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  std::memcpy(&f, &u, 4);
  return f;
}

// BF16 value nearest to v (ties to even), as its 16-bit pattern.
uint16_t bf16_round(double v) {
  const float f = static_cast<float>(v);
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return static_cast<uint16_t>(u >> 16);
}
double bf16_value(uint16_t h) {
  const uint32_t u = static_cast<uint32_t>(h) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

}  // namespace

namespace dgw {

// [Dr | Ds | LIFT | 1] as the B operand of the tensor-core kernel, in the
// operand format of product variant `prec`: nsplit tiles (hi, then lo for
// the split variants, v ~ hi + lo, split in FP64), each nn x kpp elements in
// the core-matrix layout of dgw::tc_canon (TF32, 4 bytes) or dgw::tc_canon16
// (BF16, 2 bytes), parts at the columns dgw::tc_kd describes; rows >= Np and
// padding columns are zero.  Returned as bytes.
std::vector<unsigned char> tc_operator_tiles(const dgw::RefElement& R, int prec) {
  const int N = R.N, Np = R.Np, Nafp = R.Nafp;
  const int kp = dgw::tc_kpp(N, prec), nn = dgw::tc_nn(N), npad = dgw::tc_npad(N);
  const int ns = dgw::tc_nsplit(prec);
  const bool bf = dgw::tc_is_bf16(prec);
  const size_t tile = static_cast<size_t>(nn) * kp;  // elements per tile
  std::vector<unsigned char> out(ns * tile * (bf ? 2 : 4), 0);
  float* f32 = reinterpret_cast<float*>(out.data());
  uint16_t* b16 = reinterpret_cast<uint16_t*>(out.data());
  auto put = [&](int n, int k, double v) {
    if (bf) {
      const int idx = dgw::tc_canon16(n, k, kp);
      const uint16_t hi = bf16_round(v);
      b16[idx] = hi;
      if (ns == 2) b16[tile + idx] = bf16_round(v - bf16_value(hi));
    } else {
      const int idx = dgw::tc_canon(n, k, kp);
      const float hi = tf32_round(v);
      f32[idx] = hi;
      if (ns == 2) f32[tile + idx] = tf32_round(v - static_cast<double>(hi));
    }
  };
  for (int n = 0; n < Np; ++n) {
    for (int m = 0; m < Np; ++m) {
      put(n, m, R.Dr[n * Np + m]);
      put(n, npad + m, R.Ds[n * Np + m]);
    }
    for (int j = 0; j < Nafp; ++j) put(n, 2 * npad + j, R.LIFT[n * Nafp + j]);
    put(n, 2 * npad + Nafp, 1.0);  // carries each row's linear-part term to every node
  }
  return out;
}

void media_records(const dg_op& op, double sh, std::vector<double>& out) {
  const int64_t K = op.K;
  constexpr int R = kGeoMedia;
  out.assign(static_cast<size_t>(K) * R, 0.0);
  auto eps_of = [&](int64_t k) { return op.media() ? op.eps[k] : 1.0; };
  for (int64_t k = 0; k < K; ++k) {
    double* g = &out[k * R];
    g[0] = op.geo.rx[k];
    g[1] = op.geo.ry[k];
    g[2] = op.geo.sx[k];
    g[3] = op.geo.sy[k];
    const double zM = 1.0 / std::sqrt(eps_of(k));
    for (int f = 0; f < 3; ++f) {
      const int32_t code = op.geo.conn[3 * k + f];
      const double zP = code < 0 ? zM : 1.0 / std::sqrt(eps_of(code >> 3));
      const double fsc = op.geo.Fscale[3 * k + f];
      g[4 + 4 * f] = op.geo.nx[3 * k + f];
      g[5 + 4 * f] = op.geo.ny[3 * k + f];
      g[6 + 4 * f] = fsc * zP / (zM + zP);
      g[7 + 4 * f] = fsc / (zM + zP);
    }
    g[16] = zM;
    g[17] = sh;
    g[18] = sh / eps_of(k);
  }
}

}  // namespace dgw

namespace dgw {

void operator_records(const dg_op& op, std::vector<double>& rec, std::vector<int32_t>& conn) {
  const int64_t K = op.K;
  if (op.media()) {
    media_records(op, 1.0, rec);
  } else {
    rec.assign(static_cast<size_t>(K) * kGeo, 0.0);
    for (int64_t k = 0; k < K; ++k) {
      double* g = &rec[k * kGeo];
      g[0] = op.geo.rx[k];
      g[1] = op.geo.ry[k];
      g[2] = op.geo.sx[k];
      g[3] = op.geo.sy[k];
      for (int f = 0; f < 3; ++f) {
        g[4 + 3 * f] = op.geo.nx[3 * k + f];
        g[5 + 3 * f] = op.geo.ny[3 * k + f];
        g[6 + 3 * f] = 0.5 * op.geo.Fscale[3 * k + f];
      }
    }
  }
  conn.assign(op.geo.conn.begin(), op.geo.conn.begin() + 3 * K);
}

}  // namespace dgw

namespace {

using dgw::tc_operator_tiles;

template <typename T>
dg_status upload(dg_op* op, const std::vector<double>& rec_in,
                 const std::vector<int32_t>& conn_in) {
  const int Np = op->Np, Nafp = op->Nafp;
  const int64_t K = op->K, Kpad = op->Kpad;
  std::vector<T> Dr(op->ref.Dr.begin(), op->ref.Dr.end());
  std::vector<T> Ds(op->ref.Ds.begin(), op->ref.Ds.end());
  std::vector<T> LIFT(op->ref.LIFT.begin(), op->ref.LIFT.end());
  // barycentric weights of vertices 2 and 3 at every node: the linear
  // interpolant through the vertex nodes is u1 + (u2 - u1) lam2 + (u3 - u1) lam3
  std::vector<T> lam(2 * static_cast<size_t>(Np));
  for (int n = 0; n < Np; ++n) {
    lam[n] = static_cast<T>(0.5 * (1.0 + op->ref.r[n]));
    lam[Np + n] = static_cast<T>(0.5 * (1.0 + op->ref.s[n]));
  }
  // the element-thread kernel's reference tables, FP32 (launch.h,
  // ept_ops_floats): the same roundings as the device copies above
  op->ept_ops.clear();
  if (sizeof(T) == 4 && op->N <= dgw::kEptMaxN) {
    for (double v : op->ref.Dr) op->ept_ops.push_back(static_cast<float>(v));
    for (double v : op->ref.Ds) op->ept_ops.push_back(static_cast<float>(v));
    for (double v : op->ref.LIFT) op->ept_ops.push_back(static_cast<float>(v));
    for (int n = 0; n < 2 * Np; ++n) op->ept_ops.push_back(static_cast<float>(lam[n]));
  }
  // records padded to Kpad elements: zero geometry, boundary faces
  const int rec = op->media() ? dgw::kGeoMedia : dgw::kGeo;
  std::vector<T> geo(static_cast<size_t>(Kpad) * rec, T(0));
  std::vector<int32_t> conn(static_cast<size_t>(Kpad) * 3, -1);
  for (size_t i = 0; i < static_cast<size_t>(K) * rec; ++i) geo[i] = static_cast<T>(rec_in[i]);
  std::copy(conn_in.begin(), conn_in.begin() + 3 * K, conn.begin());
  struct Up {
    void** dst;
    const void* src;
    size_t bytes;
  } ups[] = {
      {&op->d_Dr, Dr.data(), Dr.size() * sizeof(T)},
      {&op->d_Ds, Ds.data(), Ds.size() * sizeof(T)},
      {&op->d_LIFT, LIFT.data(), LIFT.size() * sizeof(T)},
      {&op->d_lam, lam.data(), lam.size() * sizeof(T)},
      {&op->d_geo, geo.data(), geo.size() * sizeof(T)},
      {&op->d_conn, conn.data(), conn.size() * sizeof(int32_t)},
  };
  for (const Up& u : ups) {
    cudaError_t err = dgw::dev_malloc(u.dst, u.bytes);
    if (err != cudaSuccess) return cuda_fail(err, "dg_operator_setup: cudaMalloc");
    err = cudaMemcpy(*u.dst, u.src, u.bytes, cudaMemcpyHostToDevice);
    if (err != cudaSuccess) return cuda_fail(err, "dg_operator_setup: cudaMemcpy");
  }
  cudaError_t err = dgw::dev_malloc(&op->d_qtmp, 3 * op->fstride * sizeof(T));
  if (err != cudaSuccess) return cuda_fail(err, "dg_operator_setup: cudaMalloc(field buffer)");
  err = cudaMemset(op->d_qtmp, 0, 3 * op->fstride * sizeof(T));
  if (err != cudaSuccess) return cuda_fail(err, "dg_operator_setup: cudaMemset");
  err = dgw::dev_malloc(&op->d_flag, sizeof(int));
  if (err != cudaSuccess) return cuda_fail(err, "dg_operator_setup: cudaMalloc(flag)");
  if (op->use_tc) {
    const std::vector<unsigned char> tiles = tc_operator_tiles(op->ref, op->tc_prec);
    err = dgw::dev_malloc(&op->d_tcop, tiles.size());
    if (err != cudaSuccess) return cuda_fail(err, "dg_operator_setup: cudaMalloc(operator tiles)");
    err = cudaMemcpy(op->d_tcop, tiles.data(), tiles.size(), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) return cuda_fail(err, "dg_operator_setup: cudaMemcpy(operator tiles)");
  }
  err = dgw::dev_malloc(&op->d_status, sizeof(int));
  if (err != cudaSuccess) return cuda_fail(err, "dg_operator_setup: cudaMalloc(status)");
  err = cudaMemset(op->d_status, 0, sizeof(int));
  if (err != cudaSuccess) return cuda_fail(err, "dg_operator_setup: cudaMemset(status)");
  (void)Np;
  (void)Nafp;
  return DG_OK;
}

template <int N>
cudaError_t launch_prec_tc(const dg_op* op, const dgw::StageArgs<float>& a, int mode,
                           cudaStream_t s) {
  switch (op->tc_prec) {
    case dgw::kTcTf32x3: return dgw::launch_stage_tc<N, dgw::kTcTf32x3>(a, mode, op->num_sms, s);
    case dgw::kTcTf32: return dgw::launch_stage_tc<N, dgw::kTcTf32>(a, mode, op->num_sms, s);
    case dgw::kTcBf16: return dgw::launch_stage_tc<N, dgw::kTcBf16>(a, mode, op->num_sms, s);
    case dgw::kTcBf16x3: return dgw::launch_stage_tc<N, dgw::kTcBf16x3>(a, mode, op->num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_order_tc(const dg_op* op, const dgw::StageArgs<float>& a, int mode,
                            cudaStream_t s) {
  switch (op->N) {
    case 1: return launch_prec_tc<1>(op, a, mode, s);
    case 2: return launch_prec_tc<2>(op, a, mode, s);
    case 3: return launch_prec_tc<3>(op, a, mode, s);
    case 4: return launch_prec_tc<4>(op, a, mode, s);
    case 5: return launch_prec_tc<5>(op, a, mode, s);
    case 6: return launch_prec_tc<6>(op, a, mode, s);
    case 7: return launch_prec_tc<7>(op, a, mode, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_order_tc_media(const dg_op* op, const dgw::StageArgs<float>& a, int mode,
                                  cudaStream_t s) {
  switch (op->N) {
    case 1: return dgw::launch_stage_tc_media<1>(a, mode, op->num_sms, s);
    case 2: return dgw::launch_stage_tc_media<2>(a, mode, op->num_sms, s);
    case 3: return dgw::launch_stage_tc_media<3>(a, mode, op->num_sms, s);
    case 4: return dgw::launch_stage_tc_media<4>(a, mode, op->num_sms, s);
    case 5: return dgw::launch_stage_tc_media<5>(a, mode, op->num_sms, s);
    case 6: return dgw::launch_stage_tc_media<6>(a, mode, op->num_sms, s);
    case 7: return dgw::launch_stage_tc_media<7>(a, mode, op->num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_order_ept_media(const dg_op* op, const dgw::StageArgs<float>& a, int mode,
                                   cudaStream_t s) {
  if (op->ept_ops.size() != static_cast<size_t>(dgw::ept_ops_floats(op->N)))
    return cudaErrorInvalidValue;
  const float* t = op->ept_ops.data();
  switch (op->N) {
    case 1: return dgw::launch_stage_ept_media<1>(a, t, mode, op->num_sms, s);
    case 2: return dgw::launch_stage_ept_media<2>(a, t, mode, op->num_sms, s);
    case 3: return dgw::launch_stage_ept_media<3>(a, t, mode, op->num_sms, s);
    case 4: return dgw::launch_stage_ept_media<4>(a, t, mode, op->num_sms, s);
    case 5: return dgw::launch_stage_ept_media<5>(a, t, mode, op->num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_order_media(const dg_op* op, const dgw::StageArgs<T>& a, int mode,
                               cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (op->use_ept) return launch_order_ept_media(op, a, mode, s);
    if (op->use_tc) return launch_order_tc_media(op, a, mode, s);
  }
  switch (op->N) {
    case 1: return dgw::launch_stage_media<T, 1>(a, mode, op->num_sms, s);
    case 2: return dgw::launch_stage_media<T, 2>(a, mode, op->num_sms, s);
    case 3: return dgw::launch_stage_media<T, 3>(a, mode, op->num_sms, s);
    case 4: return dgw::launch_stage_media<T, 4>(a, mode, op->num_sms, s);
    case 5: return dgw::launch_stage_media<T, 5>(a, mode, op->num_sms, s);
    case 6: return dgw::launch_stage_media<T, 6>(a, mode, op->num_sms, s);
    case 7: return dgw::launch_stage_media<T, 7>(a, mode, op->num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_order_ept(const dg_op* op, const dgw::StageArgs<float>& a, int mode,
                             cudaStream_t s) {
  if (op->ept_ops.size() != static_cast<size_t>(dgw::ept_ops_floats(op->N)))
    return cudaErrorInvalidValue;
  const float* t = op->ept_ops.data();
  switch (op->N) {
    case 1: return dgw::launch_stage_ept<1>(a, t, mode, op->num_sms, s);
    case 2: return dgw::launch_stage_ept<2>(a, t, mode, op->num_sms, s);
    case 3: return dgw::launch_stage_ept<3>(a, t, mode, op->num_sms, s);
    case 4: return dgw::launch_stage_ept<4>(a, t, mode, op->num_sms, s);
    case 5: return dgw::launch_stage_ept<5>(a, t, mode, op->num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_order(const dg_op* op, const dgw::StageArgs<T>& a, int mode, cudaStream_t s) {
  if (op->media()) return launch_order_media<T>(op, a, mode, s);
  if constexpr (sizeof(T) == 4) {
    if (op->use_ept) return launch_order_ept(op, a, mode, s);
    if (op->use_tc) return launch_order_tc(op, a, mode, s);
  }
  switch (op->N) {
    case 1: return dgw::launch_stage<T, 1>(a, mode, op->num_sms, s);
    case 2: return dgw::launch_stage<T, 2>(a, mode, op->num_sms, s);
    case 3: return dgw::launch_stage<T, 3>(a, mode, op->num_sms, s);
    case 4: return dgw::launch_stage<T, 4>(a, mode, op->num_sms, s);
    case 5: return dgw::launch_stage<T, 5>(a, mode, op->num_sms, s);
    case 6: return dgw::launch_stage<T, 6>(a, mode, op->num_sms, s);
    case 7: return dgw::launch_stage<T, 7>(a, mode, op->num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
dgw::StageArgs<T> base_args(const dg_op* op) {
  dgw::StageArgs<T> a;
  a.K = op->K;
  a.fstride = op->fstride;
  a.geo = static_cast<const T*>(op->d_geo);
  a.conn = static_cast<const int32_t*>(op->d_conn);
  a.Dr = static_cast<const T*>(op->d_Dr);
  a.Ds = static_cast<const T*>(op->d_Ds);
  a.LIFT = static_cast<const T*>(op->d_LIFT);
  a.lam = static_cast<const T*>(op->d_lam);
  a.status = op->d_status;
  a.tc_op = op->d_tcop;
  a.alpha = static_cast<T>(op->alpha);
  a.face_pairs = op->face_pairs;
  a.tc_alt = op->tc_alt;
  return a;
}

// The 3xTF32 tensor-core kernel of order N has an alternative element-block
// size (tc_tiles, launch.h).
bool tc_has_alt_n(int N) {
  switch (N) {
    case 1: return dgw::tc_has_alt(1, dgw::kTcTf32x3);
    case 2: return dgw::tc_has_alt(2, dgw::kTcTf32x3);
    case 3: return dgw::tc_has_alt(3, dgw::kTcTf32x3);
    case 4: return dgw::tc_has_alt(4, dgw::kTcTf32x3);
    case 5: return dgw::tc_has_alt(5, dgw::kTcTf32x3);
    case 6: return dgw::tc_has_alt(6, dgw::kTcTf32x3);
    case 7: return dgw::tc_has_alt(7, dgw::kTcTf32x3);
    default: return false;
  }
}

// Elements per block of the kernel the operator runs (alt: the alternative
// size of the tensor-core kernel).
int block_elems(const dg_op* op, int alt) {
  if (op->precision == DG_FP32 && op->use_ept) return 32;
  if (op->precision == DG_FP32 && op->use_tc)
    return 40 * dgw::tc_tiles(op->N, op->tc_prec, alt != 0 && op->tc_prec == dgw::kTcTf32x3);
  return dgw::simt_block_elems(op->N, op->precision == DG_FP64);
}

dg_status check_device_op(const dg_op* op, const char* where) {
  if (!op) return fail(DG_ERR_ARG, "%s: NULL operator", where);
  if (!op->has_device)
    return fail(DG_ERR_NO_DEVICE, "%s: operator was set up host-only", where);
  cudaError_t err = cudaSetDevice(op->device);
  if (err != cudaSuccess) return cuda_fail(err, where);
  return DG_OK;
}

bool overlaps(const void* a, const void* b, size_t bytes) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + bytes && pb < pa + bytes;
}

dg_status check_field(const dg_op* op, const void* p, const char* name, const char* where) {
  if (!p) return fail(DG_ERR_ARG, "%s: %s is NULL", where, name);
  if (reinterpret_cast<uintptr_t>(p) % 16 != 0)
    return fail(DG_ERR_ARG, "%s: %s is not 16-byte aligned", where, name);
  return DG_OK;
}

// Ricker point source of an operator (dg_operator_set_source), applied after
// a stage launch: the source element's Ez residual gains dt s(t) w and its
// Ez values b times that.  This is the LSRK stage update with s(t) w added
// to the right-hand side of Eq. dg-strong-explicit (w = M^-1 l(x_s) / J_k,
// the projected point load).  rhs_only: q is a right-hand side, which gains
// s(t) w.  s(t) = A (1 - 2 a^2) exp(-a^2), a = pi f (t - t0).
template <typename T>
__global__ void point_source_kernel(T* q, T* res, const T* w, int Np, double t, double pif,
                                    double t0, double amp, double dt, double b, int rhs_only) {
  const int n = threadIdx.x;
  if (n >= Np) return;
  const double a = (t - t0) * pif;
  const double s = amp * (1.0 - 2.0 * a * a) * exp(-a * a);
  if (rhs_only) {
    q[n] += static_cast<T>(s) * w[n];
    return;
  }
  const T v = static_cast<T>(dt * s) * w[n];
  res[n] += v;
  q[n] += static_cast<T>(b) * v;
}

// The point source after stage i of a step that starts at t (stage time
// t + c_i dt), on the stage's output fields q and residual res; nothing
// without a source.
template <typename T>
cudaError_t stage_source(const dg_op* op, T* q, T* res, double t, double dt, int i,
                         cudaStream_t s) {
  if (!op->has_src) return cudaSuccess;
  const int64_t off = 2 * op->fstride + op->src_k * op->Np;
  point_source_kernel<T><<<1, 64, 0, s>>>(q + off, res + off, static_cast<const T*>(op->d_src_w),
                                          op->Np, t + op->lsrk_c[i] * dt, M_PI * op->src.f,
                                          op->src.t0, op->src.amplitude, dt, op->lsrk_b[i], 0);
  op->launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

template <typename T>
dg_status run_steps(const dg_op* op, T* q, T* res, double t0, double dt, int32_t nsteps,
                    cudaStream_t s) {
  dgw::StageArgs<T> a = base_args<T>(op);
  a.res = res;
  a.dt = static_cast<T>(dt);
  T* cur = q;
  T* other = static_cast<T*>(op->d_qtmp);
  for (int32_t n = 0; n < nsteps; ++n) {
    for (int i = 0; i < 5; ++i) {
      a.qin = cur;
      a.qout = other;
      a.a = static_cast<T>(op->lsrk_a[i]);
      a.b = static_cast<T>(op->lsrk_b[i]);
      const int mode = (i == 0) ? dgw::kModeFirstStage : dgw::kModeStage;
      cudaError_t err = launch_order<T>(op, a, mode, s);
      if (err != cudaSuccess) return cuda_fail(err, "dg_step: kernel launch");
      op->launches.fetch_add(1, std::memory_order_relaxed);
      err = stage_source<T>(op, other, res, t0 + n * dt, dt, i, s);
      if (err != cudaSuccess) return cuda_fail(err, "dg_step: point-source launch");
      std::swap(cur, other);
    }
  }
  if (cur != q) {
    cudaError_t err = cudaMemcpyAsync(q, cur, 3 * op->fstride * sizeof(T),
                                      cudaMemcpyDeviceToDevice, s);
    if (err != cudaSuccess) return cuda_fail(err, "dg_step: copy-back");
  }
  return DG_OK;
}

__global__ void finite_scan_kernel(const float* q32, const double* q64, int64_t fstride,
                                   int64_t n, int* flag) {
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < 3 * n;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t f = idx / n;
    const int64_t o = f * fstride + (idx - f * n);
    const double v = q32 ? static_cast<double>(q32[o]) : q64[o];
    if (!isfinite(v)) {
      atomicExch(flag, 1);
      return;
    }
  }
}

}  // namespace

// ============================================================ C ABI
namespace {

// dg_operator_setup and dg_operator_setup_media; eps NULL: eps = 1.
dg_status operator_setup(const dg_mesh* mesh, int32_t N, const double* eps, int32_t precision,
                         int32_t flags, dg_op** out) {
  if (!mesh || !out) return fail(DG_ERR_ARG, "dg_operator_setup: NULL argument");
  if (N < 1 || N > DG_N_MAX)
    return fail(DG_ERR_ORDER, "dg_operator_setup: N = %d outside 1..%d", N, DG_N_MAX);
  if (precision != DG_FP32 && precision != DG_FP64)
    return fail(DG_ERR_ARG, "dg_operator_setup: unknown precision %d", precision);
  const int32_t known = DG_SETUP_HOST_ONLY | DG_SETUP_SIMT | DG_SETUP_TC_TF32 | DG_SETUP_TC_BF16 |
                        DG_SETUP_TC_BF16X3 | DG_SETUP_TC | DG_SETUP_ELEMENT_THREADS;
  const int32_t variants = flags & (DG_SETUP_TC_TF32 | DG_SETUP_TC_BF16 | DG_SETUP_TC_BF16X3);
  if (flags & ~known) return fail(DG_ERR_ARG, "dg_operator_setup: unknown flags 0x%x", flags);
  if ((flags & DG_SETUP_TC) && ((flags & DG_SETUP_SIMT) || precision != DG_FP32))
    return fail(DG_ERR_ARG, "dg_operator_setup: DG_SETUP_TC is for FP32 without DG_SETUP_SIMT");
  if (variants && ((variants & (variants - 1)) || precision != DG_FP32 || (flags & DG_SETUP_SIMT)))
    return fail(DG_ERR_ARG,
                "dg_operator_setup: at most one tensor-core product variant, FP32 only, not with "
                "DG_SETUP_SIMT");
  if ((flags & DG_SETUP_ELEMENT_THREADS) &&
      (precision != DG_FP32 || N > dgw::kEptMaxN ||
       (flags & (DG_SETUP_SIMT | DG_SETUP_TC | DG_SETUP_TC_TF32 | DG_SETUP_TC_BF16 |
                 DG_SETUP_TC_BF16X3))))
    return fail(DG_ERR_ARG,
                "dg_operator_setup: DG_SETUP_ELEMENT_THREADS is for FP32 at N <= %d, without "
                "another kernel or product flag",
                dgw::kEptMaxN);
  dg_op* op = nullptr;
  try {
    op = new dg_op;
    op->N = N;
    op->ref = dgw::build_reference(N);
    op->Np = op->ref.Np;
    op->Nfp = op->ref.Nfp;
    op->Nafp = op->ref.Nafp;
    op->precision = precision;
    op->flags = flags;
    // FP32 default: the element-thread kernel at N <= 2, the tensor cores
    // above (order sweep at ~1e7 nodal values per field, ms/step, element
    // threads / node threads / tensor cores: N = 1 0.68, 0.87, 1.39; N = 2
    // 0.50, 0.98, 0.83; N = 3 0.62, 0.90, 0.60; with a permittivity: N = 1
    // 0.70, 0.86, 1.37; N = 2 0.64, 0.95, 0.82; N = 3 0.64, 0.89, 0.61)
    op->use_tc = (precision == DG_FP32) && !(flags & DG_SETUP_SIMT) &&
                 (N >= 2 || variants != 0 || (flags & DG_SETUP_TC));
    const int32_t chosen = DG_SETUP_SIMT | DG_SETUP_TC | DG_SETUP_TC_TF32 | DG_SETUP_TC_BF16 |
                           DG_SETUP_TC_BF16X3;
    op->use_ept = (flags & DG_SETUP_ELEMENT_THREADS) ||
                  (precision == DG_FP32 && !(flags & chosen) && N <= 2);
    op->tc_prec = (flags & DG_SETUP_TC_TF32)    ? dgw::kTcTf32
                  : (flags & DG_SETUP_TC_BF16)  ? dgw::kTcBf16
                  : (flags & DG_SETUP_TC_BF16X3) ? dgw::kTcBf16x3
                                                 : dgw::kTcTf32x3;
    op->elem_size = (precision == DG_FP32) ? 4 : 8;
    op->K = mesh->K;
    op->Kpad = (mesh->K + 1 + kBlockPad - 1) / kBlockPad * kBlockPad;
    // whole blocks, and every field 256-byte aligned (64 values)
    op->fstride = (op->Kpad * op->Np + 63) / 64 * 64;
    if (op->fstride >= (int64_t(1) << 31)) {
      const long long fsz = static_cast<long long>(op->fstride);
      delete op;
      return fail(DG_ERR_ARG,
                  "dg_operator_setup: K * Np = %lld nodes per field exceeds 2^31 - 1", fsz);
    }
    op->geo = dgw::build_geometry(*mesh, op->ref);
    op->min_inradius_over_c = op->geo.min_inradius;
    if (eps) {
      op->eps.assign(eps, eps + mesh->K);
      // CFL length scale of a medium: min over elements of inradius * sqrt(eps_k)
      double m = 1e300;
      for (int64_t k = 0; k < mesh->K; ++k) {
        const int32_t* v = &mesh->EToV[3 * k];
        double per = 0.0;
        for (int f = 0; f < 3; ++f) {
          const int32_t a = v[f], b = v[(f + 1) % 3];
          per += std::hypot(mesh->vx[b] - mesh->vx[a], mesh->vy[b] - mesh->vy[a]);
        }
        m = std::min(m, 2.0 * op->geo.J[k] / (0.5 * per) * std::sqrt(op->eps[k]));
      }
      op->min_inradius_over_c = m;
    }
    dgw::lsrk_coefficients(op->lsrk_a, op->lsrk_b, op->lsrk_c);
  } catch (const std::bad_alloc&) {
    delete op;
    return fail(DG_ERR_OOM, "dg_operator_setup: out of host memory");
  } catch (const std::exception& ex) {
    delete op;
    return fail(DG_ERR_ARG, "dg_operator_setup: %s", ex.what());
  }
  if (!(flags & DG_SETUP_HOST_ONLY)) {
    cudaError_t err = cudaGetDevice(&op->device);
    if (err != cudaSuccess) {
      delete op;
      return cuda_fail(err, "dg_operator_setup: cudaGetDevice");
    }
    err = cudaDeviceGetAttribute(&op->num_sms, cudaDevAttrMultiProcessorCount, op->device);
    if (err != cudaSuccess) {
      delete op;
      return cuda_fail(err, "dg_operator_setup: device attribute");
    }
    dg_status st = DG_OK;
    try {
      std::vector<double> rec;
      std::vector<int32_t> conn;
      dgw::operator_records(*op, rec, conn);
      st = (precision == DG_FP32) ? upload<float>(op, rec, conn) : upload<double>(op, rec, conn);
    } catch (const std::bad_alloc&) {
      st = fail(DG_ERR_OOM, "dg_operator_setup: out of host memory");
    }
    if (st != DG_OK) {
      free_device(op);
      delete op;
      return st;
    }
    op->has_device = true;
  }
  *out = op;
  return DG_OK;
}

}  // namespace

extern "C" dg_status dg_operator_setup(const dg_mesh* mesh, int32_t N, int32_t precision,
                                       int32_t flags, dg_op** out) {
  dgw::clear_error();
  return operator_setup(mesh, N, nullptr, precision, flags, out);
}

extern "C" dg_status dg_operator_setup_media(const dg_mesh* mesh, int32_t N, const double* eps,
                                             int32_t precision, int32_t flags, dg_op** out) {
  dgw::clear_error();
  if (!mesh || !eps || !out) return fail(DG_ERR_ARG, "dg_operator_setup_media: NULL argument");
  for (int64_t k = 0; k < mesh->K; ++k)
    if (!(eps[k] > 0.0) || !std::isfinite(eps[k]))
      return fail(DG_ERR_ARG, "dg_operator_setup_media: eps[%lld] = %g is not a positive number",
                  static_cast<long long>(k), eps[k]);
  if (flags & (DG_SETUP_TC_TF32 | DG_SETUP_TC_BF16 | DG_SETUP_TC_BF16X3))
    return fail(DG_ERR_ARG,
                "dg_operator_setup_media: the lower-precision product variants are not "
                "available with a per-element permittivity");
  return operator_setup(mesh, N, eps, precision, flags, out);
}

extern "C" dg_status dg_operator_set_alpha(dg_op* op, double alpha) {
  dgw::clear_error();
  if (!op) return fail(DG_ERR_ARG, "dg_operator_set_alpha: NULL operator");
  if (!(alpha >= 0.0 && alpha <= 1.0))
    return fail(DG_ERR_ARG, "dg_operator_set_alpha: alpha = %g outside [0, 1]", alpha);
  if (op->media())
    return fail(DG_ERR_ARG,
                "dg_operator_set_alpha: operators with a per-element permittivity use the upwind "
                "flux of the interface Riemann solution only");
  op->alpha = alpha;
  return DG_OK;
}

extern "C" dg_status dg_operator_set_face_pairs(dg_op* op, int32_t enable) {
  dgw::clear_error();
  if (!op) return fail(DG_ERR_ARG, "dg_operator_set_face_pairs: NULL operator");
  if (enable != 0 && enable != 1)
    return fail(DG_ERR_ARG, "dg_operator_set_face_pairs: enable = %d is not 0 or 1", enable);
  op->face_pairs = enable;
  return DG_OK;
}

extern "C" dg_status dg_operator_set_source(dg_op* op, const dg_point_source* src) {
  dgw::clear_error();
  const char* where = "dg_operator_set_source";
  if (!op) return fail(DG_ERR_ARG, "%s: NULL operator", where);
  if (!src) {
    op->has_src = false;
    op->src_k = -1;
    return DG_OK;
  }
  if (!std::isfinite(src->x) || !std::isfinite(src->y) || !(src->f > 0.0) ||
      !std::isfinite(src->f) || !std::isfinite(src->t0) || !std::isfinite(src->amplitude))
    return fail(DG_ERR_ARG, "%s: bad point source parameters", where);
  std::vector<double> w;
  const int64_t k = dgw::point_source(op->ref, op->geo, op->K, src->x, src->y, w);
  if (k < 0)
    return fail(DG_ERR_ARG, "%s: source point (%g, %g) is outside the mesh", where, src->x, src->y);
  if (op->has_device) {
    dg_status st = check_device_op(op, where);
    if (st) return st;
    cudaError_t err = cudaSuccess;
    if (!op->d_src_w) err = dgw::dev_malloc(&op->d_src_w, static_cast<size_t>(op->Np) * 8);
    if (err == cudaSuccess) {
      if (op->precision == DG_FP32) {
        std::vector<float> wf(w.begin(), w.end());
        err = cudaMemcpy(op->d_src_w, wf.data(), wf.size() * 4, cudaMemcpyHostToDevice);
      } else {
        err = cudaMemcpy(op->d_src_w, w.data(), w.size() * 8, cudaMemcpyHostToDevice);
      }
    }
    if (err != cudaSuccess) return cuda_fail(err, where);
  }
  op->src = *src;
  op->src_k = k;
  op->has_src = true;
  return DG_OK;
}

extern "C" dg_status dg_get_info(const dg_op* op, int32_t* Np, int32_t* Nfp, int64_t* K,
                                 int64_t* field_stride) {
  dgw::clear_error();
  if (!op) return fail(DG_ERR_ARG, "dg_get_info: NULL operator");
  if (Np) *Np = op->Np;
  if (Nfp) *Nfp = op->Nfp;
  if (K) *K = op->K;
  if (field_stride) *field_stride = op->fstride;
  return DG_OK;
}

extern "C" dg_status dg_get_nodes(const dg_op* op, double* x, double* y) {
  dgw::clear_error();
  if (!op || !x || !y) return fail(DG_ERR_ARG, "dg_get_nodes: NULL argument");
  std::memcpy(x, op->geo.x.data(), op->geo.x.size() * sizeof(double));
  std::memcpy(y, op->geo.y.data(), op->geo.y.size() * sizeof(double));
  return DG_OK;
}

extern "C" dg_status dg_get_reference(const dg_op* op, double* r, double* s, double* Dr,
                                      double* Ds, double* LIFT, int32_t* Fmask) {
  dgw::clear_error();
  if (!op) return fail(DG_ERR_ARG, "dg_get_reference: NULL operator");
  const dgw::RefElement& R = op->ref;
  if (r) std::copy(R.r.begin(), R.r.end(), r);
  if (s) std::copy(R.s.begin(), R.s.end(), s);
  if (Dr) std::copy(R.Dr.begin(), R.Dr.end(), Dr);
  if (Ds) std::copy(R.Ds.begin(), R.Ds.end(), Ds);
  if (LIFT) std::copy(R.LIFT.begin(), R.LIFT.end(), LIFT);
  if (Fmask) std::copy(R.Fmask.begin(), R.Fmask.end(), Fmask);
  return DG_OK;
}

extern "C" dg_status dg_get_geometry(const dg_op* op, double* rx, double* ry, double* sx,
                                     double* sy, double* J, double* nx, double* ny,
                                     double* Fscale) {
  dgw::clear_error();
  if (!op) return fail(DG_ERR_ARG, "dg_get_geometry: NULL operator");
  const dgw::Geometry& G = op->geo;
  if (rx) std::copy(G.rx.begin(), G.rx.end(), rx);
  if (ry) std::copy(G.ry.begin(), G.ry.end(), ry);
  if (sx) std::copy(G.sx.begin(), G.sx.end(), sx);
  if (sy) std::copy(G.sy.begin(), G.sy.end(), sy);
  if (J) std::copy(G.J.begin(), G.J.end(), J);
  if (nx) std::copy(G.nx.begin(), G.nx.end(), nx);
  if (ny) std::copy(G.ny.begin(), G.ny.end(), ny);
  if (Fscale) std::copy(G.Fscale.begin(), G.Fscale.end(), Fscale);
  return DG_OK;
}

extern "C" dg_status dg_get_maps(const dg_op* op, int64_t* vmapM, int64_t* vmapP) {
  dgw::clear_error();
  if (!op || !vmapM || !vmapP) return fail(DG_ERR_ARG, "dg_get_maps: NULL argument");
  const int N = op->N, Np = op->Np, Nfp = op->Nfp, Nafp = op->Nafp;
  for (int64_t k = 0; k < op->K; ++k)
    for (int f = 0; f < 3; ++f) {
      const int32_t code = op->geo.conn[3 * k + f];
      for (int j = 0; j < Nfp; ++j) {
        const int64_t pos = k * Nafp + f * Nfp + j;
        vmapM[pos] = k * Np + dgw::face_node(N, f, j);
        if (code < 0) {
          vmapP[pos] = vmapM[pos];
        } else {
          const int64_t kP = code >> 3;
          const int fP = (code >> 1) & 3;
          const int jP = (code & 1) ? (N - j) : j;
          vmapP[pos] = kP * Np + dgw::face_node(N, fP, jP);
        }
      }
    }
  return DG_OK;
}

extern "C" dg_status dg_operator_tune(dg_op* op, int32_t reps, void* stream, double* ms_tc,
                                      double* ms_cuda_cores) {
  dgw::clear_error();
  dg_status st = check_device_op(op, "dg_operator_tune");
  if (st) return st;
  if (reps < 1) return fail(DG_ERR_ARG, "dg_operator_tune: reps = %d < 1", reps);
  if (ms_tc) *ms_tc = -1.0;
  if (ms_cuda_cores) *ms_cuda_cores = -1.0;
  const int32_t fixed = DG_SETUP_SIMT | DG_SETUP_TC_TF32 | DG_SETUP_TC_BF16 | DG_SETUP_TC_BF16X3 |
                        DG_SETUP_ELEMENT_THREADS;
  if (op->precision != DG_FP32 || (op->flags & fixed)) return DG_OK;  // nothing to choose
  // candidates: tensor cores (3xTF32) in the default and, where there is one,
  // the alternative element-block size; unless DG_SETUP_TC, the CUDA cores:
  // the node-per-thread kernel, and the element-thread kernel where the
  // operator has its tables (N <= kEptMaxN)
  struct Cand {
    bool tc;
    int alt;
    bool ept;
  } cand[4];
  int nc = 0;
  cand[nc++] = {true, 0, false};
  if (tc_has_alt_n(op->N)) cand[nc++] = {true, 1, false};
  if (!(op->flags & DG_SETUP_TC)) {
    cand[nc++] = {false, 0, false};
    if (op->ept_ops.size() == static_cast<size_t>(dgw::ept_ops_floats(op->N)))
      cand[nc++] = {false, 0, true};
  }
  if (nc < 2) return DG_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t err = cudaSuccess;
  if (!op->d_tcop) {  // the tensor-core kernel's operator tiles
    const std::vector<unsigned char> tiles = tc_operator_tiles(op->ref, dgw::kTcTf32x3);
    err = dgw::dev_malloc(&op->d_tcop, tiles.size());
    if (err == cudaSuccess)
      err = cudaMemcpy(op->d_tcop, tiles.data(), tiles.size(), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) return cuda_fail(err, "dg_operator_tune: operator tiles");
  }
  // scratch fields q, q_out and res (zero), stage-2 launches of each candidate
  const size_t fb = 3 * static_cast<size_t>(op->fstride) * sizeof(float);
  float* buf = nullptr;
  err = dgw::dev_malloc(reinterpret_cast<void**>(&buf), 3 * fb);
  if (err == cudaSuccess) err = cudaMemsetAsync(buf, 0, 3 * fb, s);
  if (err != cudaSuccess) {
    if (buf) cudaFree(buf);
    return cuda_fail(err, "dg_operator_tune: scratch fields");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const bool was_tc = op->use_tc, was_ept = op->use_ept;
  const int was_alt = op->tc_alt;
  float ms[4] = {0.f, 0.f, 0.f, 0.f};
  for (int v = 0; v < nc && err == cudaSuccess; ++v) {
    op->use_tc = cand[v].tc;
    op->tc_alt = cand[v].alt;
    op->use_ept = cand[v].ept;
    dgw::StageArgs<float> a = base_args<float>(op);
    a.qin = buf;
    a.qout = buf + 3 * op->fstride;
    a.res = buf + 6 * op->fstride;
    a.a = static_cast<float>(op->lsrk_a[1]);
    a.b = static_cast<float>(op->lsrk_b[1]);
    a.dt = 1e-6f;
    err = launch_order<float>(op, a, dgw::kModeStage, s);  // warm
    if (err == cudaSuccess) err = cudaEventRecord(e0, s);
    for (int r = 0; r < reps && err == cudaSuccess; ++r)
      err = launch_order<float>(op, a, dgw::kModeStage, s);
    if (err == cudaSuccess) err = cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms[v], e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  op->launches.fetch_add(nc * (reps + 1), std::memory_order_relaxed);
  if (err != cudaSuccess) {
    op->use_tc = was_tc;
    op->tc_alt = was_alt;
    op->use_ept = was_ept;
    return cuda_fail(err, "dg_operator_tune");
  }
  int best = 0;
  for (int v = 1; v < nc; ++v)
    if (ms[v] < ms[best]) best = v;
  op->use_tc = cand[best].tc;
  op->tc_alt = cand[best].alt;
  op->use_ept = cand[best].ept;
  double best_tc = -1.0, best_cc = -1.0;
  for (int v = 0; v < nc; ++v) {
    double& b = cand[v].tc ? best_tc : best_cc;
    if (b < 0 || ms[v] < b) b = ms[v];
  }
  if (ms_tc) *ms_tc = best_tc / reps;
  if (ms_cuda_cores && best_cc >= 0) *ms_cuda_cores = best_cc / reps;
  return DG_OK;
}

extern "C" dg_status dg_operator_set_block_elems(dg_op* op, int32_t elems) {
  dgw::clear_error();
  const char* where = "dg_operator_set_block_elems";
  if (!op) return fail(DG_ERR_ARG, "%s: NULL operator", where);
  const bool alt_ok = op->precision == DG_FP32 && op->use_tc && !op->use_ept &&
                      op->tc_prec == dgw::kTcTf32x3 && tc_has_alt_n(op->N);
  const int def = block_elems(op, 0), alt = alt_ok ? block_elems(op, 1) : def;
  if (elems == 0 || elems == def) {
    op->tc_alt = 0;
  } else if (alt_ok && elems == alt) {
    op->tc_alt = 1;
  } else {
    return fail(DG_ERR_ARG, "%s: %d elements per block is not a size of this operator's kernel "
                "(%d%s%s)", where, elems, def, alt_ok ? " or " : "",
                alt_ok ? std::to_string(alt).c_str() : "");
  }
  return DG_OK;
}

extern "C" dg_status dg_operator_kernel(const dg_op* op, int32_t* kernel, int32_t* elems) {
  dgw::clear_error();
  if (!op) return fail(DG_ERR_ARG, "dg_operator_kernel: NULL operator");
  const bool ept = op->precision == DG_FP32 && op->use_ept;
  const bool tc = op->precision == DG_FP32 && op->use_tc && !ept;
  if (kernel)
    *kernel = ept ? DG_KERNEL_ELEMENT_THREADS : tc ? DG_KERNEL_TENSOR_CORES : DG_KERNEL_CUDA_CORES;
  if (elems) *elems = block_elems(op, op->tc_alt && !op->face_pairs);
  return DG_OK;
}

extern "C" dg_status dg_cfl_dt(const dg_op* op, double cfl, double* dt) {
  dgw::clear_error();
  if (!op || !dt) return fail(DG_ERR_ARG, "dg_cfl_dt: NULL argument");
  if (!(cfl > 0) || !std::isfinite(cfl)) return fail(DG_ERR_ARG, "dg_cfl_dt: cfl must be > 0");
  *dt = cfl * (2.0 / 3.0) * op->min_inradius_over_c * op->ref.lgl_gap;
  return DG_OK;
}

extern "C" void dg_op_destroy(dg_op* op) {
  if (!op) return;
  if (op->has_device) {
    cudaSetDevice(op->device);
    free_device(op);
  }
  delete op;
}

extern "C" dg_status dg_rhs(const dg_op* op, const void* d_q, void* d_rhs, double t,
                            void* stream) {
  dgw::clear_error();
  if (!std::isfinite(t)) return fail(DG_ERR_ARG, "dg_rhs: t is not finite");
  dg_status st = check_device_op(op, "dg_rhs");
  if (st) return st;
  if ((st = check_field(op, d_q, "d_q", "dg_rhs"))) return st;
  if ((st = check_field(op, d_rhs, "d_rhs", "dg_rhs"))) return st;
  const size_t bytes = 3 * op->fstride * op->elem_size;
  if (overlaps(d_q, d_rhs, bytes)) return fail(DG_ERR_ARG, "dg_rhs: d_q and d_rhs overlap");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t err;
  if (op->precision == DG_FP32) {
    dgw::StageArgs<float> a = base_args<float>(op);
    a.qin = static_cast<const float*>(d_q);
    a.rhs = static_cast<float*>(d_rhs);
    err = launch_order<float>(op, a, dgw::kModeRhs, s);
  } else {
    dgw::StageArgs<double> a = base_args<double>(op);
    a.qin = static_cast<const double*>(d_q);
    a.rhs = static_cast<double*>(d_rhs);
    err = launch_order<double>(op, a, dgw::kModeRhs, s);
  }
  if (err != cudaSuccess) return cuda_fail(err, "dg_rhs: kernel launch");
  op->launches.fetch_add(1, std::memory_order_relaxed);
  if (op->has_src) {
    const int64_t off = 2 * op->fstride + op->src_k * op->Np;
    const double pif = M_PI * op->src.f;
    if (op->precision == DG_FP32)
      point_source_kernel<float><<<1, 64, 0, s>>>(
          static_cast<float*>(d_rhs) + off, nullptr, static_cast<const float*>(op->d_src_w),
          op->Np, t, pif, op->src.t0, op->src.amplitude, 0.0, 0.0, 1);
    else
      point_source_kernel<double><<<1, 64, 0, s>>>(
          static_cast<double*>(d_rhs) + off, nullptr, static_cast<const double*>(op->d_src_w),
          op->Np, t, pif, op->src.t0, op->src.amplitude, 0.0, 0.0, 1);
    err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "dg_rhs: point-source launch");
    op->launches.fetch_add(1, std::memory_order_relaxed);
  }
  return DG_OK;
}

extern "C" dg_status dg_step(const dg_op* op, void* d_q, void* d_res, double t0, double dt,
                             int32_t nsteps, void* stream) {
  dgw::clear_error();
  dg_status st = check_device_op(op, "dg_step");
  if (st) return st;
  if ((st = check_field(op, d_q, "d_q", "dg_step"))) return st;
  if ((st = check_field(op, d_res, "d_res", "dg_step"))) return st;
  if (nsteps < 0) return fail(DG_ERR_ARG, "dg_step: nsteps = %d < 0", nsteps);
  if (!std::isfinite(dt) || !std::isfinite(t0))
    return fail(DG_ERR_ARG, "dg_step: dt or t0 is not finite");
  const size_t bytes = 3 * op->fstride * op->elem_size;
  if (overlaps(d_q, d_res, bytes)) return fail(DG_ERR_ARG, "dg_step: d_q and d_res overlap");
  if (overlaps(d_q, op->d_qtmp, bytes) || overlaps(d_res, op->d_qtmp, bytes))
    return fail(DG_ERR_ARG, "dg_step: buffer overlaps the operator's internal buffer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (op->precision == DG_FP32)
    return run_steps<float>(op, static_cast<float*>(d_q), static_cast<float*>(d_res), t0, dt,
                            nsteps, s);
  return run_steps<double>(op, static_cast<double*>(d_q), static_cast<double*>(d_res), t0, dt,
                           nsteps, s);
}

extern "C" dg_status dg_solve(const dg_op* op, void* d_q, void* d_res, double T, double dt,
                              int32_t* nsteps_out, double* t_reached, void* stream) {
  dgw::clear_error();
  if (!op) return fail(DG_ERR_ARG, "dg_solve: NULL operator");
  if (!(T >= 0) || !std::isfinite(T)) return fail(DG_ERR_ARG, "dg_solve: bad final time");
  if (!(dt > 0)) {
    dg_status st = dg_cfl_dt(op, 1.0, &dt);
    if (st) return st;
  }
  const double ns = std::ceil(T / dt - 1e-12);
  if (ns > 2147483647.0) return fail(DG_ERR_ARG, "dg_solve: too many steps");
  const int32_t nsteps = static_cast<int32_t>(std::max(0.0, ns));
  const double dts = nsteps > 0 ? T / nsteps : 0.0;
  dg_status st = dg_step(op, d_q, d_res, 0.0, dts, nsteps, stream);
  if (st) return st;
  if (nsteps_out) *nsteps_out = nsteps;
  if (t_reached) *t_reached = nsteps * dts;
  return DG_OK;
}

extern "C" dg_status dg_step_host(const dg_op* op, void* h_q, void* d_q, void* d_res, double t0,
                                  double dt, int32_t nsteps, void* stream) {
  dgw::clear_error();
  dg_status st = check_device_op(op, "dg_step_host");
  if (st) return st;
  if (!h_q) return fail(DG_ERR_ARG, "dg_step_host: h_q is NULL");
  if ((st = check_field(op, d_q, "d_q", "dg_step_host"))) return st;
  if ((st = check_field(op, d_res, "d_res", "dg_step_host"))) return st;
  if (nsteps < 0 || !std::isfinite(dt)) return fail(DG_ERR_ARG, "dg_step_host: bad nsteps/dt");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = 3 * op->fstride * op->elem_size;
  cudaError_t err = cudaMemcpyAsync(d_q, h_q, bytes, cudaMemcpyHostToDevice, s);
  if (err != cudaSuccess) return cuda_fail(err, "dg_step_host: host-to-device copy");
  st = dg_step(op, d_q, d_res, t0, dt, nsteps, stream);
  if (st) return st;
  err = cudaMemcpyAsync(h_q, d_q, bytes, cudaMemcpyDeviceToHost, s);
  if (err != cudaSuccess) return cuda_fail(err, "dg_step_host: device-to-host copy");
  err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return cuda_fail(err, "dg_step_host: synchronize");
  return DG_OK;
}

namespace {

// nsteps LSRK steps ping-ponging between q and tmp (no copy back); returns
// the buffer that holds the result
template <typename T>
dg_status run_stages(const dg_op* op, T* q, T* tmp, T* res, double t0, double dt,
                     int32_t nsteps, cudaStream_t s, T** result) {
  dgw::StageArgs<T> a = base_args<T>(op);
  a.res = res;
  a.dt = static_cast<T>(dt);
  T* cur = q;
  T* other = tmp;
  for (int32_t n = 0; n < nsteps; ++n) {
    for (int i = 0; i < 5; ++i) {
      a.qin = cur;
      a.qout = other;
      a.a = static_cast<T>(op->lsrk_a[i]);
      a.b = static_cast<T>(op->lsrk_b[i]);
      const int mode = (i == 0) ? dgw::kModeFirstStage : dgw::kModeStage;
      cudaError_t err = launch_order<T>(op, a, mode, s);
      if (err != cudaSuccess) return cuda_fail(err, "dg_step_host_jobs: kernel launch");
      op->launches.fetch_add(1, std::memory_order_relaxed);
      err = stage_source<T>(op, other, res, t0 + n * dt, dt, i, s);
      if (err != cudaSuccess) return cuda_fail(err, "dg_step_host_jobs: point-source launch");
      std::swap(cur, other);
    }
  }
  *result = cur;
  return DG_OK;
}

// Pipeline of dg_step_host_jobs: slot j % kJobSlots of the work buffer holds
// job j's fields (q, tmp); the residual is shared (the first stage of a step
// overwrites it, and the stage launches of all jobs run in order on one
// stream).
constexpr int kJobSlots = 3;

struct JobPipe {
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t start = nullptr;
  cudaEvent_t in_done[kJobSlots] = {}, comp_done[kJobSlots] = {}, free_slot[kJobSlots] = {};
  bool used[kJobSlots] = {};

  cudaError_t create() {
    cudaError_t err = cudaStreamCreateWithFlags(&h2d, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&d2h, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
    for (int i = 0; i < kJobSlots && err == cudaSuccess; ++i) {
      err = cudaEventCreateWithFlags(&in_done[i], cudaEventDisableTiming);
      if (err == cudaSuccess) err = cudaEventCreateWithFlags(&comp_done[i], cudaEventDisableTiming);
      if (err == cudaSuccess) err = cudaEventCreateWithFlags(&free_slot[i], cudaEventDisableTiming);
    }
    return err;
  }
  ~JobPipe() {
    if (h2d) cudaStreamSynchronize(h2d);
    if (d2h) cudaStreamSynchronize(d2h);
    for (int i = 0; i < kJobSlots; ++i) {
      if (in_done[i]) cudaEventDestroy(in_done[i]);
      if (comp_done[i]) cudaEventDestroy(comp_done[i]);
      if (free_slot[i]) cudaEventDestroy(free_slot[i]);
    }
    if (start) cudaEventDestroy(start);
    if (h2d) cudaStreamDestroy(h2d);
    if (d2h) cudaStreamDestroy(d2h);
  }
};

template <typename T>
dg_status run_jobs(const dg_op* op, int32_t njobs, void* const* h_q, T* work, double t0,
                   double dt, int32_t nsteps, cudaStream_t s) {
  const char* where = "dg_step_host_jobs";
  const size_t fvals = 3 * static_cast<size_t>(op->fstride);
  const size_t bytes = fvals * sizeof(T);
  T* res = work + 2 * kJobSlots * fvals;
  JobPipe pipe;
  cudaError_t err = pipe.create();
  if (err != cudaSuccess) return cuda_fail(err, where);
  // the entries of each field beyond K * Np never reach a result, but the
  // per-block bulk copies read them; zero them in the buffers the host does
  // not fill, so that no value left in the work memory is ever read
  const size_t used = static_cast<size_t>(op->K) * op->Np;
  const size_t tail = (static_cast<size_t>(op->fstride) - used) * sizeof(T);
  for (int b = 0; b <= 2 * kJobSlots && tail > 0 && err == cudaSuccess; ++b) {
    if (b < 2 * kJobSlots && b % 2 == 0) continue;  // a slot's q comes from the host
    for (int f = 0; f < 3 && err == cudaSuccess; ++f)
      err = cudaMemsetAsync(work + b * fvals + f * static_cast<size_t>(op->fstride) + used, 0,
                            tail, s);
  }
  if (err != cudaSuccess) return cuda_fail(err, where);
  // the copies start after whatever the caller queued on `stream` before
  err = cudaEventRecord(pipe.start, s);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(pipe.h2d, pipe.start, 0);
  if (err != cudaSuccess) return cuda_fail(err, where);
  for (int32_t j = 0; j < njobs; ++j) {
    const int slot = j % kJobSlots;
    T* q = work + 2 * slot * fvals;
    T* tmp = q + fvals;
    // copy in once the slot's previous job has been copied out, and once any
    // earlier job still in flight that shares this host buffer has written
    // its result there (jobs j - 1 and j - 2; job j - 3 is the slot's own)
    if (pipe.used[slot]) err = cudaStreamWaitEvent(pipe.h2d, pipe.free_slot[slot], 0);
    for (int back = 1; back < kJobSlots && back <= j && err == cudaSuccess; ++back)
      if (h_q[j - back] == h_q[j])
        err = cudaStreamWaitEvent(pipe.h2d, pipe.free_slot[(j - back) % kJobSlots], 0);
    if (err == cudaSuccess) err = cudaMemcpyAsync(q, h_q[j], bytes, cudaMemcpyHostToDevice, pipe.h2d);
    if (err == cudaSuccess) err = cudaEventRecord(pipe.in_done[slot], pipe.h2d);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(s, pipe.in_done[slot], 0);
    if (err != cudaSuccess) return cuda_fail(err, where);
    T* out = nullptr;
    dg_status st = run_stages<T>(op, q, tmp, res, t0, dt, nsteps, s, &out);
    if (st) return st;
    err = cudaEventRecord(pipe.comp_done[slot], s);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(pipe.d2h, pipe.comp_done[slot], 0);
    if (err == cudaSuccess) err = cudaMemcpyAsync(h_q[j], out, bytes, cudaMemcpyDeviceToHost, pipe.d2h);
    if (err == cudaSuccess) err = cudaEventRecord(pipe.free_slot[slot], pipe.d2h);
    if (err != cudaSuccess) return cuda_fail(err, where);
    pipe.used[slot] = true;
  }
  err = cudaStreamSynchronize(pipe.d2h);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return cuda_fail(err, "dg_step_host_jobs: synchronize");
  return DG_OK;
}

}  // namespace

extern "C" int64_t dg_step_host_jobs_work_bytes(const dg_op* op) {
  if (!op) return 0;
  return static_cast<int64_t>(2 * kJobSlots + 1) * 3 * op->fstride *
         static_cast<int64_t>(op->elem_size);
}

extern "C" dg_status dg_step_host_jobs(const dg_op* op, int32_t njobs, void* const* h_q,
                                       void* d_work, double t0, double dt, int32_t nsteps,
                                       void* stream) {
  dgw::clear_error();
  const char* where = "dg_step_host_jobs";
  dg_status st = check_device_op(op, where);
  if (st) return st;
  if (njobs < 0 || nsteps < 0 || !std::isfinite(dt))
    return fail(DG_ERR_ARG, "%s: bad njobs/nsteps/dt", where);
  if (njobs == 0) return DG_OK;
  if (!h_q) return fail(DG_ERR_ARG, "%s: h_q is NULL", where);
  for (int32_t j = 0; j < njobs; ++j)
    if (!h_q[j]) return fail(DG_ERR_ARG, "%s: h_q[%d] is NULL", where, j);
  if ((st = check_field(op, d_work, "d_work", where))) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (op->precision == DG_FP32)
    return run_jobs<float>(op, njobs, h_q, static_cast<float*>(d_work), t0, dt, nsteps, s);
  return run_jobs<double>(op, njobs, h_q, static_cast<double*>(d_work), t0, dt, nsteps, s);
}

extern "C" dg_status dg_check_finite(const dg_op* op, const void* d_q, void* stream) {
  dgw::clear_error();
  dg_status st = check_device_op(op, "dg_check_finite");
  if (st) return st;
  if ((st = check_field(op, d_q, "d_q", "dg_check_finite"))) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t err = cudaMemsetAsync(op->d_flag, 0, sizeof(int), s);
  if (err != cudaSuccess) return cuda_fail(err, "dg_check_finite: memset");
  const int64_t n = op->K * op->Np;
  const int threads = 256;
  const int64_t want = (3 * n + threads - 1) / threads;
  const int blocks = static_cast<int>(std::min<int64_t>(want, 8LL * std::max(op->num_sms, 1)));
  if (op->precision == DG_FP32)
    finite_scan_kernel<<<blocks, threads, 0, s>>>(static_cast<const float*>(d_q), nullptr,
                                                  op->fstride, n, op->d_flag);
  else
    finite_scan_kernel<<<blocks, threads, 0, s>>>(nullptr, static_cast<const double*>(d_q),
                                                  op->fstride, n, op->d_flag);
  err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_fail(err, "dg_check_finite: launch");
  op->launches.fetch_add(1, std::memory_order_relaxed);
  int flag = 0;
  err = cudaMemcpyAsync(&flag, op->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (err != cudaSuccess) return cuda_fail(err, "dg_check_finite: copy");
  err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return cuda_fail(err, "dg_check_finite: synchronize");
  if (flag) return fail(DG_ERR_NONFINITE, "dg_check_finite: field holds NaN or Inf");
  return DG_OK;
}

extern "C" dg_status dg_sync_check(const dg_op* op, void* stream) {
  dgw::clear_error();
  dg_status st = check_device_op(op, "dg_sync_check");
  if (st) return st;
  cudaError_t err = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (err == cudaSuccess) err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_fail(err, "dg_sync_check");
  int status = 0;
  err = cudaMemcpy(&status, op->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (err != cudaSuccess) return cuda_fail(err, "dg_sync_check: status read");
  if (status != 0) {
    cudaMemset(op->d_status, 0, sizeof(int));
    if (status & dgw::kStatusIndex)
      return fail(DG_ERR_INDEX, "dg_sync_check: a checked kernel found an index out of range");
    return fail(DG_ERR_TIMEOUT, "dg_sync_check: a kernel's bounded wait expired");
  }
  return DG_OK;
}

extern "C" dg_status dg_test_wait_timeout(const dg_op* op, void* stream) {
  dgw::clear_error();
  dg_status st = check_device_op(op, "dg_test_wait_timeout");
  if (st) return st;
  if (!op->use_tc || op->use_ept || op->precision != DG_FP32)
    return fail(DG_ERR_ARG, "dg_test_wait_timeout: needs an operator on the tensor-core kernel");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* gate = nullptr;
  cudaError_t err = dgw::dev_malloc(reinterpret_cast<void**>(&gate), sizeof(int));
  if (err == cudaSuccess) err = cudaMemsetAsync(gate, 0, sizeof(int), s);
  if (err == cudaSuccess) {
    dgw::StageArgs<float> a = base_args<float>(op);
    a.qin = static_cast<const float*>(op->d_qtmp);  // never read: the wait runs out first
    a.rhs = static_cast<float*>(op->d_qtmp);
    a.stall_gate = gate;
    err = launch_order<float>(op, a, dgw::kModeRhs, s);
    if (err == cudaSuccess) op->launches.fetch_add(1, std::memory_order_relaxed);
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (gate) cudaFree(gate);
  if (err != cudaSuccess) return cuda_fail(err, "dg_test_wait_timeout");
  return DG_OK;
}

extern "C" int64_t dg_launch_count(const dg_op* op) {
  return op ? op->launches.load(std::memory_order_relaxed) : 0;
}

extern "C" const char* dg_last_error(void) { return dgw::last_error_cstr(); }

// ============================================================ static scratch
// dg_step_static: the second field buffer of the stage ping-pong is this
// fixed device array (one instance per device, present once the library's
// device code is loaded) instead of the operator's own buffer.
static __device__ __align__(256) unsigned char g_step_scratch[DG_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
// per device: the context the address was looked up in (its process-unique
// id, 0 = none yet) and g_step_scratch's device address in that context
unsigned long long g_scratch_ctx[kMaxDevices] = {};
void* g_scratch_addr[kMaxDevices] = {};

// Driver calls reached through the runtime's entry-point table, so that the
// library links no driver library (types from cuda.h, plain function
// pointers).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Process-unique id of the calling thread's current context.  A context that
// is destroyed and created again (cudaDeviceReset, then any CUDA call) gets a
// new id, and loads the library's device code afresh, possibly at another
// address.  Called with g_scratch_mutex held.
dg_status current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    cudaError_t err = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000,
                                                       cudaEnableDefault, &q1);
    if (err == cudaSuccess)
      err = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (err != cudaSuccess) return cuda_fail(err, "dg_step_static: driver entry points");
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return fail(DG_ERR_CUDA, "dg_step_static: cuCtxGetCurrent / cuCtxGetId not available");
    get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, id) != CUDA_SUCCESS || *id == 0)
    return fail(DG_ERR_CUDA, "dg_step_static: no current CUDA context");
  return DG_OK;
}

// Device address of g_step_scratch on `device` (the caller made it
// current), looked up with cudaGetSymbolAddress once per device and context:
// again after the context was destroyed and re-created.
dg_status static_scratch(int device, void** out) {
  if (device < 0 || device >= kMaxDevices)
    return fail(DG_ERR_CUDA, "dg_step_static: device %d out of range", device);
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  unsigned long long ctx = 0;
  dg_status st = current_context_id(&ctx);
  if (st) return st;
  if (!g_scratch_addr[device] || g_scratch_ctx[device] != ctx) {
    void* p = nullptr;
    cudaError_t err = cudaGetSymbolAddress(&p, g_step_scratch);
    if (err != cudaSuccess) return cuda_fail(err, "dg_step_static: cudaGetSymbolAddress");
    g_scratch_addr[device] = p;
    g_scratch_ctx[device] = ctx;
  }
  *out = g_scratch_addr[device];
  return DG_OK;
}

// Same launch sequence as run_steps, with `tmp` as the ping-pong buffer.
template <typename T>
dg_status run_steps_static(const dg_op* op, T* q, T* res, double t0, double dt, int32_t nsteps,
                           T* tmp, cudaStream_t s) {
  dgw::StageArgs<T> a = base_args<T>(op);
  a.res = res;
  a.dt = static_cast<T>(dt);
  T* cur = q;
  T* other = tmp;
  for (int32_t n = 0; n < nsteps; ++n) {
    for (int i = 0; i < 5; ++i) {
      a.qin = cur;
      a.qout = other;
      a.a = static_cast<T>(op->lsrk_a[i]);
      a.b = static_cast<T>(op->lsrk_b[i]);
      const int mode = (i == 0) ? dgw::kModeFirstStage : dgw::kModeStage;
      cudaError_t err = launch_order<T>(op, a, mode, s);
      if (err != cudaSuccess) return cuda_fail(err, "dg_step_static: kernel launch");
      op->launches.fetch_add(1, std::memory_order_relaxed);
      err = stage_source<T>(op, other, res, t0 + n * dt, dt, i, s);
      if (err != cudaSuccess) return cuda_fail(err, "dg_step_static: point-source launch");
      std::swap(cur, other);
    }
  }
  if (cur != q) {
    cudaError_t err = cudaMemcpyAsync(q, cur, 3 * op->fstride * sizeof(T),
                                      cudaMemcpyDeviceToDevice, s);
    if (err != cudaSuccess) return cuda_fail(err, "dg_step_static: copy-back");
  }
  return DG_OK;
}

}  // namespace

extern "C" dg_status dg_step_static(const dg_op* op, void* d_q, void* d_res, double t0,
                                    double dt, int32_t nsteps, void* stream) {
  dgw::clear_error();
  dg_status st = check_device_op(op, "dg_step_static");  // makes op->device current
  if (st) return st;
  if ((st = check_field(op, d_q, "d_q", "dg_step_static"))) return st;
  if ((st = check_field(op, d_res, "d_res", "dg_step_static"))) return st;
  if (nsteps < 0) return fail(DG_ERR_ARG, "dg_step_static: nsteps = %d < 0", nsteps);
  if (!std::isfinite(dt) || !std::isfinite(t0))
    return fail(DG_ERR_ARG, "dg_step_static: dt or t0 is not finite");
  const size_t bytes = 3 * op->fstride * op->elem_size;
  if (bytes > static_cast<size_t>(DG_STATIC_SCRATCH_BYTES))
    return fail(DG_ERR_ARG,
                "dg_step_static: the fields need %zu bytes of scratch (K = %lld, N = %d), more "
                "than the %zu-byte static scratch; use dg_step",
                bytes, static_cast<long long>(op->K), op->N,
                static_cast<size_t>(DG_STATIC_SCRATCH_BYTES));
  if (overlaps(d_q, d_res, bytes))
    return fail(DG_ERR_ARG, "dg_step_static: d_q and d_res overlap");
  void* scratch = nullptr;
  if ((st = static_scratch(op->device, &scratch))) return st;
  if (overlaps(d_q, scratch, bytes) || overlaps(d_res, scratch, bytes))
    return fail(DG_ERR_ARG, "dg_step_static: buffer overlaps the static scratch");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The entries of each scratch field beyond K*Np never reach a result, but
  // the per-block bulk copies read them; zero them so that no value another
  // operator left there is ever read.
  const int64_t used = op->K * op->Np;
  const size_t tail = static_cast<size_t>(op->fstride - used) * op->elem_size;
  if (tail > 0) {
    for (int f = 0; f < 3; ++f) {
      unsigned char* p = static_cast<unsigned char*>(scratch) +
                         (static_cast<size_t>(f) * op->fstride + used) * op->elem_size;
      cudaError_t err = cudaMemsetAsync(p, 0, tail, s);
      if (err != cudaSuccess) return cuda_fail(err, "dg_step_static: cudaMemsetAsync");
    }
  }
  if (op->precision == DG_FP32)
    return run_steps_static<float>(op, static_cast<float*>(d_q), static_cast<float*>(d_res), t0,
                                   dt, nsteps, static_cast<float*>(scratch), s);
  return run_steps_static<double>(op, static_cast<double*>(d_q), static_cast<double*>(d_res), t0,
                                  dt, nsteps, static_cast<double*>(scratch), s);
}

namespace dgw {

dg_status upload_operator(dg_op* op, const std::vector<double>& rec,
                          const std::vector<int32_t>& conn) {
  const dg_status st =
      (op->precision == DG_FP32) ? upload<float>(op, rec, conn) : upload<double>(op, rec, conn);
  if (st != DG_OK) free_device(op);
  return st;
}

cudaError_t op_stage(const dg_op* op, const void* qin, void* qout, void* res, int stage,
                     double dt, cudaStream_t s) {
  const int mode = (stage == 0) ? kModeFirstStage : kModeStage;
  if (op->precision == DG_FP32) {
    StageArgs<float> a = base_args<float>(op);
    a.qin = static_cast<const float*>(qin);
    a.qout = static_cast<float*>(qout);
    a.res = static_cast<float*>(res);
    a.a = static_cast<float>(op->lsrk_a[stage]);
    a.b = static_cast<float>(op->lsrk_b[stage]);
    a.dt = static_cast<float>(dt);
    return launch_order<float>(op, a, mode, s);
  }
  StageArgs<double> a = base_args<double>(op);
  a.qin = static_cast<const double*>(qin);
  a.qout = static_cast<double*>(qout);
  a.res = static_cast<double*>(res);
  a.a = op->lsrk_a[stage];
  a.b = op->lsrk_b[stage];
  a.dt = dt;
  return launch_order<double>(op, a, mode, s);
}

}  // namespace dgw

extern "C" dg_status dg_test_fail_alloc(int32_t n) {
  dgw::clear_error();
  if (n < 0) return fail(DG_ERR_ARG, "dg_test_fail_alloc: n = %d < 0", n);
  dgw::g_fail_alloc.store(n, std::memory_order_relaxed);
  return DG_OK;
}

extern "C" int32_t dg_test_fail_alloc_pending(void) {
  return dgw::g_fail_alloc.load(std::memory_order_relaxed);
}
