// Private declarations shared by the host set-up (host_setup.cpp), the C ABI
// (api.cu) and the kernels (kernels.cuh).  Not part of the public interface.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "dgwave.h"

struct dg_mesh {
  int64_t K = 0;
  int64_t Nv = 0;
  std::vector<double> vx, vy;
  std::vector<int32_t> EToV;  // K*3, counter-clockwise
  std::vector<int32_t> EToE;  // K*3
  std::vector<int32_t> EToF;  // K*3
  int64_t n_flipped = 0;
  int64_t n_boundary = 0;
};

namespace dgw {

// Thread-local error message; returns `code` for convenient `return fail(...)`.
dg_status fail(dg_status code, const char* fmt, ...);
void clear_error();

// Reference triangle of order N, all FP64, row-major matrices.
struct RefElement {
  int N = 0, Np = 0, Nfp = 0, Nafp = 0;
  std::vector<double> r, s;        // Np
  std::vector<double> V;           // Np*Np, V[i*Np+j] = psi_j(r_i, s_i)
  std::vector<double> Dr, Ds;      // Np*Np
  std::vector<double> LIFT;        // Np*Nafp
  std::vector<int32_t> Fmask;      // 3*Nfp
  double lgl_gap = 0.0;            // spacing of the first two GLL points
};

RefElement build_reference(int N);

// Per-element geometry of an affine triangle mesh, FP64.
struct Geometry {
  std::vector<double> rx, ry, sx, sy, J;  // K
  std::vector<double> nx, ny, Fscale;     // 3K (index 3k+f)
  std::vector<double> x, y;               // K*Np
  // face connection codes, 3K: -1 on a boundary face, otherwise
  // kP*8 + fP*2 + rev where rev = 1 when face-node order is reversed
  std::vector<int32_t> conn;
  double min_inradius = 0.0;
};

Geometry build_geometry(const dg_mesh& mesh, const RefElement& ref);

// Point load delta(x - x_s) projected onto the nodal basis of the element
// that contains (xs, ys) (the lowest-numbered one whose barycentric
// coordinates are all >= -1e-12): w = M^-1 l(x_s) / J_k = V psi(r_s, s_s) /
// J_k.  Returns k, or -1 if no element contains the point.
int64_t point_source(const RefElement& R, const Geometry& G, int64_t K, double xs, double ys,
                     std::vector<double>& w);

// Face f's node j in the lattice numbering (same as RefElement::Fmask).
inline int face_node(int N, int f, int j) {
  // index of lattice point (row, col): rows below hold N+1, N, ... points
  auto idx = [N](int row, int col) { return row * (N + 1) - row * (row - 1) / 2 + col; };
  if (f == 0) return j;
  if (f == 1) return idx(j, N - j);
  return idx(j, 0);
}

// LSRK(5,4) 2N-storage coefficients and stage times.
void lsrk_coefficients(double a[5], double b[5], double c[5]);

// Device allocations of the library go through dev_malloc.  Test hook
// (dg_test_fail_alloc): while g_fail_alloc = n > 0, each allocation counts
// it down, and the one that takes it from 1 to 0 fails with
// cudaErrorMemoryAllocation without allocating.
extern std::atomic<int> g_fail_alloc;

template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  int n = g_fail_alloc.load(std::memory_order_relaxed);
  while (n > 0 && !g_fail_alloc.compare_exchange_weak(n, n - 1)) {
  }
  if (n == 1) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

}  // namespace dgw

// Operator handle (dg_op of the C ABI).
struct dg_op {
  int N = 0, Np = 0, Nfp = 0, Nafp = 0;
  int precision = DG_FP32;
  int flags = 0;
  int64_t K = 0, Kpad = 0, fstride = 0;
  size_t elem_size = 4;
  dgw::RefElement ref;
  dgw::Geometry geo;
  // per-element permittivity (dg_operator_setup_media); empty: eps = 1
  std::vector<double> eps;
  // min over elements of inradius / wave speed (wave speed 1 / sqrt(eps))
  double min_inradius_over_c = 0.0;
  // flux parameter of Eq. max2d-numflux: 1 upwind (default), 0 central
  double alpha = 1.0;
  int face_pairs = 0;  // dg_operator_set_face_pairs
  int tc_alt = 0;      // the tensor-core kernel's alternative block size (dg_operator_set_block_elems)
  // Ricker point source (dg_operator_set_source): element src_k, projected
  // point load in d_src_w (Np values of the field precision)
  bool has_src = false;
  int64_t src_k = -1;
  dg_point_source src{};
  void* d_src_w = nullptr;
  bool has_device = false;
  int device = 0;
  int num_sms = 0;
  void* d_Dr = nullptr;
  void* d_Ds = nullptr;
  void* d_LIFT = nullptr;
  void* d_lam = nullptr;   // vertex-interpolant weights per node
  void* d_geo = nullptr;
  void* d_conn = nullptr;
  void* d_qtmp = nullptr;  // second field buffer for the stage ping-pong
  int* d_flag = nullptr;   // finiteness scan result
  int* d_status = nullptr; // kernel status word (bounded-wait expiry)
  void* d_tcop = nullptr;  // tensor-core operator tiles for FP32 (see tc_operator_tiles)
  bool use_tc = false;     // FP32 products on the tensor cores
  bool use_ept = false;    // FP32: the element-thread kernel (takes precedence over use_tc)
  // FP32 operators of order <= kEptMaxN: the element-thread kernel's
  // reference tables (launch.h, ept_ops_floats)
  std::vector<float> ept_ops;
  int tc_prec = 0;         // their product variant (dgw::TcPrecision)
  double lsrk_a[5], lsrk_b[5], lsrk_c[5];
  mutable std::atomic<int64_t> launches{0};

  bool media() const { return !eps.empty(); }
};

namespace dgw {

// [Dr | Ds | LIFT | 1] as the B operand of the tensor-core kernel in the
// operand format of product variant `prec` (see api.cu).
std::vector<unsigned char> tc_operator_tiles(const RefElement& R, int prec);

// Geometry records of kGeoMedia values (layout in launch.h) for the K
// elements of `op`, with row scales sH = sh and sE = sh / eps_k, as doubles
// (out[k * kGeoMedia + i]); eps = 1 where the operator has none.
void media_records(const dg_op& op, double sh, std::vector<double>& out);

// Per-element records of `op` in the kernels' layout (kGeo values, or
// kGeoMedia for an operator with a permittivity) and its face connection
// codes (3 per element), K elements, as doubles.
void operator_records(const dg_op& op, std::vector<double>& rec, std::vector<int32_t>& conn);

// Uploads the reference-element tables of `op` and the given K element
// records and connection codes (padded to Kpad), and allocates its ping-pong
// field buffer (3 * fstride values), flag and status words.  `op` must have
// N, Np, Nafp, ref, precision, use_tc, tc_prec, elem_size, K, Kpad, fstride
// and eps (for media()) set.  On failure the partial device state is freed.
dg_status upload_operator(dg_op* op, const std::vector<double>& rec,
                          const std::vector<int32_t>& conn);

// One fused LSRK(5,4) stage (stage 0..4) of operator `op`: reads the fields
// qin and the residual res, writes the updated fields to qout and the new
// residual to res, asynchronously on stream s.
cudaError_t op_stage(const dg_op* op, const void* qin, void* qout, void* res, int stage,
                     double dt, cudaStream_t s);

}  // namespace dgw
