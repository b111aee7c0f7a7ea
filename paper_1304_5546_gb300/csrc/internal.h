// Private declarations shared by the host set-up (host_setup.cpp), the C ABI
// (api.cu) and the kernels (kernels.cuh).  Not part of the public interface.
#pragma once

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

}  // namespace dgw
