// FP64 host set-up of the nodal DG operator (Section "Implementation
// Aspects"): Warburton nodes, orthonormal-basis Vandermonde matrix, Dr/Ds,
// face mass matrices and LIFT, mesh connectivity, affine geometry, normals,
// Fscale and the face connection codes the kernels use.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <stdexcept>

#include "internal.h"

namespace dgw {

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

dg_status fail(dg_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

void clear_error() { g_last_error.clear(); }

const char* last_error_cstr() { return g_last_error.c_str(); }

// ------------------------------------------------------ 1D polynomials
// Orthonormal Jacobi polynomials p_k^(a,b) (weight (1-x)^a (1+x)^b) and
// their derivatives, from the normalised recurrence
//   x p_k = A_{k+1} p_{k+1} + B_k p_k + A_k p_{k-1},
// differentiated term by term for p_k'.
static double rec_A(int k, double a, double b) {
  const double c = 2.0 * k + a + b;
  return 2.0 / c * std::sqrt(k * (k + a + b) * (k + a) * (k + b) / ((c - 1.0) * (c + 1.0)));
}

static double rec_B(int k, double a, double b) {
  if (k == 0) return (b - a) / (a + b + 2.0);
  const double c = 2.0 * k + a + b;
  return (b * b - a * a) / (c * (c + 2.0));
}

static void jacobi_value_deriv(double x, double a, double b, int n, double* p, double* dp) {
  const double h0 = std::pow(2.0, a + b + 1.0) * std::tgamma(a + 1.0) * std::tgamma(b + 1.0) /
                    std::tgamma(a + b + 2.0);
  double pm = 0.0, dpm = 0.0;
  double pk = 1.0 / std::sqrt(h0), dpk = 0.0;
  for (int k = 0; k < n; ++k) {
    const double A1 = rec_A(k + 1, a, b);
    const double Bk = rec_B(k, a, b);
    const double Ak = (k == 0) ? 0.0 : rec_A(k, a, b);
    const double pn = ((x - Bk) * pk - Ak * pm) / A1;
    const double dpn = (pk + (x - Bk) * dpk - Ak * dpm) / A1;
    pm = pk;
    dpm = dpk;
    pk = pn;
    dpk = dpn;
  }
  *p = pk;
  if (dp) *dp = dpk;
}

// Classical Legendre P_n and its first two derivatives at x.
static void legendre3(int n, double x, double* P, double* dP, double* d2P) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0, e0 = 0.0, e1 = 0.0;
  if (n == 0) {
    *P = 1.0;
    *dP = 0.0;
    *d2P = 0.0;
    return;
  }
  for (int k = 1; k < n; ++k) {
    // (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}, differentiated twice
    const double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    const double d2 = ((2 * k + 1) * (p1 + x * d1) - k * d0) / (k + 1);
    const double e2 = ((2 * k + 1) * (2.0 * d1 + x * e1) - k * e0) / (k + 1);
    p0 = p1;
    p1 = p2;
    d0 = d1;
    d1 = d2;
    e0 = e1;
    e1 = e2;
  }
  *P = p1;
  *dP = d1;
  *d2P = e1;
}

// Gauss-Lobatto-Legendre points of order N: -1, 1 and the roots of P_N',
// by Newton's method from the Chebyshev-Lobatto points.
static std::vector<double> gll_points(int N) {
  std::vector<double> x(N + 1);
  x[0] = -1.0;
  x[N] = 1.0;
  for (int j = 1; j < N; ++j) {
    double t = -std::cos(M_PI * j / N);
    for (int it = 0; it < 100; ++it) {
      double P, dP, d2P;
      legendre3(N, t, &P, &dP, &d2P);
      const double step = dP / d2P;
      t -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    x[j] = t;
  }
  std::sort(x.begin(), x.end());
  return x;
}

// Gauss-Legendre rule with n points (roots of P_n), by Newton's method.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int j = 0; j < n; ++j) {
    double t = -std::cos(M_PI * (j + 0.75) / (n + 0.5));
    double P = 0, dP = 1, d2P = 0;
    for (int it = 0; it < 100; ++it) {
      legendre3(n, t, &P, &dP, &d2P);
      const double step = P / dP;
      t -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    legendre3(n, t, &P, &dP, &d2P);
    x[j] = t;
    w[j] = 2.0 / ((1.0 - t * t) * dP * dP);
  }
}

// ------------------------------------------------------------- helpers
// In-place inverse of a dense n x n row-major matrix (Gauss-Jordan with
// partial pivoting).
static void invert(std::vector<double>& A, int n) {
  std::vector<double> I(n * n, 0.0);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) throw std::runtime_error("singular matrix");
    if (piv != c) {
      for (int k = 0; k < n; ++k) {
        std::swap(A[c * n + k], A[piv * n + k]);
        std::swap(I[c * n + k], I[piv * n + k]);
      }
    }
    const double inv = 1.0 / A[c * n + c];
    for (int k = 0; k < n; ++k) {
      A[c * n + k] *= inv;
      I[c * n + k] *= inv;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        A[r * n + k] -= f * A[c * n + k];
        I[r * n + k] -= f * I[c * n + k];
      }
    }
  }
  A.swap(I);
}

// C = A (m x k) * B (k x n), row-major
static std::vector<double> matmul(const std::vector<double>& A, const std::vector<double>& B, int m,
                                  int k, int n) {
  std::vector<double> C(static_cast<size_t>(m) * n, 0.0);
  for (int i = 0; i < m; ++i)
    for (int l = 0; l < k; ++l) {
      const double a = A[i * k + l];
      if (a == 0.0) continue;
      for (int j = 0; j < n; ++j) C[i * n + j] += a * B[l * n + j];
    }
  return C;
}

// Lagrange basis on `nodes` evaluated at t.
static double lagrange(const std::vector<double>& nodes, int i, double t) {
  double v = 1.0;
  for (size_t j = 0; j < nodes.size(); ++j)
    if (static_cast<int>(j) != i) v *= (t - nodes[j]) / (nodes[i] - nodes[j]);
  return v;
}

// --------------------------------------------------- Warburton nodes
static double warburton_alpha(int N) {
  static const double table[] = {0.0,    0.0,    0.0,    1.4152, 0.1001, 0.2751,
                                 0.9800, 1.0999, 1.2832, 1.3648, 1.4773};
  return (N <= 10) ? table[N] : 5.0 / 3.0;
}

// Warp-and-blend construction on the equilateral triangle
// A = (-1, -1/sqrt3), B = (1, -1/sqrt3), C = (0, 2/sqrt3): each equidistant
// lattice point moves along every edge (P -> Q, opposite vertex R) by
//   4 l_P l_Q (1 + (alpha l_R)^2) * g(l_Q - l_P),
// g(t) = [interpolated (GLL - equidistant) shift at t] / (1 - t^2); then the
// moved point's barycentrics place it on the reference triangle
// (A -> (-1,-1), B -> (1,-1), C -> (-1,1)).
static void warburton_nodes(int N, std::vector<double>& r, std::vector<double>& s) {
  const double alpha = warburton_alpha(N);
  const std::vector<double> gll = gll_points(N);
  std::vector<double> equi(N + 1), shift(N + 1);
  for (int i = 0; i <= N; ++i) {
    equi[i] = -1.0 + 2.0 * i / N;
    shift[i] = gll[i] - equi[i];
  }
  auto g = [&](double t) {
    if (std::fabs(t) >= 1.0 - 1e-10) return 0.0;
    double w = 0.0;
    for (int i = 0; i <= N; ++i) w += shift[i] * lagrange(equi, i, t);
    return w / (1.0 - t * t);
  };
  const double sq3 = std::sqrt(3.0);
  const double Ax = -1.0, Ay = -1.0 / sq3, Bx = 1.0, By = -1.0 / sq3, Cx = 0.0, Cy = 2.0 / sq3;
  // unit edge directions
  auto unit = [](double x, double y, double* ux, double* uy) {
    const double n = std::sqrt(x * x + y * y);
    *ux = x / n;
    *uy = y / n;
  };
  double dABx, dABy, dBCx, dBCy, dCAx, dCAy;
  unit(Bx - Ax, By - Ay, &dABx, &dABy);
  unit(Cx - Bx, Cy - By, &dBCx, &dBCy);
  unit(Ax - Cx, Ay - Cy, &dCAx, &dCAy);
  r.clear();
  s.clear();
  for (int row = 0; row <= N; ++row) {
    for (int col = 0; col + row <= N; ++col) {
      const double lB = static_cast<double>(col) / N;
      const double lC = static_cast<double>(row) / N;
      const double lA = 1.0 - lB - lC;
      double X = lA * Ax + lB * Bx + lC * Cx;
      double Y = lA * Ay + lB * By + lC * Cy;
      const double mAB = 4.0 * lA * lB * (1.0 + (alpha * lC) * (alpha * lC)) * g(lB - lA);
      const double mBC = 4.0 * lB * lC * (1.0 + (alpha * lA) * (alpha * lA)) * g(lC - lB);
      const double mCA = 4.0 * lC * lA * (1.0 + (alpha * lB) * (alpha * lB)) * g(lA - lC);
      X += mAB * dABx + mBC * dBCx + mCA * dCAx;
      Y += mAB * dABy + mBC * dBCy + mCA * dCAy;
      // barycentrics of the moved point (C's from Y, then A/B from X)
      const double c3 = (sq3 * Y + 1.0) / 3.0;
      const double b3 = 0.5 * (1.0 - c3 + X);
      const double a3 = 0.5 * (1.0 - c3 - X);
      r.push_back(-a3 + b3 - c3);
      s.push_back(-a3 - b3 + c3);
    }
  }
}

// ------------------------------------------- orthonormal simplex basis
// psi_ij(r, s) = sqrt2 p_i^(0,0)(a) p_j^(2i+1,0)(b) (1-b)^i with the
// collapsed coordinates a = 2(1+r)/(1-s) - 1 (a = -1 at s = 1), b = s, and
// its r/s derivatives by the chain rule, written with (1-b)^(i-1).
static void simplex_psi(int i, int j, double r, double s, double* psi, double* dr, double* ds) {
  const double a = (std::fabs(1.0 - s) > 1e-14) ? 2.0 * (1.0 + r) / (1.0 - s) - 1.0 : -1.0;
  const double b = s;
  double fa, dfa, gb, dgb;
  jacobi_value_deriv(a, 0.0, 0.0, i, &fa, &dfa);
  jacobi_value_deriv(b, 2.0 * i + 1.0, 0.0, j, &gb, &dgb);
  const double sq2 = std::sqrt(2.0);
  const double omb = 1.0 - b;
  *psi = sq2 * fa * gb * std::pow(omb, i);
  if (i == 0) {
    *dr = 0.0;
    *ds = sq2 * fa * dgb;
  } else {
    const double w = std::pow(omb, i - 1);
    *dr = sq2 * 2.0 * dfa * gb * w;
    *ds = sq2 * (dfa * (1.0 + a) * gb * w + fa * (dgb * omb * w * 1.0 - i * gb * w));
  }
}

RefElement build_reference(int N) {
  RefElement R;
  R.N = N;
  R.Np = (N + 1) * (N + 2) / 2;
  R.Nfp = N + 1;
  R.Nafp = 3 * R.Nfp;
  const int Np = R.Np, Nfp = R.Nfp, Nafp = R.Nafp;
  warburton_nodes(N, R.r, R.s);

  // Vandermonde and its derivatives; basis order (i, j), i outer
  std::vector<double> V(Np * Np), Vr(Np * Np), Vs(Np * Np);
  for (int n = 0; n < Np; ++n) {
    int col = 0;
    for (int i = 0; i <= N; ++i)
      for (int j = 0; i + j <= N; ++j, ++col)
        simplex_psi(i, j, R.r[n], R.s[n], &V[n * Np + col], &Vr[n * Np + col], &Vs[n * Np + col]);
  }
  R.V = V;
  std::vector<double> Vinv = V;
  invert(Vinv, Np);
  R.Dr = matmul(Vr, Vinv, Np, Np, Np);
  R.Ds = matmul(Vs, Vinv, Np, Np, Np);

  // face node table
  R.Fmask.resize(3 * Nfp);
  for (int f = 0; f < 3; ++f)
    for (int j = 0; j < Nfp; ++j) R.Fmask[f * Nfp + j] = face_node(N, f, j);

  // combined face mass matrix E (Np x Nafp): each face's 1D mass matrix in
  // its own coordinate (r on faces 0 and 1, s on face 2), by Gauss-Legendre
  // quadrature of products of the 1D Lagrange polynomials on the face nodes
  std::vector<double> gx, gw;
  gauss_legendre(N + 1, gx, gw);
  std::vector<double> E(static_cast<size_t>(Np) * Nafp, 0.0);
  for (int f = 0; f < 3; ++f) {
    std::vector<double> fn(Nfp);
    for (int j = 0; j < Nfp; ++j) {
      const int n = R.Fmask[f * Nfp + j];
      fn[j] = (f == 2) ? R.s[n] : R.r[n];
    }
    for (int i = 0; i < Nfp; ++i)
      for (int j = 0; j < Nfp; ++j) {
        double m = 0.0;
        for (size_t q = 0; q < gx.size(); ++q)
          m += gw[q] * lagrange(fn, i, gx[q]) * lagrange(fn, j, gx[q]);
        E[static_cast<size_t>(R.Fmask[f * Nfp + i]) * Nafp + f * Nfp + j] = m;
      }
  }
  // LIFT = M^{-1} E with M^{-1} = V V^T
  std::vector<double> Vt(Np * Np);
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) Vt[j * Np + i] = V[i * Np + j];
  const std::vector<double> Minv = matmul(V, Vt, Np, Np, Np);
  R.LIFT = matmul(Minv, E, Np, Np, Nafp);

  const std::vector<double> gll = gll_points(N);
  R.lgl_gap = gll[1] - gll[0];
  return R;
}

// ------------------------------------------------------------ geometry
Geometry build_geometry(const dg_mesh& mesh, const RefElement& ref) {
  Geometry G;
  const int64_t K = mesh.K;
  const int Np = ref.Np, N = ref.N;
  G.rx.resize(K);
  G.ry.resize(K);
  G.sx.resize(K);
  G.sy.resize(K);
  G.J.resize(K);
  G.nx.resize(3 * K);
  G.ny.resize(3 * K);
  G.Fscale.resize(3 * K);
  G.x.resize(static_cast<size_t>(K) * Np);
  G.y.resize(static_cast<size_t>(K) * Np);
  G.conn.resize(3 * K);
  double min_in = 1e300;
  for (int64_t k = 0; k < K; ++k) {
    const int32_t* v = &mesh.EToV[3 * k];
    const double x1 = mesh.vx[v[0]], y1 = mesh.vy[v[0]];
    const double x2 = mesh.vx[v[1]], y2 = mesh.vy[v[1]];
    const double x3 = mesh.vx[v[2]], y3 = mesh.vy[v[2]];
    // affine map x = (-(r+s) v1 + (1+r) v2 + (1+s) v3)/2: constant derivatives
    const double xr = 0.5 * (x2 - x1), xs = 0.5 * (x3 - x1);
    const double yr = 0.5 * (y2 - y1), ys = 0.5 * (y3 - y1);
    const double J = xr * ys - xs * yr;
    G.J[k] = J;
    G.rx[k] = ys / J;
    G.ry[k] = -xs / J;
    G.sx[k] = -yr / J;
    G.sy[k] = xr / J;
    const double ex[3] = {x2 - x1, x3 - x2, x1 - x3};
    const double ey[3] = {y2 - y1, y3 - y2, y1 - y3};
    double perim = 0.0;
    for (int f = 0; f < 3; ++f) {
      const double len = std::sqrt(ex[f] * ex[f] + ey[f] * ey[f]);
      perim += len;
      // outward normal of a counter-clockwise triangle: edge rotated by -90
      G.nx[3 * k + f] = ey[f] / len;
      G.ny[3 * k + f] = -ex[f] / len;
      // edge parametrised over [-1, 1]: surface Jacobian len/2
      G.Fscale[3 * k + f] = (0.5 * len) / J;
    }
    min_in = std::min(min_in, 2.0 * J / (0.5 * perim));  // area = 2J
    for (int n = 0; n < Np; ++n) {
      const double r = ref.r[n], s = ref.s[n];
      G.x[k * Np + n] = 0.5 * (-(r + s) * x1 + (1.0 + r) * x2 + (1.0 + s) * x3);
      G.y[k * Np + n] = 0.5 * (-(r + s) * y1 + (1.0 + r) * y2 + (1.0 + s) * y3);
    }
    // face connection codes.  In node order, face 0 runs v1 -> v2, face 1
    // runs v2 -> v3 and face 2 runs v1 -> v3; the neighbour's face nodes are
    // in the same order when both faces start at the same vertex.
    for (int f = 0; f < 3; ++f) {
      const int64_t kP = mesh.EToE[3 * k + f];
      const int fP = mesh.EToF[3 * k + f];
      if (kP == k && fP == f) {
        G.conn[3 * k + f] = -1;
        continue;
      }
      const int32_t start = (f == 1) ? v[1] : v[0];
      const int32_t* vP = &mesh.EToV[3 * kP];
      const int32_t startP = (fP == 1) ? vP[1] : vP[0];
      const int rev = (start == startP) ? 0 : 1;
      G.conn[3 * k + f] = static_cast<int32_t>(kP * 8 + fP * 2 + rev);
    }
  }
  G.min_inradius = min_in;
  (void)N;
  return G;
}

// ------------------------------------------------------- point source
int64_t point_source(const RefElement& R, const Geometry& G, int64_t K, double xs, double ys,
                     std::vector<double>& w) {
  const int N = R.N, Np = R.Np;
  for (int64_t k = 0; k < K; ++k) {
    // vertices are the nodes 0 (v1), N (v2) and Np - 1 (v3)
    const double x1 = G.x[k * Np], y1 = G.y[k * Np];
    const double x2 = G.x[k * Np + N], y2 = G.y[k * Np + N];
    const double x3 = G.x[k * Np + Np - 1], y3 = G.y[k * Np + Np - 1];
    const double det = (x2 - x1) * (y3 - y1) - (x3 - x1) * (y2 - y1);
    const double l2 = ((xs - x1) * (y3 - y1) - (x3 - x1) * (ys - y1)) / det;
    const double l3 = ((x2 - x1) * (ys - y1) - (xs - x1) * (y2 - y1)) / det;
    const double l1 = 1.0 - l2 - l3;
    if (l1 < -1e-12 || l2 < -1e-12 || l3 < -1e-12) continue;
    const double r = 2.0 * l2 - 1.0, s = 2.0 * l3 - 1.0;
    // M^-1 l(x_s) = V V^T V^-T psi(r, s) = V psi(r, s)
    std::vector<double> psi(Np);
    int col = 0;
    for (int i = 0; i <= N; ++i)
      for (int j = 0; i + j <= N; ++j, ++col) {
        double dr, ds;
        simplex_psi(i, j, r, s, &psi[col], &dr, &ds);
      }
    w.assign(Np, 0.0);
    for (int n = 0; n < Np; ++n) {
      double acc = 0.0;
      for (int c = 0; c < Np; ++c) acc += R.V[n * Np + c] * psi[c];
      w[n] = acc / G.J[k];
    }
    return k;
  }
  return -1;
}

// --------------------------------------------------------------- LSRK
void lsrk_coefficients(double a[5], double b[5], double c[5]) {
  // Carpenter & Kennedy (1994), five-stage fourth-order 2N-storage scheme
  const double A[5] = {0.0, -567301805773.0 / 1357537059087.0,
                       -2404267990393.0 / 2016746695238.0, -3550918686646.0 / 2091501179385.0,
                       -1275806237668.0 / 842570457699.0};
  const double B[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                       1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                       2277821191437.0 / 14882151754819.0};
  for (int i = 0; i < 5; ++i) {
    a[i] = A[i];
    b[i] = B[i];
  }
  // stage times: stage i evaluates at u_{i-1} = u_0 + dt sum_j w_ij f_j;
  // run the 2N-storage recurrence on the coefficient vectors to get the
  // row sums c_i = sum_j w_ij
  double kvec = 0.0, cu = 0.0;  // sums of the residual / solution weights
  for (int i = 0; i < 5; ++i) {
    c[i] = cu;
    kvec = A[i] * kvec + 1.0;  // one new f with weight 1 in the residual
    cu = cu + B[i] * kvec;
  }
}

}  // namespace dgw

// ======================================================= mesh C ABI
using dgw::fail;

extern "C" dg_status dg_mesh_create(const double* vx, const double* vy, int64_t Nv,
                                    const int32_t* EToV, int64_t K, dg_mesh** out) {
  dgw::clear_error();
  if (!vx || !vy || !EToV || !out) return fail(DG_ERR_ARG, "dg_mesh_create: NULL argument");
  if (Nv < 3) return fail(DG_ERR_ARG, "dg_mesh_create: Nv = %lld < 3", (long long)Nv);
  if (K < 1) return fail(DG_ERR_ARG, "dg_mesh_create: K = %lld < 1", (long long)K);
  if (K >= (int64_t(1) << 28))
    return fail(DG_ERR_ARG, "dg_mesh_create: K = %lld exceeds 2^28 - 1", (long long)K);
  dg_mesh* m = nullptr;
  try {
    m = new dg_mesh;
    m->K = K;
    m->Nv = Nv;
    m->vx.assign(vx, vx + Nv);
    m->vy.assign(vy, vy + Nv);
    m->EToV.assign(EToV, EToV + 3 * K);
    for (int64_t i = 0; i < 3 * K; ++i) {
      if (m->EToV[i] < 0 || m->EToV[i] >= Nv) {
        const int bad = m->EToV[i];
        delete m;
        return fail(DG_ERR_ARG, "dg_mesh_create: EToV[%lld] = %d out of range", (long long)i,
                    bad);
      }
    }
    for (int64_t k = 0; k < K; ++k) {
      int32_t* v = &m->EToV[3 * k];
      const double a2 = (m->vx[v[1]] - m->vx[v[0]]) * (m->vy[v[2]] - m->vy[v[0]]) -
                        (m->vx[v[2]] - m->vx[v[0]]) * (m->vy[v[1]] - m->vy[v[0]]);
      if (!(a2 != 0.0) || !std::isfinite(a2)) {
        delete m;
        return fail(DG_ERR_MESH_DEGENERATE, "dg_mesh_create: element %lld has zero area",
                    (long long)k);
      }
      if (a2 < 0) {
        std::swap(v[1], v[2]);
        ++m->n_flipped;
      }
    }
    // faces keyed by their sorted vertex pair; equal keys are the same face
    struct FaceRec {
      uint64_t key;
      int64_t k;
      int f;
    };
    std::vector<FaceRec> faces(3 * K);
    for (int64_t k = 0; k < K; ++k)
      for (int f = 0; f < 3; ++f) {
        uint64_t a = static_cast<uint32_t>(m->EToV[3 * k + f]);
        uint64_t b = static_cast<uint32_t>(m->EToV[3 * k + (f + 1) % 3]);
        if (a > b) std::swap(a, b);
        faces[3 * k + f] = {a * static_cast<uint64_t>(Nv) + b, k, f};
      }
    std::sort(faces.begin(), faces.end(), [](const FaceRec& x, const FaceRec& y) {
      return x.key != y.key ? x.key < y.key : (x.k != y.k ? x.k < y.k : x.f < y.f);
    });
    m->EToE.resize(3 * K);
    m->EToF.resize(3 * K);
    for (int64_t k = 0; k < K; ++k)
      for (int f = 0; f < 3; ++f) {
        m->EToE[3 * k + f] = static_cast<int32_t>(k);
        m->EToF[3 * k + f] = f;
      }
    size_t i = 0;
    while (i < faces.size()) {
      size_t j = i + 1;
      while (j < faces.size() && faces[j].key == faces[i].key) ++j;
      if (j - i > 2) {
        const int64_t kk = faces[i].k;
        delete m;
        return fail(DG_ERR_MESH_NONCONFORMING,
                    "dg_mesh_create: a face of element %lld is shared by %zu elements",
                    (long long)kk, j - i);
      }
      if (j - i == 2) {
        const FaceRec& p = faces[i];
        const FaceRec& q = faces[i + 1];
        m->EToE[3 * p.k + p.f] = static_cast<int32_t>(q.k);
        m->EToF[3 * p.k + p.f] = q.f;
        m->EToE[3 * q.k + q.f] = static_cast<int32_t>(p.k);
        m->EToF[3 * q.k + q.f] = p.f;
      } else {
        ++m->n_boundary;
      }
      i = j;
    }
  } catch (const std::bad_alloc&) {
    delete m;
    return fail(DG_ERR_OOM, "dg_mesh_create: out of host memory");
  }
  *out = m;
  return DG_OK;
}

extern "C" dg_status dg_mesh_info(const dg_mesh* mesh, int64_t* K, int64_t* n_flipped,
                                  int64_t* n_boundary_faces) {
  dgw::clear_error();
  if (!mesh) return fail(DG_ERR_ARG, "dg_mesh_info: NULL mesh");
  if (K) *K = mesh->K;
  if (n_flipped) *n_flipped = mesh->n_flipped;
  if (n_boundary_faces) *n_boundary_faces = mesh->n_boundary;
  return DG_OK;
}

extern "C" dg_status dg_mesh_connectivity(const dg_mesh* mesh, int32_t* EToE, int32_t* EToF,
                                          int32_t* EToV_out) {
  dgw::clear_error();
  if (!mesh) return fail(DG_ERR_ARG, "dg_mesh_connectivity: NULL mesh");
  const size_t n = 3 * static_cast<size_t>(mesh->K);
  if (EToE) std::memcpy(EToE, mesh->EToE.data(), n * sizeof(int32_t));
  if (EToF) std::memcpy(EToF, mesh->EToF.data(), n * sizeof(int32_t));
  if (EToV_out) std::memcpy(EToV_out, mesh->EToV.data(), n * sizeof(int32_t));
  return DG_OK;
}

extern "C" void dg_mesh_destroy(dg_mesh* mesh) { delete mesh; }

extern "C" dg_status dg_lsrk_coefficients(double* a, double* b, double* c) {
  double A[5], B[5], C[5];
  dgw::lsrk_coefficients(A, B, C);
  for (int i = 0; i < 5; ++i) {
    if (a) a[i] = A[i];
    if (b) b[i] = B[i];
    if (c) c[i] = C[i];
  }
  return DG_OK;
}
