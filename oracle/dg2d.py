"""ORACLE (test infrastructure only): plain FP64 nodal DG for 2D TM Maxwell.

Follows the chapter "Solving Wave Equations on Unstructured Geometries"
(Kloeckner, Warburton, Hesthaven):

* Section "A Precise Mathematical Problem Statement", Eq. tm-maxwells: the
  TM system for (Hx, Hy, Ez), eps = mu = 1, PEC wall Ez = 0.
* Section "Construction of the Method", Eq. dg-strong and Eq.
  max2d-numflux: strong DG form with the upwind flux (alpha = 1; alpha = 0
  is the central flux).
* Section "Implementation Aspects", Eqs. dg-diff-local-to-global,
  dg-strong-matrix, dg-lift, dg-strong-explicit: affine element maps,
  reference differentiation matrices, the chain rule, face mass matrices and
  the LIFT matrix, Lagrange basis on the Warburton nodes built through the
  orthonormal (Koornwinder-Dubiner) basis.
* Section "Computing the Surface Contribution": the boundary indicator
  (Ez+ = -Ez-, H+ = H- at PEC faces) and Fscale = surface Jacobian / volume
  Jacobian; the flux enters the right-hand side with a factor 1/2 (the
  chapter's CPU and GPU listings both carry it; Eq. max2d-numflux as printed
  does not -- reading: keep the 1/2, which makes alpha = 0 the central flux
  of Eq. dg-strong).
* "a simple Runge-Kutta time integrator": read as the Carpenter-Kennedy
  five-stage fourth-order 2N-storage scheme, LSRK(5,4).

Array conventions: fields are float64 arrays of shape (3, K, Np) ordered
(Hx, Hy, Ez); element k's node n is q[:, k, n]; nodes are numbered row by
row of the equidistant lattice (rows of constant s from s = -1 upward, r
increasing within a row).

Parity status: every function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py``.  The Warburton blending parameters
(``WARBURTON_ALPHA``) are a reading (the chapter cites the table but does not
print it); the node-set properties that do not depend on them are pinned.
"""
import math

import numpy as np

# ---------------------------------------------------------------------------
# 1D building blocks: orthonormal Jacobi polynomials and Gauss(-Lobatto) nodes
# ---------------------------------------------------------------------------


def _jacobi_norm2(a, b, n):
    """Squared L2 norm of the classical Jacobi polynomial P_n^(a,b) under the
    weight (1-x)^a (1+x)^b on [-1, 1]."""
    return (2.0 ** (a + b + 1) / (2 * n + a + b + 1)
            * math.gamma(n + a + 1) * math.gamma(n + b + 1)
            / (math.gamma(n + a + b + 1) * math.factorial(n)))


def jacobi_p(x, a, b, n):
    """Orthonormal Jacobi polynomial of degree n at points x.

    The classical polynomial comes from the standard three-term recurrence
    (P_0 = 1, P_1 = ((a - b) + (a + b + 2) x) / 2) and is divided by the
    square root of its weighted norm.
    """
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0 / math.sqrt(_jacobi_norm2(a, b, 0))
    p1 = 0.5 * ((a - b) + (a + b + 2) * x)
    for m in range(1, n):
        c = 2 * m + a + b
        lead = 2.0 * (m + 1) * (m + a + b + 1) * c
        p2 = ((c + 1) * ((c + 2) * c * x + a * a - b * b) * p1
              - 2.0 * (m + a) * (m + b) * (c + 2) * p0) / lead
        p0, p1 = p1, p2
    return p1 / math.sqrt(_jacobi_norm2(a, b, n))


def grad_jacobi_p(x, a, b, n):
    """d/dx of the orthonormal Jacobi polynomial: sqrt(n (n+a+b+1)) times the
    orthonormal polynomial of degree n-1 with parameters (a+1, b+1)."""
    x = np.asarray(x, dtype=np.float64)
    if n == 0:
        return np.zeros_like(x)
    return math.sqrt(n * (n + a + b + 1)) * jacobi_p(x, a + 1, b + 1, n - 1)


def gauss_jacobi_nodes(a, b, m):
    """The m roots of P_m^(a,b), as the eigenvalues of the symmetric tridiagonal
    Jacobi matrix of the orthonormal recurrence (Golub-Welsch)."""
    if m <= 0:
        return np.zeros(0)
    k = np.arange(m, dtype=np.float64)
    c = 2 * k + a + b
    diag = np.empty(m)
    diag[0] = (b - a) / (a + b + 2)
    if m > 1:
        kk = k[1:]
        cc = c[1:]
        diag[1:] = (b * b - a * a) / (cc * (cc + 2))
        off = (2.0 / cc) * np.sqrt(kk * (kk + a) * (kk + b) * (kk + a + b)
                                   / ((cc - 1) * (cc + 1)))
    else:
        off = np.zeros(0)
    Jm = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    return np.sort(np.linalg.eigvalsh(Jm))


def lgl_nodes(N):
    """Legendre-Gauss-Lobatto nodes of order N: -1, 1 and the N-1 roots of
    P_{N-1}^(1,1) (the interior extrema of the Legendre polynomial P_N)."""
    if N < 1:
        raise ValueError("N >= 1")
    return np.concatenate([[-1.0], gauss_jacobi_nodes(1.0, 1.0, N - 1), [1.0]])


def vandermonde_1d(N, r):
    """V[i, j] = orthonormal Legendre polynomial j at r[i]."""
    return np.stack([jacobi_p(r, 0.0, 0.0, j) for j in range(N + 1)], axis=1)


# ---------------------------------------------------------------------------
# Warburton warp-and-blend nodes on the triangle
# ---------------------------------------------------------------------------

#: Blending parameter alpha per order N (Warburton 2006, as cited in Section
#: "Construction of the Method" for the choice of interpolation points).
#: Reading: the chapter names the construction but not the values.
WARBURTON_ALPHA = {1: 0.0, 2: 0.0, 3: 1.4152, 4: 0.1001, 5: 0.2751,
                   6: 0.9800, 7: 1.0999, 8: 1.2832, 9: 1.3648, 10: 1.4773}


def _equidistant_lagrange(N, t):
    """Lagrange basis on N+1 equidistant points of [-1, 1], evaluated at t:
    returns L[m, i] = l_i(t[m])."""
    xe = np.linspace(-1.0, 1.0, N + 1)
    t = np.asarray(t, dtype=np.float64)
    L = np.ones((t.size, N + 1))
    for i in range(N + 1):
        for j in range(N + 1):
            if j != i:
                L[:, i] *= (t - xe[j]) / (xe[i] - xe[j])
    return L


def warp_function(N, t):
    """Edge warp of the warp-and-blend construction: the interpolant on
    equidistant points of the shift (LGL node - equidistant node), divided by
    (1 - t^2) away from the edge end points (where it is set to 0)."""
    t = np.asarray(t, dtype=np.float64)
    shift = lgl_nodes(N) - np.linspace(-1.0, 1.0, N + 1)
    w = _equidistant_lagrange(N, t) @ shift
    denom = 1.0 - t * t
    inside = np.abs(t) < 1.0 - 1e-10
    out = np.zeros_like(t)
    out[inside] = w[inside] / denom[inside]
    return out


def nodes_2d(N, alpha=None):
    """Warburton nodes (r, s) on the reference triangle v1=(-1,-1), v2=(1,-1),
    v3=(-1,1), in lattice order (rows of constant s bottom-up, r increasing).

    Construction on the equilateral triangle A=(-1,-1/sqrt3), B=(1,-1/sqrt3),
    C=(0,2/sqrt3) with barycentrics (la, lb, lc): every equidistant lattice
    point is displaced along each edge's direction by
    4 l_i l_j (1 + (alpha l_k)^2) warp(l_j - l_i), where (i -> j) runs along
    the edge and k is the opposite vertex; the point is then mapped affinely
    (same barycentrics) to the reference triangle A->v1, B->v2, C->v3.
    """
    if alpha is None:
        alpha = WARBURTON_ALPHA.get(N, 5.0 / 3.0)
    lb_list, lc_list = [], []
    for row in range(N + 1):
        for col in range(N + 1 - row):
            lb_list.append(col / N)
            lc_list.append(row / N)
    lb = np.array(lb_list)
    lc = np.array(lc_list)
    la = 1.0 - lb - lc
    s3 = math.sqrt(3.0)
    A = np.array([-1.0, -1.0 / s3])
    B = np.array([1.0, -1.0 / s3])
    C = np.array([0.0, 2.0 / s3])
    X = la * A[0] + lb * B[0] + lc * C[0]
    Y = la * A[1] + lb * B[1] + lc * C[1]
    # (start-vertex barycentric, end-vertex barycentric, opposite barycentric,
    #  unit direction start -> end)
    edges = [
        (la, lb, lc, (B - A) / np.linalg.norm(B - A)),
        (lb, lc, la, (C - B) / np.linalg.norm(C - B)),
        (lc, la, lb, (A - C) / np.linalg.norm(A - C)),
    ]
    dX = np.zeros_like(X)
    dY = np.zeros_like(Y)
    for li, lj, lk, d in edges:
        amp = 4.0 * li * lj * (1.0 + (alpha * lk) ** 2) * warp_function(N, lj - li)
        dX += amp * d[0]
        dY += amp * d[1]
    X = X + dX
    Y = Y + dY
    # back to barycentrics, then to (r, s)
    lc2 = (s3 * Y + 1.0) / 3.0
    lb2 = (1.0 - lc2 + X) / 2.0
    la2 = (1.0 - lc2 - X) / 2.0
    r = -la2 + lb2 - lc2
    s = -la2 - lb2 + lc2
    return r, s


# ---------------------------------------------------------------------------
# Orthonormal basis on the triangle, Vandermonde, Dr/Ds, mass, LIFT
# ---------------------------------------------------------------------------


def rs_to_ab(r, s):
    """Collapsed coordinates a = 2(1+r)/(1-s) - 1 (a = -1 at s = 1), b = s."""
    r = np.asarray(r, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    a = np.full_like(r, -1.0)
    ok = np.abs(1.0 - s) > 1e-14
    a[ok] = 2.0 * (1.0 + r[ok]) / (1.0 - s[ok]) - 1.0
    return a, s.copy()


def simplex_basis(r, s, i, j):
    """Orthonormal Koornwinder-Dubiner polynomial psi_ij on the reference
    triangle: sqrt(2) P_i^(0,0)(a) P_j^(2i+1,0)(b) (1-b)^i."""
    a, b = rs_to_ab(r, s)
    return (math.sqrt(2.0) * jacobi_p(a, 0.0, 0.0, i)
            * jacobi_p(b, 2.0 * i + 1.0, 0.0, j) * (1.0 - b) ** i)


def grad_simplex_basis(r, s, i, j):
    """(d psi_ij/dr, d psi_ij/ds) by the chain rule through (a, b), written
    with (1-b)^(i-1) so that it is regular at the top vertex s = 1."""
    a, b = rs_to_ab(r, s)
    fa = jacobi_p(a, 0.0, 0.0, i)
    dfa = grad_jacobi_p(a, 0.0, 0.0, i)
    gb = jacobi_p(b, 2.0 * i + 1.0, 0.0, j)
    dgb = grad_jacobi_p(b, 2.0 * i + 1.0, 0.0, j)
    if i == 0:
        dr = np.zeros_like(a)
        ds = fa * dgb
    else:
        w = (1.0 - b) ** (i - 1)
        dr = 2.0 * dfa * gb * w
        ds = dfa * (1.0 + a) * gb * w + fa * (dgb * (1.0 - b) ** i - i * gb * w)
    c = math.sqrt(2.0)
    return c * dr, c * ds


def basis_indices(N):
    """Basis ordering (i, j) with i + j <= N, i outer."""
    return [(i, j) for i in range(N + 1) for j in range(N + 1 - i)]


def vandermonde_2d(N, r, s):
    return np.stack([simplex_basis(r, s, i, j) for i, j in basis_indices(N)], axis=1)


def grad_vandermonde_2d(N, r, s):
    cols = [grad_simplex_basis(r, s, i, j) for i, j in basis_indices(N)]
    Vr = np.stack([c[0] for c in cols], axis=1)
    Vs = np.stack([c[1] for c in cols], axis=1)
    return Vr, Vs


def face_masks(r, s, tol=1e-10):
    """Node indices on each face, in increasing node index:
    face 1: s = -1 (v1 -> v2); face 2: r + s = 0 (v2 -> v3);
    face 3: r = -1 (listed v1 -> v3)."""
    f1 = np.nonzero(np.abs(s + 1.0) < tol)[0]
    f2 = np.nonzero(np.abs(r + s) < tol)[0]
    f3 = np.nonzero(np.abs(r + 1.0) < tol)[0]
    return np.stack([f1, f2, f3])


class ReferenceElement:
    """Order-N reference triangle: nodes, V, Dr, Ds, M, Fmask, LIFT
    (Section "Implementation Aspects", Eqs. dg-diff-local-to-global and
    dg-lift)."""

    def __init__(self, N, alpha=None):
        if N < 1:
            raise ValueError("N >= 1")
        self.N = N
        self.Np = (N + 1) * (N + 2) // 2
        self.Nfp = N + 1
        self.Nfaces = 3
        self.Nafp = 3 * self.Nfp
        self.r, self.s = nodes_2d(N, alpha)
        self.V = vandermonde_2d(N, self.r, self.s)
        Vr, Vs = grad_vandermonde_2d(N, self.r, self.s)
        # D = V_r V^{-1}: solve V^T D^T = V_r^T
        self.Dr = np.linalg.solve(self.V.T, Vr.T).T
        self.Ds = np.linalg.solve(self.V.T, Vs.T).T
        self.M = np.linalg.inv(self.V @ self.V.T)
        self.Fmask = face_masks(self.r, self.s)
        # combined face mass matrix (Eq. dg-lift): each face's 1D mass matrix
        # (in the face's own coordinate, r on faces 1 and 2, s on face 3)
        # placed at that face's node rows.
        E = np.zeros((self.Np, self.Nafp))
        for f in range(3):
            coord = self.s if f == 2 else self.r
            V1 = vandermonde_1d(N, coord[self.Fmask[f]])
            mass1 = np.linalg.inv(V1 @ V1.T)
            E[np.ix_(self.Fmask[f], np.arange(f * self.Nfp, (f + 1) * self.Nfp))] = mass1
        self.Emat = E
        # LIFT = M^{-1} E = V V^T E
        self.LIFT = self.V @ (self.V.T @ E)


# ---------------------------------------------------------------------------
# Mesh: orientation, connectivity, nodal coordinates, geometry, maps
# ---------------------------------------------------------------------------


class MeshError(ValueError):
    pass


def orient_ccw(VX, VY, EToV):
    """Re-list clockwise triangles counter-clockwise by swapping their 2nd and
    3rd vertices; returns (EToV, number flipped).  Zero-area triangles raise."""
    EToV = np.array(EToV, dtype=np.int64, copy=True)
    x = VX[EToV]
    y = VY[EToV]
    area2 = (x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0])
    if np.any(area2 == 0):
        raise MeshError("degenerate (zero-area) triangle")
    cw = area2 < 0
    EToV[cw, 1], EToV[cw, 2] = EToV[cw, 2].copy(), EToV[cw, 1].copy()
    return EToV, int(cw.sum())


def connectivity(EToV):
    """EToE, EToF: face f of element k (face 1 = v1v2, 2 = v2v3, 3 = v3v1;
    0-based f = 0, 1, 2) is shared with face EToF[k, f] of element EToE[k, f];
    a boundary face points to itself.  Two faces are the same face when they
    join the same pair of vertices."""
    K = EToV.shape[0]
    EToE = np.tile(np.arange(K)[:, None], (1, 3))
    EToF = np.tile(np.arange(3)[None, :], (K, 1))
    owner = {}
    for k in range(K):
        v = EToV[k]
        for f in range(3):
            key = tuple(sorted((int(v[f]), int(v[(f + 1) % 3]))))
            if key in owner:
                k2, f2 = owner[key]
                if k2 < 0:
                    raise MeshError("face shared by more than two elements")
                EToE[k, f], EToF[k, f] = k2, f2
                EToE[k2, f2], EToF[k2, f2] = k, f
                owner[key] = (-1, -1)
            else:
                owner[key] = (k, f)
    return EToE, EToF


class Discretization:
    """Nodal DG discretisation of a triangle mesh at order N (all FP64)."""

    def __init__(self, VX, VY, EToV, N, ref=None, match_chunk=200000):
        self.VX = np.asarray(VX, dtype=np.float64)
        self.VY = np.asarray(VY, dtype=np.float64)
        self.EToV, self.n_flipped = orient_ccw(self.VX, self.VY, EToV)
        self.ref = ref if ref is not None else ReferenceElement(N)
        R = self.ref
        self.N, self.Np, self.Nfp, self.Nafp = R.N, R.Np, R.Nfp, R.Nafp
        K = self.K = self.EToV.shape[0]
        self.EToE, self.EToF = connectivity(self.EToV)

        # affine map of Section "Implementation Aspects":
        # x = (-(r+s) v1 + (1+r) v2 + (1+s) v3) / 2
        va, vb, vc = self.EToV[:, 0], self.EToV[:, 1], self.EToV[:, 2]
        r, s = R.r, R.s
        self.x = 0.5 * (-np.outer(self.VX[va], r + s) + np.outer(self.VX[vb], 1 + r)
                        + np.outer(self.VX[vc], 1 + s))
        self.y = 0.5 * (-np.outer(self.VY[va], r + s) + np.outer(self.VY[vb], 1 + r)
                        + np.outer(self.VY[vc], 1 + s))

        # geometric factors: entries of A_k of the affine map
        # Psi(r, s) = A_k (r, s)^T + b_k and of its inverse (Eq.
        # dg-diff-local-to-global), taken straight from the map's definition
        # (constant on each element)
        ones = np.ones(self.Np)
        xr = np.outer(0.5 * (self.VX[vb] - self.VX[va]), ones)
        xs = np.outer(0.5 * (self.VX[vc] - self.VX[va]), ones)
        yr = np.outer(0.5 * (self.VY[vb] - self.VY[va]), ones)
        ys = np.outer(0.5 * (self.VY[vc] - self.VY[va]), ones)
        J = xr * ys - xs * yr
        if np.any(J <= 0):
            raise MeshError("non-positive Jacobian")
        self.J = J
        self.rx = ys / J
        self.sx = -yr / J
        self.ry = -xs / J
        self.sy = xr / J

        # outward face normals from the map derivatives at the face nodes
        Fm = R.Fmask
        fxr = xr[:, Fm]  # (K, 3, Nfp)
        fxs = xs[:, Fm]
        fyr = yr[:, Fm]
        fys = ys[:, Fm]
        nx = np.empty((K, 3, self.Nfp))
        ny = np.empty((K, 3, self.Nfp))
        nx[:, 0], ny[:, 0] = fyr[:, 0], -fxr[:, 0]
        nx[:, 1], ny[:, 1] = fys[:, 1] - fyr[:, 1], fxr[:, 1] - fxs[:, 1]
        nx[:, 2], ny[:, 2] = -fys[:, 2], fxs[:, 2]
        sJ = np.sqrt(nx * nx + ny * ny)
        self.nx = (nx / sJ).reshape(K, self.Nafp)
        self.ny = (ny / sJ).reshape(K, self.Nafp)
        self.sJ = sJ.reshape(K, self.Nafp)
        self.Fscale = self.sJ / J[:, Fm.reshape(-1)]

        # vmapM / vmapP: global node numbers (k * Np + n) of the interior and
        # exterior traces; exterior nodes found by matching coordinates.
        Np, Nfp = self.Np, self.Nfp
        flat_fm = Fm.reshape(-1)
        self.vmapM = (np.arange(K)[:, None] * Np + flat_fm[None, :])  # (K, Nafp)
        vmapP = self.vmapM.copy()
        xf = self.x.reshape(-1)
        yf = self.y.reshape(-1)
        h = np.sqrt(J[:, 0])  # element length scale
        for k0 in range(0, K, match_chunk):
            k1 = min(K, k0 + match_chunk)
            kk = np.arange(k0, k1)
            for f in range(3):
                kP = self.EToE[kk, f]
                fP = self.EToF[kk, f]
                interior = kP != kk
                if not np.any(interior):
                    continue
                ki = kk[interior]
                kPi = kP[interior]
                fPi = fP[interior]
                idM = ki[:, None] * Np + Fm[f][None, :]            # (n, Nfp)
                idP = kPi[:, None] * Np + Fm[fPi]                   # (n, Nfp)
                d2 = ((xf[idM][:, :, None] - xf[idP][:, None, :]) ** 2
                      + (yf[idM][:, :, None] - yf[idP][:, None, :]) ** 2)
                jbest = np.argmin(d2, axis=2)
                dmin = np.sqrt(np.take_along_axis(d2, jbest[:, :, None], axis=2)[:, :, 0])
                if np.any(dmin > 1e-8 * h[ki][:, None] + 1e-14):
                    raise MeshError("face nodes of neighbouring elements do not match")
                vmapP[ki, f * Nfp:(f + 1) * Nfp] = np.take_along_axis(idP, jbest, axis=1)
        self.vmapP = vmapP
        self.mapB = np.nonzero((vmapP == self.vmapM).reshape(-1))[0]
        self.vmapB = self.vmapM.reshape(-1)[self.mapB]

    # ------------------------------------------------------------------
    def nodes(self):
        return self.x, self.y


# ---------------------------------------------------------------------------
# Semi-discrete right-hand side (Eq. dg-strong-explicit with Eq. max2d-numflux)
# ---------------------------------------------------------------------------


def maxwell_rhs(d, q, alpha=1.0, flux=True):
    """Right-hand side (dHx/dt, dHy/dt, dEz/dt) of the semi-discrete TM system.

    Volume part: grad Ez and curl H through the chain rule
    d/dx = rx Dr + sx Ds, d/dy = ry Dr + sy Ds (Eq. dg-diff-local-to-global);
    dHx/dt = -dEz/dy, dHy/dt = dEz/dx, dEz/dt = dHy/dx - dHx/dy
    (Eq. tm-maxwells; the code's reading of the printed typo).

    Surface part: jumps [q] = q- - q+ at every face node; at PEC faces
    [Hx] = [Hy] = 0 and [Ez] = 2 Ez-; upwind flux n.(F - F*) of
    Eq. max2d-numflux (with the H-entries read as
    alpha (n (n.[H]) - [H]), the energy-stable form); then
    rhs += LIFT (Fscale * flux) / 2 (Eq. dg-lift / dg-strong-explicit).
    ``flux=False`` drops the surface part (volume-only debug switch).
    """
    R = d.ref
    Hx, Hy, Ez = q[0], q[1], q[2]
    # local derivatives along the reference axes
    def ddx(u):
        return d.rx * (u @ R.Dr.T) + d.sx * (u @ R.Ds.T)

    def ddy(u):
        return d.ry * (u @ R.Dr.T) + d.sy * (u @ R.Ds.T)

    rhsHx = -ddy(Ez)
    rhsHy = ddx(Ez)
    rhsEz = ddx(Hy) - ddy(Hx)
    if not flux:
        return np.stack([rhsHx, rhsHy, rhsEz])

    vM = d.vmapM.reshape(-1)
    vP = d.vmapP.reshape(-1)
    dHx = Hx.reshape(-1)[vM] - Hx.reshape(-1)[vP]
    dHy = Hy.reshape(-1)[vM] - Hy.reshape(-1)[vP]
    dEz = Ez.reshape(-1)[vM] - Ez.reshape(-1)[vP]
    # PEC: Ez+ = -Ez-, H+ = H-
    dHx[d.mapB] = 0.0
    dHy[d.mapB] = 0.0
    dEz[d.mapB] = 2.0 * Ez.reshape(-1)[d.vmapB]
    shape = (d.K, d.Nafp)
    dHx, dHy, dEz = dHx.reshape(shape), dHy.reshape(shape), dEz.reshape(shape)
    nx, ny = d.nx, d.ny
    ndotdH = nx * dHx + ny * dHy
    fHx = ny * dEz + alpha * (ndotdH * nx - dHx)
    fHy = -nx * dEz + alpha * (ndotdH * ny - dHy)
    fEz = ny * dHx - nx * dHy - alpha * dEz
    rhsHx = rhsHx + (d.Fscale * fHx) @ R.LIFT.T / 2.0
    rhsHy = rhsHy + (d.Fscale * fHy) @ R.LIFT.T / 2.0
    rhsEz = rhsEz + (d.Fscale * fEz) @ R.LIFT.T / 2.0
    return np.stack([rhsHx, rhsHy, rhsEz])


def maxwell_rhs_media(d, q, eps):
    """Right-hand side with a piecewise-constant permittivity eps[k] per
    element (mu = 1), the variable-coefficient form of Eq. tm-maxwells:
    dHx/dt = -dEz/dy, dHy/dt = dEz/dx, eps dEz/dt = dHy/dx - dHx/dy.

    Upwind flux from the exact Riemann solution along the face normal.
    With Ht = ny Hx - nx Hy the normal system is dHt/dt + dEz/dxi = 0,
    eps dEz/dt + dHt/dxi = 0, impedance Z = 1/sqrt(eps); the interface
    state follows from the outgoing characteristic of each side, and with
    jumps [u] = u- - u+ the flux differences n.(F- - F*) are
        Ez:        (Z+ [Ht] - [Ez]) / (Z- + Z+)
        (Hx, Hy):  (ny, -nx) Z- ([Ez] - Z+ [Ht]) / (Z- + Z+)
    (the normal H component has no flux).  PEC faces: Ez+ = -Ez-, H+ = H-,
    Z+ = Z-.  Then rhs = vol + LIFT (Fscale * n.(F - F*)), and the Ez row
    is divided by eps[k].  With eps = 1 this is maxwell_rhs with alpha = 1
    (there the flux carries the factor 1/2 as (Z- + Z+) = 2).
    """
    R = d.ref
    eps = np.asarray(eps, dtype=np.float64).reshape(d.K)
    Z = 1.0 / np.sqrt(eps)
    vol = maxwell_rhs(d, q, flux=False)
    Hx, Hy, Ez = q[0], q[1], q[2]
    vM = d.vmapM.reshape(-1)
    vP = d.vmapP.reshape(-1)
    jHx = Hx.reshape(-1)[vM] - Hx.reshape(-1)[vP]
    jHy = Hy.reshape(-1)[vM] - Hy.reshape(-1)[vP]
    jEz = Ez.reshape(-1)[vM] - Ez.reshape(-1)[vP]
    ZM = np.repeat(Z, d.Nafp)                # interior side of every face node
    ZP = Z[vP // d.Np]                       # the neighbour's element
    jHx[d.mapB] = 0.0
    jHy[d.mapB] = 0.0
    jEz[d.mapB] = 2.0 * Ez.reshape(-1)[d.vmapB]
    ZP[d.mapB] = ZM[d.mapB]
    nx, ny = d.nx.reshape(-1), d.ny.reshape(-1)
    jHt = ny * jHx - nx * jHy
    fEz = (ZP * jHt - jEz) / (ZM + ZP)
    g = ZM * (jEz - ZP * jHt) / (ZM + ZP)
    shape = (d.K, d.Nafp)
    Fs = d.Fscale
    rhsHx = vol[0] + (Fs * (ny * g).reshape(shape)) @ R.LIFT.T
    rhsHy = vol[1] + (Fs * (-nx * g).reshape(shape)) @ R.LIFT.T
    rhsEz = (vol[2] + (Fs * fEz.reshape(shape)) @ R.LIFT.T) / eps[:, None]
    return np.stack([rhsHx, rhsHy, rhsEz])


def ricker(t, f=10.0, t0=None, amplitude=1.0):
    """Ricker wavelet s(t) = A (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2),
    tau = t - t0, peak frequency f; t0 defaults to 1.2 / f (reading: the
    source term f of the problem statement is unspecified there)."""
    if t0 is None:
        t0 = 1.2 / f
    a = (math.pi * f * (np.asarray(t, dtype=np.float64) - t0)) ** 2
    return amplitude * (1.0 - 2.0 * a) * np.exp(-a)


def locate_point(d, xs, ys):
    """Element k that contains (xs, ys) (barycentric coordinates of its three
    vertices all >= -1e-12; the lowest such k) and the point's reference
    coordinates (r, s) under that element's affine map
    x = (-(r+s) v1 + (1+r) v2 + (1+s) v3) / 2."""
    x = d.VX[d.EToV]
    y = d.VY[d.EToV]
    det = (x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0])
    l2 = ((xs - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (ys - y[:, 0])) / det
    l3 = ((x[:, 1] - x[:, 0]) * (ys - y[:, 0]) - (xs - x[:, 0]) * (y[:, 1] - y[:, 0])) / det
    l1 = 1.0 - l2 - l3
    inside = np.nonzero((l1 >= -1e-12) & (l2 >= -1e-12) & (l3 >= -1e-12))[0]
    if inside.size == 0:
        raise ValueError("point outside the mesh")
    k = int(inside[0])
    return k, 2.0 * l2[k] - 1.0, 2.0 * l3[k] - 1.0


def point_source_weights(d, xs, ys):
    """Projection of the point load delta(x - x_s) onto the nodal basis of
    the element k that contains x_s: the field w on element k with
    integral_k w v = v(x_s) for every polynomial v of degree <= N, i.e.
    w = M^-1 l(x_s) / J_k, where l(x_s) holds the Lagrange basis functions of
    the element's nodes at x_s (l = V^-T psi(r_s, s_s), psi the orthonormal
    basis) and M^-1 = V V^T.  Returns (k, w[Np])."""
    k, r, s = locate_point(d, xs, ys)
    R = d.ref
    psi = vandermonde_2d(R.N, np.array([r]), np.array([s]))[0]
    lag = np.linalg.solve(R.V.T, psi)
    w = R.V @ (R.V.T @ lag) / d.J[k, 0]
    return k, w


def point_source_rhs(d, k, w, amplitude):
    """Right-hand-side contribution amplitude * w on the Ez field of element
    k (reading: the source adds to dEz/dt directly, after any division by
    eps)."""
    out = np.zeros((3, d.K, d.Np))
    out[2, k] = amplitude * np.asarray(w)
    return out


def energy_media(d, q, eps):
    """1/2 sum_k J_k (Hx^T M Hx + Hy^T M Hy + eps_k Ez^T M Ez)."""
    M = d.ref.M
    Jk = d.J[:, 0]
    w = [Jk, Jk, Jk * np.asarray(eps, dtype=np.float64).reshape(d.K)]
    return 0.5 * sum(np.sum(w[f] * np.einsum("kn,nm,km->k", q[f], M, q[f])) for f in range(3))


# ---------------------------------------------------------------------------
# LSRK(5,4): Carpenter & Kennedy (1994), five-stage fourth-order, 2N storage
# ---------------------------------------------------------------------------

LSRK_A = np.array([
    0.0,
    -567301805773.0 / 1357537059087.0,
    -2404267990393.0 / 2016746695238.0,
    -3550918686646.0 / 2091501179385.0,
    -1275806237668.0 / 842570457699.0,
])
LSRK_B = np.array([
    1432997174477.0 / 9575080441755.0,
    5161836677717.0 / 13612068292357.0,
    1720146321549.0 / 2090206949498.0,
    3134564353537.0 / 4481467310338.0,
    2277821191437.0 / 14882151754819.0,
])
#: Stage times.  Reading: c_i = sum_j A_ij of the Butcher form of (LSRK_A,
#: LSRK_B) (see ``butcher_form``); the commonly printed fraction for c_4,
#: 2006345519317/3224776611391, is 9.0e-5 below that sum, the others agree.
LSRK_C_PUBLISHED = np.array([
    0.0,
    1432997174477.0 / 9575080441755.0,
    2526269341429.0 / 6820363962896.0,
    2006345519317.0 / 3224776611391.0,
    2802321613138.0 / 2924317926251.0,
])


def butcher_form(a=None, b=None):
    """Butcher matrix and weights of a 2N-storage scheme
    (K_i = a_i K_{i-1} + dt f(u_{i-1}), u_i = u_{i-1} + b_i K_i):
    the weight of f_j in u_i is sum_{m=j..i-1} b_m prod_{l=j+1..m} a_l."""
    a = LSRK_A if a is None else np.asarray(a, dtype=np.float64)
    b = LSRK_B if b is None else np.asarray(b, dtype=np.float64)
    s = len(a)
    W = np.zeros((s + 1, s))
    for i in range(1, s + 1):
        for j in range(i):
            tot = 0.0
            for m in range(j, i):
                prod = 1.0
                for l in range(j + 1, m + 1):
                    prod *= a[l]
                tot += b[m] * prod
            W[i, j] = tot
    return W[:s], W[s]


LSRK_C = butcher_form()[0].sum(axis=1)


def lsrk_step(d, q, t, dt, rhs=None):
    """One LSRK(5,4) step: for each stage i,
    res <- a_i res + dt rhs(q, t + c_i dt);  q <- q + b_i res.
    Returns the new q (res starts at zero and a_1 = 0)."""
    f = rhs if rhs is not None else (lambda u, tt: maxwell_rhs(d, u))
    q = np.array(q, dtype=np.float64, copy=True)
    res = np.zeros_like(q)
    for i in range(5):
        res = LSRK_A[i] * res + dt * f(q, t + LSRK_C[i] * dt)
        q = q + LSRK_B[i] * res
    return q


def lsrk_stage(d, q, res, i, t, dt):
    """Stage i (0-based) of an LSRK(5,4) step; returns (q_new, res_new)."""
    res_new = LSRK_A[i] * res + dt * maxwell_rhs(d, q)
    return q + LSRK_B[i] * res_new, res_new


def solve(d, q, T, dt, nsteps=None):
    """Advance q from t = 0 by LSRK(5,4) steps of size dt (nsteps of them, or
    ceil(T/dt) with dt shrunk to land on T exactly)."""
    if nsteps is None:
        nsteps = int(math.ceil(T / dt - 1e-12))
        dt = T / nsteps
    t = 0.0
    for _ in range(nsteps):
        q = lsrk_step(d, q, t, dt)
        t += dt
    return q, t


# ---------------------------------------------------------------------------
# Diagnostics
# ---------------------------------------------------------------------------


def energy(d, q):
    """Discrete energy 1/2 sum_k J_k (Hx^T M Hx + Hy^T M Hy + Ez^T M Ez)."""
    M = d.ref.M
    Jk = d.J[:, 0]
    e = 0.0
    for f in range(3):
        u = q[f]
        e += np.sum(Jk * np.einsum("kn,nm,km->k", u, M, u))
    return 0.5 * e


def energy_rate(d, q, rhs):
    """d/dt of the discrete energy along the semi-discrete flow:
    sum_k J_k sum_f u_f^T M rhs_f."""
    M = d.ref.M
    Jk = d.J[:, 0]
    return float(sum(np.sum(Jk * np.einsum("kn,nm,km->k", q[f], M, rhs[f])) for f in range(3)))


def cfl_dt(d, cfl=1.0):
    """Time step reading: dt = cfl * (2/3) * min_k(inradius_k) * (LGL_1 - LGL_0)."""
    x = d.VX[d.EToV]
    y = d.VY[d.EToV]
    la = np.hypot(x[:, 1] - x[:, 0], y[:, 1] - y[:, 0])
    lb = np.hypot(x[:, 2] - x[:, 1], y[:, 2] - y[:, 1])
    lc = np.hypot(x[:, 0] - x[:, 2], y[:, 0] - y[:, 2])
    area = 0.5 * np.abs((x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0])
                        - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0]))
    inradius = area / (0.5 * (la + lb + lc))
    g = lgl_nodes(d.N)
    return cfl * (2.0 / 3.0) * inradius.min() * (g[1] - g[0])


def rhs_flops(K, N):
    """FLOPs of one right-hand-side evaluation by the chapter's count
    (Section "Computing the Surface Contribution", rhs_flops):
    6 reference-axis products of 2 Np^2, chain rule 2 Np 13, three LIFT
    products of 2 Np Nafp + Np, and 18 flux FLOPs per face node."""
    Np = (N + 1) * (N + 2) // 2
    Nafp = 3 * (N + 1)
    return K * (6 * 2 * Np * Np + 2 * Np * 13 + 3 * (2 * Np * Nafp + Np) + Nafp * 18)
