"""Seeded triangle meshes of the kind the chapter's solver runs on: straight
sided, face-conforming triangles covering a polygonal domain (Section
"Construction of the Method").

Every generator returns ``(VX, VY, EToV)``: float64 vertex coordinates of
shape ``(Nv,)`` and an int32 element-to-vertex table of shape ``(K, 3)``,
0-based, with every triangle listed counter-clockwise.
"""
import numpy as np


def _ccw(VX, VY, EToV):
    """Return EToV with clockwise triangles re-listed counter-clockwise by
    swapping their 2nd and 3rd vertices."""
    EToV = np.array(EToV, dtype=np.int64, copy=True)
    x = VX[EToV]
    y = VY[EToV]
    area2 = (x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0])
    cw = area2 < 0
    EToV[cw, 1], EToV[cw, 2] = EToV[cw, 2].copy(), EToV[cw, 1].copy()
    return EToV


def square_grid_mesh(nx, ny, xmin=-1.0, xmax=1.0, ymin=-1.0, ymax=1.0):
    """Structured grid of ``nx * ny`` squares, each split into two triangles by
    its lower-left to upper-right diagonal (``K = 2 nx ny``).

    Elements are listed square by square, row-major from the bottom row; the
    lower-right triangle of a square comes before its upper-left one.
    """
    xs = np.linspace(xmin, xmax, nx + 1)
    ys = np.linspace(ymin, ymax, ny + 1)
    VX = np.tile(xs, ny + 1)
    VY = np.repeat(ys, nx + 1)
    EToV = np.empty((2 * nx * ny, 3), dtype=np.int32)
    e = 0
    for j in range(ny):
        for i in range(nx):
            v00 = j * (nx + 1) + i
            v10 = v00 + 1
            v01 = v00 + (nx + 1)
            v11 = v01 + 1
            EToV[e] = (v00, v10, v11)
            EToV[e + 1] = (v00, v11, v01)
            e += 2
    return VX, VY, EToV


def n_for_target_elements(k_target):
    """Grid resolution ``n`` whose jittered Delaunay mesh has ``2 n^2`` ~ k_target triangles."""
    return max(1, int(round(np.sqrt(k_target / 2.0))))


def jittered_delaunay_mesh(n, seed, jitter=0.3):
    """Seeded jittered-grid Delaunay triangulation of the unit square.

    Vertices start on an ``(n+1) x (n+1)`` grid of spacing ``h = 1/n``.
    Interior vertices move by independent ``U(-jitter h, +jitter h)`` offsets
    in x and y; boundary vertices move only along their side; the four corners
    stay fixed.  The Delaunay triangulation (scipy's Qhull) of these points has
    exactly ``2 n^2`` triangles (Euler's formula with all ``4n`` boundary points
    on the hull), which is checked.

    Triangles are re-listed counter-clockwise and sorted by (row band of their
    centroid, centroid x) so that face neighbours sit close in element index.
    """
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)
    h = 1.0 / n
    g = np.linspace(0.0, 1.0, n + 1)
    X, Y = np.meshgrid(g, g)  # X[j, i] = g[i], Y[j, i] = g[j]
    dx = rng.uniform(-jitter * h, jitter * h, size=X.shape)
    dy = rng.uniform(-jitter * h, jitter * h, size=Y.shape)
    bottom_top = np.zeros(X.shape, dtype=bool)
    bottom_top[0, :] = True
    bottom_top[-1, :] = True
    left_right = np.zeros(X.shape, dtype=bool)
    left_right[:, 0] = True
    left_right[:, -1] = True
    # y-sides (left/right) may slide in y only; bottom/top may slide in x only.
    dx[left_right] = 0.0
    dy[bottom_top] = 0.0
    X = X + dx
    Y = Y + dy
    VX = X.ravel()
    VY = Y.ravel()
    tri = Delaunay(np.column_stack([VX, VY]))
    if len(tri.coplanar):
        raise RuntimeError("Delaunay dropped %d points" % len(tri.coplanar))
    EToV = _ccw(VX, VY, tri.simplices)
    K = EToV.shape[0]
    if K != 2 * n * n:
        raise RuntimeError("expected %d triangles, got %d" % (2 * n * n, K))
    cx = VX[EToV].mean(axis=1)
    cy = VY[EToV].mean(axis=1)
    band = np.floor(cy / h).astype(np.int64)
    order = np.lexsort((cx, band))
    EToV = EToV[order].astype(np.int32)
    x = VX[EToV]
    y = VY[EToV]
    area2 = (x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0])
    if not np.all(area2 > 0):
        raise RuntimeError("degenerate triangle in jittered mesh")
    return VX, VY, EToV


def relabel_mesh(EToV, seed):
    """Randomly permute the elements and cyclically rotate each element's
    vertex list (orientation is kept).

    Returns ``(EToV2, perm, rot)`` with ``EToV2[i] = roll(EToV[perm[i]], -rot[i])``.
    """
    rng = np.random.default_rng(seed)
    K = EToV.shape[0]
    perm = rng.permutation(K)
    rot = rng.integers(0, 3, size=K)
    E = np.asarray(EToV)[perm]
    idx = (np.arange(3)[None, :] + rot[:, None]) % 3
    EToV2 = np.take_along_axis(E, idx, axis=1).astype(np.int32)
    return EToV2, perm, rot
