"""Pins for the oracle's mesh handling: orientation, connectivity (against
brute force), geometric factors, normals, Fscale and the trace maps."""
import numpy as np
import pytest

import oracle as O
from synth import jittered_delaunay_mesh, square_grid_mesh


def _brute_connectivity(EToV):
    K = EToV.shape[0]
    EToE = np.tile(np.arange(K)[:, None], (1, 3))
    EToF = np.tile(np.arange(3)[None, :], (K, 1))
    for k in range(K):
        for f in range(3):
            a, b = EToV[k, f], EToV[k, (f + 1) % 3]
            for k2 in range(K):
                if k2 == k:
                    continue
                for f2 in range(3):
                    c, d = EToV[k2, f2], EToV[k2, (f2 + 1) % 3]
                    if {a, b} == {c, d}:
                        EToE[k, f], EToF[k, f] = k2, f2
    return EToE, EToF


def test_connectivity_matches_brute_force():
    VX, VY, EToV = jittered_delaunay_mesh(5, seed=3)
    EToE, EToF = O.connectivity(EToV)
    bE, bF = _brute_connectivity(EToV)
    assert np.array_equal(EToE, bE) and np.array_equal(EToF, bF)


def test_orientation_fix_and_errors():
    VX, VY, EToV = square_grid_mesh(2, 2)
    bad = EToV.copy()
    bad[[0, 3]] = bad[[0, 3]][:, [0, 2, 1]]
    fixed, nflip = O.orient_ccw(VX, VY, bad)
    assert nflip == 2
    assert np.array_equal(fixed, EToV)
    with pytest.raises(O.MeshError):
        O.orient_ccw(np.array([0.0, 1.0, 2.0]), np.zeros(3), np.array([[0, 1, 2]]))
    # a face shared by three elements
    VX2 = np.array([0.0, 1.0, 0.5, 0.5, 0.5])
    VY2 = np.array([0.0, 0.0, 1.0, -1.0, 2.0])
    with pytest.raises(O.MeshError):
        O.connectivity(np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]]))


@pytest.mark.parametrize("N", [1, 3, 5])
def test_geometry_pins(N):
    VX, VY, EToV = jittered_delaunay_mesh(6, seed=11)
    d = O.Discretization(VX, VY, EToV, N)
    x = VX[d.EToV]
    y = VY[d.EToV]
    area = 0.5 * ((x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0]))
    # J = area / 2 (reference triangle has area 2), constant per element
    assert np.allclose(d.J, (area / 2)[:, None], rtol=1e-12)
    # 2 sJ = edge length; |n| = 1; outward
    for f in range(3):
        a, b = f, (f + 1) % 3
        L = np.hypot(x[:, b] - x[:, a], y[:, b] - y[:, a])
        sl = slice(f * d.Nfp, (f + 1) * d.Nfp)
        assert np.allclose(2 * d.sJ[:, sl], L[:, None], rtol=1e-12)
        mx = 0.5 * (x[:, a] + x[:, b]) - x.mean(axis=1)
        my = 0.5 * (y[:, a] + y[:, b]) - y.mean(axis=1)
        assert np.all(d.nx[:, sl] * mx[:, None] + d.ny[:, sl] * my[:, None] > 0)
    assert np.allclose(np.hypot(d.nx, d.ny), 1.0, atol=1e-14)
    assert np.allclose(d.Fscale, d.sJ / (area / 2)[:, None], rtol=1e-12)
    # the chain-rule factors invert the map: [rx ry; sx sy] [xr xs; yr ys] = I
    xr = (x[:, 1] - x[:, 0]) / 2
    xs = (x[:, 2] - x[:, 0]) / 2
    yr = (y[:, 1] - y[:, 0]) / 2
    ys = (y[:, 2] - y[:, 0]) / 2
    assert np.allclose(d.rx[:, 0] * xr + d.ry[:, 0] * yr, 1, atol=1e-11)
    assert np.allclose(d.rx[:, 0] * xs + d.ry[:, 0] * ys, 0, atol=1e-11)
    assert np.allclose(d.sx[:, 0] * xr + d.sy[:, 0] * yr, 0, atol=1e-11)
    assert np.allclose(d.sx[:, 0] * xs + d.sy[:, 0] * ys, 1, atol=1e-11)


@pytest.mark.parametrize("N", [2, 4])
def test_trace_maps(N):
    VX, VY, EToV = jittered_delaunay_mesh(5, seed=2)
    d = O.Discretization(VX, VY, EToV, N)
    vM = d.vmapM.reshape(-1)
    vP = d.vmapP.reshape(-1)
    xf, yf = d.x.reshape(-1), d.y.reshape(-1)
    assert np.allclose(xf[vM], xf[vP], atol=1e-13) and np.allclose(yf[vM], yf[vP], atol=1e-13)
    interior = vP != vM
    # exterior of the exterior is the interior: build node -> face-node position
    pos = {}
    for i, g in enumerate(vM):
        pos.setdefault(g, []).append(i)
    for i in np.nonzero(interior)[0]:
        assert vM[i] in [vP[j] for j in pos[vP[i]]]
    # normals flip across interior faces
    nx = d.nx.reshape(-1)
    ny = d.ny.reshape(-1)
    owner = {}
    for i in np.nonzero(interior)[0]:
        owner[(vM[i], vP[i])] = i
    for (a, b), i in owner.items():
        j = owner[(b, a)]
        assert abs(nx[i] + nx[j]) < 1e-12 and abs(ny[i] + ny[j]) < 1e-12
    # boundary nodes: 4n boundary faces on the unit-square jittered mesh
    assert d.mapB.size == 4 * 5 * d.Nfp
    bx, by = xf[d.vmapB], yf[d.vmapB]
    assert np.all(np.minimum.reduce([np.abs(bx), np.abs(bx - 1), np.abs(by), np.abs(by - 1)]) < 1e-14)
