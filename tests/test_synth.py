"""The seeded input generators: deterministic, valid meshes of the stated size."""
import numpy as np

from synth import jittered_delaunay_mesh, relabel_mesh, square_grid_mesh


def _area2(VX, VY, EToV):
    x = VX[EToV]
    y = VY[EToV]
    return (x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0])


def test_jittered_mesh_size_orientation_and_determinism():
    for n in (3, 10, 41):
        VX, VY, EToV = jittered_delaunay_mesh(n, seed=7)
        assert EToV.shape == (2 * n * n, 3) and EToV.dtype == np.int32
        assert np.all(_area2(VX, VY, EToV) > 0)
        assert abs(_area2(VX, VY, EToV).sum() / 2 - 1.0) < 1e-12
        VX2, VY2, E2 = jittered_delaunay_mesh(n, seed=7)
        assert np.array_equal(E2, EToV) and np.array_equal(VX2, VX)
    VX3, _, _ = jittered_delaunay_mesh(10, seed=8)
    assert not np.array_equal(VX3, jittered_delaunay_mesh(10, seed=7)[0])


def test_square_grid_mesh():
    VX, VY, EToV = square_grid_mesh(8, 8)
    assert EToV.shape == (128, 3)
    assert np.all(_area2(VX, VY, EToV) > 0)
    assert abs(_area2(VX, VY, EToV).sum() / 2 - 4.0) < 1e-12


def test_relabel_keeps_orientation():
    VX, VY, EToV = jittered_delaunay_mesh(6, seed=1)
    E2, perm, rot = relabel_mesh(EToV, seed=3)
    assert np.all(_area2(VX, VY, E2) > 0)
    assert sorted(map(tuple, np.sort(E2, axis=1))) == sorted(map(tuple, np.sort(EToV, axis=1)))
