"""Host-side checks of checkpoints (dg_checkpoint_save / _load with host
fields): a round trip restores fields, time and step exactly; a file written
for another operator or mesh, a damaged file and a missing file are
refused."""
import numpy as np
import pytest

from synth import jittered_delaunay_mesh, random_fields


@pytest.fixture(scope="module")
def dgw():
    from paper_1304_5546_gb300 import build as B
    B.build()
    import paper_1304_5546_gb300 as P
    return P


def _op(dgw, n, seed, N, prec):
    VX, VY, EToV = jittered_delaunay_mesh(n, seed=seed)
    mesh = dgw.dg_mesh_create(VX, VY, EToV)
    op = dgw.dg_operator_setup(mesh, N, prec, dgw.DG_SETUP_HOST_ONLY)
    Np, _, K, _ = dgw.dg_get_info(op)
    return mesh, op, K, Np


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_round_trip(dgw, tmp_path, prec):
    p = dgw.DG_FP64 if prec == "fp64" else dgw.DG_FP32
    dtype = np.float64 if prec == "fp64" else np.float32
    mesh, op, K, Np = _op(dgw, 5, 3, 4, p)
    q = np.ascontiguousarray(random_fields(K, Np, seed=1).astype(dtype))
    path = tmp_path / "state.ckpt"
    dgw.dg_checkpoint_save(op, q, K * Np, 0.375, 12, path)
    back = np.zeros_like(q)
    t, step = dgw.dg_checkpoint_load(op, path, back, K * Np)
    assert (t, step) == (0.375, 12)
    assert np.array_equal(back, q)
    # a wider stride (a padded field buffer): only K * Np values per field move
    wide = np.full((3, K * Np + 7), -1.0, dtype)
    dgw.dg_checkpoint_load(op, path, wide, K * Np + 7)
    assert np.array_equal(wide[:, : K * Np].reshape(q.shape), q)
    assert np.all(wide[:, K * Np:] == -1.0)
    dgw.dg_op_destroy(op)
    dgw.dg_mesh_destroy(mesh)


def test_refuses_other_operator_mesh_and_damage(dgw, tmp_path):
    from paper_1304_5546_gb300 import DGError
    mesh, op, K, Np = _op(dgw, 5, 3, 4, dgw.DG_FP64)
    q = np.ascontiguousarray(random_fields(K, Np, seed=2))
    path = tmp_path / "a.ckpt"
    dgw.dg_checkpoint_save(op, q, K * Np, 1.0, 3, path)
    others = [_op(dgw, 5, 3, 3, dgw.DG_FP64),   # another order
              _op(dgw, 5, 4, 4, dgw.DG_FP64),   # another mesh, same K
              _op(dgw, 5, 3, 4, dgw.DG_FP32)]   # another precision
    for m2, op2, K2, Np2 in others:
        buf = np.zeros((3, K2 * Np2), np.float64)
        with pytest.raises(DGError):
            dgw.dg_checkpoint_load(op2, path, buf, K2 * Np2)
        dgw.dg_op_destroy(op2)
        dgw.dg_mesh_destroy(m2)
    raw = bytearray(path.read_bytes())
    raw[-5] ^= 0x40  # one flipped bit in the field data
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(bytes(raw))
    with pytest.raises(DGError):
        dgw.dg_checkpoint_load(op, bad, np.zeros_like(q), K * Np)
    with pytest.raises(DGError):
        dgw.dg_checkpoint_load(op, tmp_path / "missing.ckpt", np.zeros_like(q), K * Np)
    dgw.dg_op_destroy(op)
    dgw.dg_mesh_destroy(mesh)
