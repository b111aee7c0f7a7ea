"""GPU: face pairs (dg_operator_set_face_pairs) on the tensor-core stage
kernel.  A face whose two elements lie in the same element block is done
once, by one task, for both sides (Section "Further Tuning Opportunities":
otherwise each side fetches the pair separately).  With face pairs on, every
face node's flux is computed by the same explicitly rounded operations,
whether its element's task or its neighbour's does it, so an element's
result must not depend on whether its neighbour shares its block:

* a mesh split into parts (dg_partition_*: other blocks, faces across the
  cuts computed per side) gives, with face pairs on, the unpartitioned
  result bit for bit;
* the results with face pairs on and off agree within the FP32 tolerance
  (1e-5 of max |value|; they round differently: the default kernel lets the
  compiler contract multiply-adds);
* the flag is ignored by the other product variants and is checked.

Oracle parity with face pairs on, at sizes where every CTA walks many
blocks, is in test_parity_large_gpu.py.
"""
import numpy as np
import pytest

from synth import gaussian_pulse, jittered_delaunay_mesh, random_fields, random_permittivity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1304_5546_gb300 import build as B
    B.build()
    import paper_1304_5546_gb300 as P
    return P


@pytest.fixture(scope="module")
def mesh():
    # K = 28,800: several 40/80-element blocks per CTA
    return jittered_delaunay_mesh(120, seed=31)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _run(P, s, q0, pairs):
    P.dg_operator_set_face_pairs(s.op, pairs)
    q = s.from_numpy(q0)
    rhs = s.to_numpy(s.rhs(q))
    res = s.new_fields()
    s.step(q, res, s.cfl_dt(), nsteps=2)
    P.dg_sync_check(s.op)
    return rhs, s.to_numpy(q)


@pytest.mark.parametrize("N", list(range(1, 8)))
def test_pairs_match_per_side_flux(P, mesh, N):
    s = P.Solver(*mesh, N=N, precision="fp32tc")
    q0 = random_fields(s.K, s.Np, seed=N)
    off, on = _run(P, s, q0, 0), _run(P, s, q0, 1)
    for a, b in zip(on, off):
        assert _rel(a, b) <= 1e-5, _rel(a, b)
    s.close()


@pytest.mark.parametrize("N,parts,media", [(2, 3, False), (5, 2, False), (7, 4, False),
                                           (3, 2, True), (6, 3, True)])
def test_pairs_result_independent_of_blocks(P, N, parts, media):
    import torch
    VX, VY, EToV = jittered_delaunay_mesh(60, seed=40 + N)
    eps = random_permittivity(EToV.shape[0], seed=N) if media else None
    s = P.Solver(VX, VY, EToV, N=N, precision="fp32tc" if not media else "fp32", eps=eps)
    P.dg_operator_set_face_pairs(s.op, 1)
    x, y = s.nodes()
    q0 = s.from_numpy(np.stack(gaussian_pulse(x, y, 0.4, 0.6, 0.15))
                      + 0.1 * random_fields(s.K, s.Np, seed=N))
    dt = 0.9 * s.cfl_dt()
    q, res = q0.clone(), s.new_fields()
    s.step(q, res, dt, 2)
    part = P.Partition(s, parts)
    part.set_fields(q0)
    part.step(dt, 2)
    out = s.new_fields()
    part.get_fields(out)
    part.sync_check()
    P.dg_sync_check(s.op)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(s.to_numpy(out), s.to_numpy(q))
    part.close()
    s.close()


def test_pairs_ignored_by_other_variants(P, mesh):
    s = P.Solver(*mesh, N=4, precision="bf16x3")
    q0 = random_fields(s.K, s.Np, seed=9)
    off, on = _run(P, s, q0, 0), _run(P, s, q0, 1)
    for a, b in zip(off, on):
        np.testing.assert_array_equal(a, b)
    s.close()


def test_pairs_flag_checked(P):
    s = P.Solver(*jittered_delaunay_mesh(4, seed=1), N=3, precision="fp32")
    with pytest.raises(P.DGError) as ex:
        P._lib.check(P._lib.load().dg_operator_set_face_pairs(s.op, 2), "set")
    assert ex.value.status == P._lib.DG_ERR_ARG
    s.close()
