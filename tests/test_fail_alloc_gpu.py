"""Allocation failures made on the host (dg_test_fail_alloc): the n-th device
allocation of the library fails with DG_ERR_OOM without allocating.  For
every n up to the number of allocations a set-up call makes, the call must
report DG_ERR_OOM, give back everything it had allocated (device memory
returns to its level before the call), and leave the library usable; one
more than that and the call succeeds untouched."""
import numpy as np
import pytest

from synth import gaussian_pulse, jittered_delaunay_mesh, random_permittivity

pytestmark = pytest.mark.gpu

SLACK = 16 << 20  # bytes: driver allocation granularity


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1304_5546_gb300 import build as B
    B.build()
    import paper_1304_5546_gb300 as P
    return P


def _free():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _sweep(P, make, destroy, max_n=64):
    """Plant a failure at allocation n = 1, 2, ... until `make` succeeds;
    returns the number of allocations it makes."""
    from paper_1304_5546_gb300 import _lib
    destroy(make())  # warm: lazily loaded code and pools are in place before the baseline
    base = _free()
    for n in range(1, max_n):
        P.dg_test_fail_alloc(n)
        try:
            obj = make()
        except P.DGError as e:
            assert e.status == _lib.DG_ERR_OOM, (n, e)
            assert P.dg_test_fail_alloc_pending() == 0
            assert abs(_free() - base) <= SLACK, (n, base - _free())
            continue
        finally:
            pending = P.dg_test_fail_alloc_pending()
            P.dg_test_fail_alloc(0)
        assert pending > 0  # the planted failure was never reached
        destroy(obj)
        assert abs(_free() - base) <= SLACK
        return n - 1
    raise AssertionError("set-up never succeeded")


def test_operator_setup(P):
    VX, VY, EToV = jittered_delaunay_mesh(30, seed=1)
    mesh = P.dg_mesh_create(VX, VY, EToV)
    try:
        for prec, flags in ((P.DG_FP32, 0), (P.DG_FP64, 0), (P.DG_FP32, 2)):  # 2: CUDA cores
            n = _sweep(P, lambda: P.dg_operator_setup(mesh, 5, prec, flags), P.dg_op_destroy)
            assert n >= 8
        # N = 2: the element-thread kernel's operator (default FP32 at that order)
        _sweep(P, lambda: P.dg_operator_setup(mesh, 2, P.DG_FP32, 0), P.dg_op_destroy)
        eps = random_permittivity(EToV.shape[0], seed=2)
        _sweep(P, lambda: P.dg_operator_setup_media(mesh, 4, eps, P.DG_FP32, 0), P.dg_op_destroy)
    finally:
        P.dg_mesh_destroy(mesh)
    # still usable
    s = P.Solver(VX, VY, EToV, N=3)
    x, y = s.nodes()
    q = s.from_numpy(np.stack(gaussian_pulse(x, y)))
    s.step(q, s.new_fields(), s.cfl_dt(), 2)
    P.dg_sync_check(s.op)
    assert np.isfinite(s.to_numpy(q)).all()


def test_batch_and_server(P):
    n = _sweep(P, lambda: P.dg_batch_create([0, 0, 2000, 0, 2000, 0, 0], 0),
               P.dg_batch_destroy)
    assert n >= 5
    _sweep(P, lambda: P.dg_server_create([0, 0, 2000, 0, 0, 0, 0], False), P.dg_server_destroy)
    # a batch made after the failures steps correctly
    s = P.Solver(*jittered_delaunay_mesh(8, seed=3), N=3, host_only=True)
    b = P.Batch({3: 256})
    slot = b.add(s, 0.8 * s.cfl_dt())
    x, y = s.nodes()
    b.set_fields(slot, np.stack(gaussian_pulse(x, y)).astype(np.float32))
    b.step(2)
    b.sync_check()
    assert np.isfinite(b.get_fields(slot)).all()
    b.close()


def test_partition(P):
    s = P.Solver(*jittered_delaunay_mesh(20, seed=4), N=4)
    n = _sweep(P, lambda: P.dg_partition_create(s.op, 3), P.dg_partition_destroy)
    assert n >= 3 * 10
    part = P.Partition(s, 3)
    x, y = s.nodes()
    q0 = s.from_numpy(np.stack(gaussian_pulse(x, y)))
    part.set_fields(q0)
    part.step(s.cfl_dt(), 1)
    part.sync_check()
    part.close()
