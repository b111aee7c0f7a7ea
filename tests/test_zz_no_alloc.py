"""dg_step_static (ping-pong buffer in a fixed per-device array, no device
allocation) against dg_step through the C ABI, two calls in a row.

Both entry points launch the same stage kernels in the same order on the
same inputs; only the address of the second field buffer differs.  So the
results must be bit-identical, and are compared exactly: a stale value of
the shared array reaching a result would show.

That the call allocates nothing is checked twice: with the library's
allocation hook armed (dg_test_fail_alloc(1): the next allocation through it
would fail), the call still succeeds and leaves the hook armed; and the
device's free memory is the same before and after a call.

Collected last on purpose: it must also pass after every other GPU test
has run in the same process, and alone in a fresh one.
"""
import numpy as np
import pytest

from synth import gaussian_pulse, jittered_delaunay_mesh, random_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1304_5546_gb300 import build as B
    B.build()
    import paper_1304_5546_gb300 as P
    return P


def _pair(P, n, N, prec, seed):
    mesh = jittered_delaunay_mesh(n, seed=seed)
    s = P.Solver(*mesh, N=N, precision=prec)
    x, y = s.nodes()
    q0 = np.stack(gaussian_pulse(x, y, 0.5, 0.5, 0.1)) + 0.1 * random_fields(s.K, s.Np, seed)
    return s, q0


def _assert_same(s, qa, ra, qb, rb):
    np.testing.assert_array_equal(s.to_numpy(qb), s.to_numpy(qa))
    np.testing.assert_array_equal(s.to_numpy(rb), s.to_numpy(ra))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("N", [1, 5, 7])
def test_static_matches_dg_step_two_calls(P, N, prec):
    s, q0 = _pair(P, 12, N, prec, seed=40 + N)
    dt = s.cfl_dt()
    qa, ra = s.from_numpy(q0), s.new_fields()
    qb, rb = s.from_numpy(q0), s.new_fields()
    # two calls in a row: an odd step count (copy-back from the scratch),
    # then an even one continuing from the first call's result
    for call, nsteps in enumerate([1, 2]):
        t0 = (0 if call == 0 else 1) * dt
        P.dg_step(s.op, qa, ra, t0, dt, nsteps)
        P.dg_step_static(s.op, qb, rb, t0, dt, nsteps)
        P.dg_sync_check(s.op)
        assert np.isfinite(s.to_numpy(qb)).all()
        _assert_same(s, qa, ra, qb, rb)
    s.close()


def test_static_after_another_operator_used_the_scratch(P):
    # a larger operator leaves its values in the shared array first
    big, qbig = _pair(P, 40, 5, "fp32", seed=3)
    qg, rg = big.from_numpy(qbig), big.new_fields()
    P.dg_step_static(big.op, qg, rg, 0.0, big.cfl_dt(), 1)
    P.dg_sync_check(big.op)
    s, q0 = _pair(P, 9, 5, "fp32", seed=4)
    dt = s.cfl_dt()
    qa, ra = s.from_numpy(q0), s.new_fields()
    qb, rb = s.from_numpy(q0), s.new_fields()
    P.dg_step(s.op, qa, ra, 0.0, dt, 3)
    P.dg_step_static(s.op, qb, rb, 0.0, dt, 3)
    P.dg_sync_check(s.op)
    _assert_same(s, qa, ra, qb, rb)
    s.close()
    big.close()


def test_static_allocates_nothing(P):
    import torch
    s, q0 = _pair(P, 30, 4, "fp32", seed=7)
    dt = s.cfl_dt()
    qa, ra = s.from_numpy(q0), s.new_fields()
    qb, rb = s.from_numpy(q0), s.new_fields()
    P.dg_step_static(s.op, qb, rb, 0.0, dt, 1)  # warm-up: kernels loaded
    P.dg_step(s.op, qa, ra, 0.0, dt, 1)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    P.dg_test_fail_alloc(1)
    try:
        P.dg_step_static(s.op, qb, rb, dt, dt, 3)
        torch.cuda.synchronize()
        # the hook was not reached: nothing went through the allocator
        assert P.dg_test_fail_alloc_pending() == 1
    finally:
        P.dg_test_fail_alloc(0)
    assert torch.cuda.mem_get_info()[0] == free0
    P.dg_step(s.op, qa, ra, dt, dt, 3)
    P.dg_sync_check(s.op)
    _assert_same(s, qa, ra, qb, rb)
    s.close()


def test_static_largest_fitting_operator(P):
    # n = 257: K = 132,098 elements at N = 5, 3 fields of field_stride floats
    # just under the 32 MiB array
    s, q0 = _pair(P, 257, 5, "fp32", seed=5)
    assert 3 * s.fstride * 4 <= P._lib.DG_STATIC_SCRATCH_BYTES
    dt = s.cfl_dt()
    qa, ra = s.from_numpy(q0), s.new_fields()
    qb, rb = s.from_numpy(q0), s.new_fields()
    for nsteps in (1, 1):
        P.dg_step(s.op, qa, ra, 0.0, dt, nsteps)
        P.dg_step_static(s.op, qb, rb, 0.0, dt, nsteps)
        P.dg_sync_check(s.op)
        _assert_same(s, qa, ra, qb, rb)
    s.close()


def test_static_rejects_fields_larger_than_the_array(P):
    s, q0 = _pair(P, 260, 5, "fp32", seed=6)  # K = 135,200: 34 MB of scratch
    assert 3 * s.fstride * 4 > P._lib.DG_STATIC_SCRATCH_BYTES
    q, r = s.from_numpy(q0), s.new_fields()
    before = s.to_numpy(q)
    with pytest.raises(P.DGError) as ex:
        P.dg_step_static(s.op, q, r, 0.0, s.cfl_dt(), 1)
    assert ex.value.status == P._lib.DG_ERR_ARG
    assert "static scratch" in P.dg_last_error()
    P.dg_sync_check(s.op)
    np.testing.assert_array_equal(s.to_numpy(q), before)  # untouched
    s.close()
