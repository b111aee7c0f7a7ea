"""GPU checks of resume and of the timeout path.

* Resume: 7 LSRK steps in one go equal, bit for bit, 3 steps, a checkpoint
  of the device fields, a fresh operator and buffers loaded from it, and 4
  more steps.
* Timeout: dg_test_wait_timeout makes a bounded wait run out (a flag that
  nothing sets); dg_sync_check reports DG_ERR_TIMEOUT, and the operator then
  steps correctly.
"""
import numpy as np
import pytest

import oracle as O
from synth import gaussian_pulse, jittered_delaunay_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1304_5546_gb300 import build as B
    B.build()
    import paper_1304_5546_gb300 as P
    return P


@pytest.mark.parametrize("prec,N", [("fp32", 5), ("fp64", 5), ("fp32", 2)])
def test_resume_is_bitwise(P, tmp_path, prec, N):
    # N = 2 in FP32 runs the element-thread kernel
    mesh = jittered_delaunay_mesh(9, seed=31)
    a = P.Solver(*mesh, N=N, precision=prec)
    x, y = a.nodes()
    q0 = np.stack(gaussian_pulse(x, y, 0.5, 0.5, 0.15))
    dt = a.cfl_dt()
    q = a.from_numpy(q0)
    a.step(q, a.new_fields(), dt, nsteps=7)
    full = a.to_numpy(q)
    q = a.from_numpy(q0)
    res = a.new_fields()
    a.step(q, res, dt, nsteps=3)
    path = tmp_path / "resume.ckpt"
    a.save(q, path, t=3 * dt, step=3)
    a.close()
    b = P.Solver(*mesh, N=N, precision=prec)
    q2 = b.new_fields()
    t, step = b.load(path, q2)
    assert step == 3 and t == 3 * dt
    b.step(q2, b.new_fields(), dt, nsteps=4)
    resumed = b.to_numpy(q2)
    b.close()
    assert np.array_equal(resumed, full)


def test_bounded_wait_times_out_and_operator_recovers(P):
    from paper_1304_5546_gb300 import DGError, _lib
    mesh = jittered_delaunay_mesh(6, seed=2)
    s = P.Solver(*mesh, N=3, precision="fp32")
    P.dg_test_wait_timeout(s.op)
    with pytest.raises(DGError) as ex:
        P.dg_sync_check(s.op)
    assert ex.value.status == _lib.DG_ERR_TIMEOUT
    P.dg_sync_check(s.op)  # the status word was cleared
    d = O.Discretization(*mesh, 3)
    q0 = np.stack(gaussian_pulse(d.x, d.y, 0.5, 0.5, 0.2)).astype(np.float32).astype(np.float64)
    dt = s.cfl_dt()
    q = s.from_numpy(q0)
    s.step(q, s.new_fields(), dt, nsteps=2)
    P.dg_sync_check(s.op)
    want = O.lsrk_step(d, O.lsrk_step(d, q0, 0.0, dt), dt, dt)
    got = s.to_numpy(q)
    s.close()
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
