"""GPU checks of dg_step_host_jobs: independent host-resident field sets,
each copied in, stepped and copied back, with one job's copies overlapping
the next job's steps.  Every result must equal, bit for bit, dg_step_host on
the same fields (same stage launches in the same order), including a host
buffer listed twice in a row (the second job then steps the first one's
result)."""
import numpy as np
import pytest

from synth import jittered_delaunay_mesh, random_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1304_5546_gb300 import build as B
    B.build()
    import paper_1304_5546_gb300 as P
    return P


def _host(s, q3):
    return s.from_numpy(q3).cpu().pin_memory()


@pytest.mark.parametrize("precision,N,nsteps", [("fp32", 5, 1), ("fp32", 3, 2), ("fp64", 4, 1),
                                                ("fp32", 2, 2)])  # N = 2: element threads
def test_jobs_equal_step_host(P, precision, N, nsteps):
    import torch
    s = P.Solver(*jittered_delaunay_mesh(24, seed=5), N=N, precision=precision)
    dt = 0.8 * s.cfl_dt()
    states = [random_fields(s.K, s.Np, seed=10 + i) for i in range(7)]
    dq, dres = s.new_fields(), s.new_fields()
    want = []
    for q3 in states:
        h = _host(s, q3)
        P.dg_step_host(s.op, h, dq, dres, 0.0, dt, nsteps)
        want.append(h)
    hs = [_host(s, q3) for q3 in states]
    work = torch.empty(P.dg_step_host_jobs_work_bytes(s.op), dtype=torch.uint8, device="cuda")
    P.dg_step_host_jobs(s.op, hs, work, 0.0, dt, nsteps)
    n = s.K * s.Np
    for h, w in zip(hs, want):
        assert torch.equal(h.view(3, -1)[:, :n], w.view(3, -1)[:, :n])
    P.dg_sync_check(s.op)


def test_repeated_buffer_steps_in_order(P):
    import torch
    s = P.Solver(*jittered_delaunay_mesh(16, seed=2), N=4, precision="fp32")
    dt = 0.8 * s.cfl_dt()
    q3 = random_fields(s.K, s.Np, seed=3)
    dq, dres = s.new_fields(), s.new_fields()
    want = _host(s, q3)
    for _ in range(4):
        P.dg_step_host(s.op, want, dq, dres, 0.0, dt, 1)
    a, b = _host(s, q3), _host(s, random_fields(s.K, s.Np, seed=4))
    work = torch.empty(P.dg_step_host_jobs_work_bytes(s.op), dtype=torch.uint8, device="cuda")
    # a four times (twice back to back), b in between
    P.dg_step_host_jobs(s.op, [a, a, b, a, a], work, 0.0, dt, 1)
    n = s.K * s.Np
    assert torch.equal(a.view(3, -1)[:, :n], want.view(3, -1)[:, :n])


def test_bad_arguments(P):
    import torch
    s = P.Solver(*jittered_delaunay_mesh(4, seed=1), N=2, precision="fp32")
    work = torch.empty(P.dg_step_host_jobs_work_bytes(s.op), dtype=torch.uint8, device="cuda")
    with pytest.raises(P.DGError):
        P.dg_step_host_jobs(s.op, [_host(s, random_fields(s.K, s.Np, seed=1))], work, 0.0,
                            float("nan"), 1)
    P.dg_step_host_jobs(s.op, [], work, 0.0, 0.1, 1)  # no jobs: nothing to do
    assert P.dg_step_host_jobs_work_bytes(s.op) == 7 * 3 * s.fstride * 4
    assert np.isfinite(s.cfl_dt())
