"""GPU checks of dg_operator_tune: the FP32 kernel choice by measurement on
the operator's own mesh.  Both kernels are timed, the faster is kept, and
the results still match the oracle within the FP32 tolerance; operators
whose set-up fixed the kernel are left alone."""
import numpy as np
import pytest

import oracle as O
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


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("N", [1, 3, 5])
def test_tune_times_both_kernels_and_keeps_parity(P, N):
    mesh = jittered_delaunay_mesh(10, seed=90 + N)
    d = O.Discretization(*mesh, N)
    q = random_fields(d.K, d.Np, seed=N).astype(np.float32).astype(np.float64)
    s = P.Solver(*mesh, N=N, precision="fp32")
    n0 = P.dg_launch_count(s.op)
    ms_tc, ms_cc = s.tune(reps=3)
    assert ms_tc > 0 and ms_cc > 0
    assert P.dg_launch_count(s.op) - n0 == 2 * 4
    got = s.to_numpy(s.rhs(s.from_numpy(q)))
    P.dg_sync_check(s.op)
    s.close()
    assert _rel(got, O.maxwell_rhs(d, q)) <= 1e-5


@pytest.mark.parametrize("prec", ["fp64", "fp32simt", "fp32tc", "tf32"])
def test_tune_leaves_fixed_kernels_alone(P, prec):
    s = P.Solver(*jittered_delaunay_mesh(4, seed=1), N=3, precision=prec)
    assert s.tune(reps=2) == (-1.0, -1.0)
    s.close()
