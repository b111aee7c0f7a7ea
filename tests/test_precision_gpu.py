"""GPU: the precision path of the element-local contractions (FP32 fields and
accumulation; Dr, Ds, LIFT products in TF32, BF16 or split BF16) against the
FP64 oracle.

Tolerances follow from the operand rounding.  A product of operands rounded
to unit roundoff u has relative error up to about 2u per term; summed over
a row, the error relative to the largest right-hand-side value is 2u times
the ratio of sum |x_k op_k| to |sum x_k op_k|.  That ratio is small for the
smooth, deflated operands the kernels build (a few units), so the bound is
set at 32u:
  TF32 (one product)          u = 2^-11  -> 1.6e-2
  BF16 (one product)          u = 2^-8   -> 1.25e-1
  BF16 hi/lo, three products  u ~ 2^-16  -> 4.9e-4
The errors must also come in the order the arithmetic predicts.
"""
import numpy as np
import pytest

import oracle as O
from synth import gaussian_pulse, jittered_delaunay_mesh

pytestmark = pytest.mark.gpu

U = {"tf32": 2.0 ** -11, "bf16": 2.0 ** -8, "bf16x3": 2.0 ** -16, "fp32": 2.0 ** -22}


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1304_5546_gb300 import build as B
    B.build()
    import paper_1304_5546_gb300 as P
    return P


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _f32(q):
    return q.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("N", [1, 3, 5, 7])
def test_rhs_error_bounds_and_order(P, N):
    mesh = jittered_delaunay_mesh(10, seed=300 + N)
    d = O.Discretization(*mesh, N)
    q = _f32(np.stack(gaussian_pulse(d.x, d.y, 0.5, 0.5, 0.15)))
    want = O.maxwell_rhs(d, q)
    err = {}
    for v in ("fp32", "bf16x3", "tf32", "bf16"):
        s = P.Solver(*mesh, N=N, precision=v)
        got = s.to_numpy(s.rhs(s.from_numpy(q)))
        P.dg_sync_check(s.op)
        s.close()
        assert np.isfinite(got).all(), v
        err[v] = _rel(got, want)
        assert err[v] <= 32 * U[v], (v, err[v])
    assert err["fp32"] <= 1e-5
    assert err["fp32"] < err["bf16x3"] < err["tf32"] < err["bf16"], err


@pytest.mark.parametrize("variant", ["tf32", "bf16", "bf16x3"])
def test_steps_stay_close_to_fp64(P, variant):
    # 20 LSRK steps on the pulse.  They move the fields by about
    # 20 dt max|rhs|, which is below max|q| here, so the accumulated
    # product error relative to max|q| stays within the one-evaluation bound
    mesh = jittered_delaunay_mesh(12, seed=77)
    N = 5
    d = O.Discretization(*mesh, N)
    q0 = _f32(np.stack(gaussian_pulse(d.x, d.y, 0.5, 0.5, 0.1)))
    dt = O.cfl_dt(d)
    want = q0
    for n in range(20):
        want = O.lsrk_step(d, want, n * dt, dt)
    s = P.Solver(*mesh, N=N, precision=variant)
    q = s.from_numpy(q0)
    res = s.new_fields()
    s.step(q, res, dt, nsteps=20)
    got = s.to_numpy(q)
    P.dg_sync_check(s.op)
    s.close()
    assert np.isfinite(got).all()
    assert 20 * dt * np.abs(O.maxwell_rhs(d, q0)).max() < np.abs(q0).max()
    assert _rel(got, want) <= 32 * U[variant], _rel(got, want)


def test_variant_flags_are_checked(P):
    mesh = jittered_delaunay_mesh(3, seed=1)
    m = P.dg_mesh_create(*mesh)
    try:
        for flags, prec in ((P._lib.DG_SETUP_TC_TF32 | P._lib.DG_SETUP_TC_BF16, P.DG_FP32),
                            (P._lib.DG_SETUP_TC_BF16, P.DG_FP64),
                            (P._lib.DG_SETUP_TC_BF16X3 | P._lib.DG_SETUP_SIMT, P.DG_FP32),
                            (1 << 10, P.DG_FP32)):
            with pytest.raises(P.DGError) as ex:
                P.dg_operator_setup(m, 3, prec, flags)
            assert ex.value.status == P._lib.DG_ERR_ARG
    finally:
        P.dg_mesh_destroy(m)
