"""GPU parity of operators with a per-element permittivity
(dg_operator_setup_media) against the oracle's maxwell_rhs_media, through
the C ABI.

Tolerances (max nodal error relative to max |value| of the compared
quantity): FP64 <= 1e-12, FP32 <= 1e-5, as for the uniform medium.  FP32
runs feed the oracle the FP32-rounded input the solver holds.
"""
import numpy as np
import pytest

import oracle as O
from synth import gaussian_pulse, jittered_delaunay_mesh, random_fields, random_permittivity

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp32simt": 1e-5}


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


def _as_held(q, prec):
    return q if prec == "fp64" else q.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32simt"])
@pytest.mark.parametrize("N", [1, 3, 5, 7])
def test_media_rhs_parity(P, N, prec):
    mesh = jittered_delaunay_mesh(9, seed=300 + N)  # K = 162: several blocks, ragged tail
    d = O.Discretization(*mesh, N)
    eps = random_permittivity(d.K, seed=N)
    q = _as_held(random_fields(d.K, d.Np, seed=10 + N), prec)
    want = O.maxwell_rhs_media(d, q, eps)
    s = P.Solver(*mesh, N=N, precision=prec, eps=eps)
    got = s.to_numpy(s.rhs(s.from_numpy(q)))
    P.dg_sync_check(s.op)
    s.close()
    assert _rel(got, want) <= TOL[prec], _rel(got, want)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("N", [2, 5, 7])
def test_media_steps_parity(P, N, prec):
    mesh = jittered_delaunay_mesh(7, seed=40 + N)  # K = 98
    d = O.Discretization(*mesh, N)
    eps = random_permittivity(d.K, seed=7 * N)
    q0 = _as_held(np.stack(gaussian_pulse(d.x, d.y, 0.5, 0.5, 0.15)), prec)
    s = P.Solver(*mesh, N=N, precision=prec, eps=eps)
    dt = s.cfl_dt()
    want = q0
    rhs = lambda u, t: O.maxwell_rhs_media(d, u, eps)  # noqa: E731
    for n in range(3):
        want = O.lsrk_step(d, want, n * dt, dt, rhs=rhs)
    q = s.from_numpy(q0)
    res = s.new_fields()
    s.step(q, res, dt, nsteps=3)
    P.dg_sync_check(s.op)
    got = s.to_numpy(q)
    s.close()
    assert _rel(got, want) <= TOL[prec], _rel(got, want)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_unit_permittivity_equals_plain_operator(P, prec):
    mesh = jittered_delaunay_mesh(8, seed=5)
    N = 4
    d = O.Discretization(*mesh, N)
    q = _as_held(random_fields(d.K, d.Np, seed=3), prec)
    a = P.Solver(*mesh, N=N, precision=prec)
    b = P.Solver(*mesh, N=N, precision=prec, eps=np.ones(d.K))
    ra = a.to_numpy(a.rhs(a.from_numpy(q)))
    rb = b.to_numpy(b.rhs(b.from_numpy(q)))
    a.close()
    b.close()
    assert _rel(rb, ra) <= TOL[prec]


def test_media_energy_does_not_grow(P):
    # eps-weighted energy of the FP64 GPU solution over 20 steps
    mesh = jittered_delaunay_mesh(6, seed=21)
    N = 3
    d = O.Discretization(*mesh, N)
    eps = random_permittivity(d.K, seed=22)
    q0 = np.stack(gaussian_pulse(d.x, d.y, 0.4, 0.6, 0.15))
    s = P.Solver(*mesh, N=N, precision="fp64", eps=eps)
    dt = s.cfl_dt()
    q = s.from_numpy(q0)
    res = s.new_fields()
    e_prev = O.energy_media(d, q0, eps)
    for _ in range(20):
        s.step(q, res, dt, nsteps=1)
        e = O.energy_media(d, s.to_numpy(q), eps)
        assert e <= e_prev * (1 + 1e-13)
        e_prev = e
    s.close()
