"""GPU: a Ricker point source on a single operator (dg_operator_set_source),
against the FP64 oracle.

The source term f of the problem statement is read as dEz/dt += s(t) delta
(x - x_s), projected onto the nodal basis of the element containing x_s
(oracle: point_source_weights / point_source_rhs, pinned in
test_oracle_source.py).  The library adds it after each stage launch (the
stage update with s(t) w in the right-hand side), at the stage times
t0 + (n + c_i) dt.  Tolerances: FP32 1e-5, FP64 1e-12 of max |value|.
"""
import numpy as np
import pytest

import oracle as O
from synth import gaussian_pulse, jittered_delaunay_mesh, random_permittivity

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


def _setup(P, N, prec, n=14, seed=3, media=False):
    mesh = jittered_delaunay_mesh(n, seed=seed)
    d = O.Discretization(*mesh, N)
    eps = random_permittivity(d.K, seed=seed) if media else None
    s = P.Solver(*mesh, N=N, precision=prec, eps=eps)
    dt = s.cfl_dt()
    # wavelet with its peak inside the run, a = pi f (t - t0) spanning +-1.6
    src = (0.43, 0.58, 0.12 / dt, 2.2 * dt, 1.7)
    P.dg_operator_set_source(s.op, src)
    q0 = np.stack(gaussian_pulse(d.x, d.y, 0.5, 0.5, 0.2))
    if prec != "fp64":
        q0 = q0.astype(np.float32).astype(np.float64)
    return s, d, eps, dt, src, q0


def _oracle_rhs(d, eps, src):
    xs, ys, f, t0, amp = src
    k, w = O.point_source_weights(d, xs, ys)

    def rhs(u, t):
        base = O.maxwell_rhs(d, u) if eps is None else O.maxwell_rhs_media(d, u, eps)
        return base + O.point_source_rhs(d, k, w, O.ricker(t, f, t0, amp))
    return rhs


@pytest.mark.parametrize("N,prec,media", [(3, "fp32", False), (5, "fp32simt", False),
                                          (4, "fp64", False), (5, "fp32", True),
                                          (1, "fp32", False), (7, "fp32", False),
                                          (2, "fp32", True)])
def test_steps_with_source_match_oracle(P, N, prec, media):
    s, d, eps, dt, src, q0 = _setup(P, N, prec, media=media)
    rhs = _oracle_rhs(d, eps, src)
    want = q0
    for n in range(5):
        want = O.lsrk_step(d, want, n * dt, dt, rhs=rhs)
    q, res = s.from_numpy(q0), s.new_fields()
    # two calls: 2 steps from t0 = 0, then 3 steps from t0 = 2 dt
    s.step(q, res, dt, nsteps=2, t0=0.0)
    s.step(q, res, dt, nsteps=3, t0=2 * dt)
    P.dg_sync_check(s.op)
    got = s.to_numpy(q)
    assert _rel(got, want) <= TOL[prec], _rel(got, want)
    # the source did something: the run without it differs by far more
    nosrc = q0
    for n in range(5):
        nosrc = O.lsrk_step(d, nosrc, n * dt, dt,
                            rhs=(lambda u, t: O.maxwell_rhs(d, u)) if eps is None
                            else (lambda u, t: O.maxwell_rhs_media(d, u, eps)))
    assert _rel(nosrc, want) > 1e3 * TOL[prec]
    s.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_rhs_with_source_at_time_t(P, prec):
    s, d, eps, dt, src, q0 = _setup(P, 5, prec)
    t = 2.5 * dt
    out = s.new_fields()
    P.dg_rhs(s.op, s.from_numpy(q0), out, t)
    got = s.to_numpy(out)
    want = _oracle_rhs(d, eps, src)(q0, t)
    assert _rel(got, want) <= TOL[prec], _rel(got, want)
    s.close()


def test_solve_with_source(P):
    s, d, eps, dt, src, q0 = _setup(P, 4, "fp64")
    T = 4.3 * dt
    q, res = s.from_numpy(q0), s.new_fields()
    nsteps, t_end = s.solve(q, res, T)
    dts = t_end / nsteps
    rhs = _oracle_rhs(d, eps, src)
    want = q0
    for n in range(nsteps):
        want = O.lsrk_step(d, want, n * dts, dts, rhs=rhs)
    assert _rel(s.to_numpy(q), want) <= 1e-12
    s.close()


def test_static_step_with_source_equals_step(P):
    s, d, eps, dt, src, q0 = _setup(P, 5, "fp32", n=10)
    qa, ra = s.from_numpy(q0), s.new_fields()
    qb, rb = s.from_numpy(q0), s.new_fields()
    P.dg_step(s.op, qa, ra, 0.5 * dt, dt, 3)
    P.dg_step_static(s.op, qb, rb, 0.5 * dt, dt, 3)
    P.dg_sync_check(s.op)
    np.testing.assert_array_equal(s.to_numpy(qb), s.to_numpy(qa))
    s.close()


def test_source_removed(P):
    s, d, eps, dt, src, q0 = _setup(P, 3, "fp32", n=10)
    P.dg_operator_set_source(s.op, None)
    plain = P.Solver(*jittered_delaunay_mesh(10, seed=3), N=3, precision="fp32")
    qa, ra = s.from_numpy(q0), s.new_fields()
    qb, rb = plain.from_numpy(q0), plain.new_fields()
    s.step(qa, ra, dt, 3)
    plain.step(qb, rb, dt, 3)
    np.testing.assert_array_equal(s.to_numpy(qa), plain.to_numpy(qb))
    s.close()
    plain.close()


def test_partition_refuses_an_operator_with_a_source(P):
    s, *_ = _setup(P, 3, "fp32", n=8)
    with pytest.raises(P.DGError) as ex:
        P.Partition(s, 2)
    assert ex.value.status == P._lib.DG_ERR_ARG
    s.close()
