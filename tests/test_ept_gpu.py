"""GPU parity of the element-thread stage kernel (DG_SETUP_ELEMENT_THREADS,
precision "fp32ept": FP32 on the CUDA cores, one thread per element, the
reference matrices as constant operands; N = 1..5, uniform medium and
per-element permittivity) against the FP64 oracle on the same seeded inputs.

Each warp of that kernel walks blocks of 32 elements through its own ring
of S = 2 stage buffers (from N = 2 on with one residual buffer beside
them).  Besides small
meshes, every order runs on a mesh large enough that each warp of the
launch handles at least S + 2 blocks, so the ring wraps, the one-block-ahead
neighbour gather crosses blocks many times, and the last block is ragged.
The bound on the number of warps comes from shared memory alone (other
limits only shrink the grid, which gives each warp more blocks).

Tolerance: max nodal error <= 1e-5 relative to max |value| (FP32 fields).
"""
import numpy as np
import pytest

import oracle as O
from synth import gaussian_pulse, jittered_delaunay_mesh, random_fields, random_permittivity

pytestmark = pytest.mark.gpu

TOL = 1e-5
ORDERS = [1, 2, 3, 4, 5]


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


def _warps_bound(N, sms=152, smem_per_sm=233472, reserved=1024, max_ctas=32):
    # one warp per CTA; its shared memory is S = 2 stage buffers of 32
    # elements (q: 3 Np values, 13 geometry values), the residual (3 Np
    # values: in each stage buffer at N = 1, in one buffer of its own above)
    # and three blocks' face codes (3 each); more with media records or the
    # operator table, which only lowers the bound
    Np = (N + 1) * (N + 2) // 2
    S = 2
    res = S if N == 1 else 1
    smem = S * 128 * (3 * Np + 13) + res * 128 * 3 * Np + 3 * 384
    return sms * min(max_ctas, smem_per_sm // (smem + reserved)), S


def _n_for(N):
    # smallest jittered grid n (K = 2 n^2) with >= S + 2 blocks per warp and
    # a ragged last block
    warps, S = _warps_bound(N)
    n = int(np.ceil(np.sqrt((S + 2) * warps * 32 / 2)))
    while (2 * n * n) % 32 == 0:
        n += 1
    return n


def test_large_sizes_walk_the_ring():
    for N in ORDERS:
        warps, S = _warps_bound(N)
        K = 2 * _n_for(N) ** 2
        assert -(-K // 32) / warps >= S + 2 and K % 32 != 0, (N, K)


@pytest.mark.parametrize("N", ORDERS)
def test_kernel_report(P, N):
    s = P.Solver(*jittered_delaunay_mesh(5, seed=N), N=N, precision="fp32ept")
    assert s.kernel() == ("element threads", 32)
    s.close()


@pytest.mark.parametrize("N", ORDERS)
def test_rhs_parity_small(P, N):
    # 162 elements: several warps, a ragged last block
    mesh = jittered_delaunay_mesh(9, seed=100 + N)
    d = O.Discretization(*mesh, N)
    q = random_fields(d.K, d.Np, seed=N)
    s = P.Solver(*mesh, N=N, precision="fp32ept")
    got = s.to_numpy(s.rhs(s.from_numpy(q)))
    P.dg_sync_check(s.op)
    s.close()
    assert _rel(got, O.maxwell_rhs(d, q)) <= TOL


@pytest.mark.parametrize("N", ORDERS)
def test_lsrk_steps_parity_small(P, N):
    mesh = jittered_delaunay_mesh(8, seed=7 * N)
    d = O.Discretization(*mesh, N)
    q0 = np.stack(gaussian_pulse(d.x, d.y, 0.5, 0.5, 0.15))
    dt = O.cfl_dt(d)
    want = q0
    for n in range(3):
        want = O.lsrk_step(d, want, n * dt, dt)
    s = P.Solver(*mesh, N=N, precision="fp32ept")
    q = s.from_numpy(q0)
    res = s.new_fields()
    s.step(q, res, dt, nsteps=3)
    got = s.to_numpy(q)
    P.dg_sync_check(s.op)
    s.close()
    assert _rel(got, want) <= TOL


@pytest.mark.parametrize("alpha", [0.0, 0.5])
def test_flux_parameter(P, alpha):
    mesh = jittered_delaunay_mesh(10, seed=31)
    d = O.Discretization(*mesh, 3)
    q = random_fields(d.K, d.Np, seed=3)
    s = P.Solver(*mesh, N=3, precision="fp32ept")
    P.dg_operator_set_alpha(s.op, alpha)
    got = s.to_numpy(s.rhs(s.from_numpy(q)))
    s.close()
    assert _rel(got, O.maxwell_rhs(d, q, alpha=alpha)) <= TOL


@pytest.mark.parametrize("N", ORDERS)
def test_large_rhs_and_two_steps(P, N):
    mesh = jittered_delaunay_mesh(_n_for(N), seed=900 + N)
    d = O.Discretization(*mesh, N)
    q0 = random_fields(d.K, d.Np, seed=N + 1).astype(np.float32).astype(np.float64)
    s = P.Solver(*mesh, N=N, precision="fp32ept")
    try:
        dt = s.cfl_dt()
        q = s.from_numpy(q0)
        rhs = s.to_numpy(s.rhs(q))
        res = s.new_fields()
        s.step(q, res, dt, nsteps=2)
        got = s.to_numpy(q)
        P.dg_sync_check(s.op)
    finally:
        s.close()
    assert _rel(rhs, O.maxwell_rhs(d, q0)) <= TOL, ("rhs", _rel(rhs, O.maxwell_rhs(d, q0)))
    want = q0
    for n in range(2):
        want = O.lsrk_step(d, want, n * dt, dt)
    assert _rel(got, want) <= TOL, ("2 steps", _rel(got, want))


def test_same_result_as_node_thread_kernel_up_to_rounding(P):
    # same inputs through the element-thread and the node-thread CUDA-core
    # kernels: equal within FP32 rounding of the same arithmetic
    mesh = jittered_delaunay_mesh(40, seed=17)
    q = random_fields(2 * 40 * 40, 10, seed=5)
    out = []
    for prec in ("fp32ept", "fp32simt"):
        s = P.Solver(*mesh, N=3, precision=prec)
        out.append(s.to_numpy(s.rhs(s.from_numpy(q))))
        s.close()
    assert _rel(out[0], out[1]) <= 1e-6


@pytest.mark.parametrize("N", [1, 2, 3])
def test_media_rhs_and_steps_small(P, N):
    # per-element permittivity: the flux of the exact interface Riemann
    # solution and the 1/eps row scale of the Ez right-hand side
    mesh = jittered_delaunay_mesh(9, seed=300 + N)
    d = O.Discretization(*mesh, N)
    eps = random_permittivity(d.K, seed=N)
    q = random_fields(d.K, d.Np, seed=N + 7)
    s = P.Solver(*mesh, N=N, precision="fp32ept", eps=eps)
    assert s.kernel() == ("element threads", 32)
    got = s.to_numpy(s.rhs(s.from_numpy(q)))
    q0 = np.stack(gaussian_pulse(d.x, d.y, 0.5, 0.5, 0.15))
    dt = s.cfl_dt()
    qq = s.from_numpy(q0)
    res = s.new_fields()
    s.step(qq, res, dt, nsteps=3)
    stepped = s.to_numpy(qq)
    P.dg_sync_check(s.op)
    s.close()
    assert _rel(got, O.maxwell_rhs_media(d, q, eps)) <= TOL
    want = q0
    for n in range(3):
        want = O.lsrk_step(d, want, n * dt, dt, rhs=lambda u, t: O.maxwell_rhs_media(d, u, eps))
    assert _rel(stepped, want) <= TOL


@pytest.mark.parametrize("N", [1, 2])
def test_media_large_rhs_and_two_steps(P, N):
    mesh = jittered_delaunay_mesh(_n_for(N), seed=950 + N)
    d = O.Discretization(*mesh, N)
    eps = random_permittivity(d.K, seed=960 + N)
    q0 = random_fields(d.K, d.Np, seed=N + 3).astype(np.float32).astype(np.float64)
    s = P.Solver(*mesh, N=N, precision="fp32ept", eps=eps)
    try:
        dt = s.cfl_dt()
        q = s.from_numpy(q0)
        rhs = s.to_numpy(s.rhs(q))
        res = s.new_fields()
        s.step(q, res, dt, nsteps=2)
        got = s.to_numpy(q)
        P.dg_sync_check(s.op)
    finally:
        s.close()

    def f(u, t):
        return O.maxwell_rhs_media(d, u, eps)
    assert _rel(rhs, f(q0, 0.0)) <= TOL, ("rhs", _rel(rhs, f(q0, 0.0)))
    want = q0
    for n in range(2):
        want = O.lsrk_step(d, want, n * dt, dt, rhs=f)
    assert _rel(got, want) <= TOL, ("2 steps", _rel(got, want))


def test_media_same_result_as_node_thread_kernel_up_to_rounding(P):
    mesh = jittered_delaunay_mesh(40, seed=19)
    K = 2 * 40 * 40
    eps = random_permittivity(K, seed=4)
    q = random_fields(K, 6, seed=6)
    out = []
    for prec in ("fp32ept", "fp32simt"):
        s = P.Solver(*mesh, N=2, precision=prec, eps=eps)
        out.append(s.to_numpy(s.rhs(s.from_numpy(q))))
        s.close()
    assert _rel(out[0], out[1]) <= 1e-6


def test_tiny_meshes(P):
    # K = 1 (all faces PEC), 2 and 3: one partly filled block, every order
    from synth import square_grid_mesh
    meshes = [
        (np.array([0.0, 1.0, 0.2]), np.array([0.0, 0.1, 0.9]), np.array([[0, 1, 2]])),
        square_grid_mesh(1, 1),
        (np.array([0.0, 1.0, 0.0, 1.0, 2.0]), np.array([0.0, 0.0, 1.0, 1.0, 0.5]),
         np.array([[0, 1, 3], [0, 3, 2], [1, 4, 3]])),
    ]
    for mesh in meshes:
        for N in ORDERS:
            d = O.Discretization(*mesh, N)
            q = random_fields(d.K, d.Np, seed=N)
            s = P.Solver(*mesh, N=N, precision="fp32ept")
            got = s.to_numpy(s.rhs(s.from_numpy(q)))
            P.dg_sync_check(s.op)
            s.close()
            assert _rel(got, O.maxwell_rhs(d, q)) <= TOL, (d.K, N)


@pytest.mark.parametrize("N,media", [(1, False), (2, False), (2, True)])
def test_hundred_steps_against_oracle(P, N, media):
    # accumulated error of the default FP32 kernel at N <= 2 over 100 LSRK
    # steps of a smooth pulse (the FP32 start rounded for both sides)
    mesh = jittered_delaunay_mesh(60, seed=70 + N)
    d = O.Discretization(*mesh, N)
    eps = random_permittivity(d.K, seed=71) if media else None
    q0 = np.stack(gaussian_pulse(d.x, d.y, 0.5, 0.5, 0.1)).astype(np.float32).astype(np.float64)
    s = P.Solver(*mesh, N=N, precision="fp32", eps=eps)
    assert s.kernel()[0] == "element threads"
    dt = s.cfl_dt()
    q = s.from_numpy(q0)
    s.step(q, s.new_fields(), dt, nsteps=100)
    got = s.to_numpy(q)
    P.dg_sync_check(s.op)
    s.close()

    def f(u, t):
        return O.maxwell_rhs(d, u) if eps is None else O.maxwell_rhs_media(d, u, eps)
    want = q0
    for n in range(100):
        want = O.lsrk_step(d, want, n * dt, dt, rhs=f)
    assert _rel(got, want) <= TOL, _rel(got, want)
