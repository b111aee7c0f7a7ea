"""Host-side checks of the batch planner and of operators with a
per-element permittivity (no GPU needed).

The planner (dg_batch_plan_ctas) splits a launch's CTAs among the orders of
a batch so that the slowest order finishes first: order g with nblk blocks on
c CTAs takes ceil(nblk / c) block iterations of cost[g].  Its greedy split is
checked against brute force over every split on small cases, where the
minimum of the largest finish time is unique even when the split is not.
"""
import itertools
import math

import numpy as np
import pytest

from synth import jittered_delaunay_mesh, random_permittivity


@pytest.fixture(scope="module")
def dgw():
    from paper_1304_5546_gb300 import build as B
    B.build()
    import paper_1304_5546_gb300 as P
    return P


def _makespan(nblk, cost, cta):
    return max((math.ceil(n / c) * w if n else 0.0) for n, w, c in zip(nblk, cost, cta)
               if n or c)


def _brute_force(nblk, cost, num_ctas):
    active = [g for g in range(7) if nblk[g] > 0]
    best = None
    for split in itertools.product(range(1, num_ctas + 1), repeat=len(active)):
        if sum(split) > num_ctas:
            continue
        cta = [0] * 7
        for g, c in zip(active, split):
            cta[g] = c
        m = _makespan(nblk, cost, cta)
        best = m if best is None else min(best, m)
    return best


@pytest.mark.parametrize("seed", range(12))
def test_plan_is_optimal_on_small_cases(dgw, seed):
    rng = np.random.default_rng(seed)
    num_ctas = int(rng.integers(3, 11))
    nblk = [0] * 7
    cost = [0.0] * 7
    for g in rng.choice(7, size=int(rng.integers(1, 4)), replace=False):
        nblk[g] = int(rng.integers(1, 40))
        cost[g] = float(rng.uniform(0.5, 3.0))
    cta = dgw.dg_batch_plan_ctas(nblk, cost, num_ctas)
    assert cta.sum() <= num_ctas
    for g in range(7):
        if nblk[g]:
            assert 1 <= cta[g] <= nblk[g]
        else:
            assert cta[g] == 0
    assert _makespan(nblk, cost, cta) == pytest.approx(_brute_force(nblk, cost, num_ctas))


def test_plan_uses_every_cta_when_blocks_allow(dgw):
    nblk = [0, 0, 5000, 0, 12000, 0, 3000]
    cost = [0, 0, 1.0, 0, 2.1, 0, 4.0]
    cta = dgw.dg_batch_plan_ctas(nblk, cost, 152)
    assert cta.sum() == 152
    # finish times within one block iteration of each other
    fin = [math.ceil(nblk[g] / cta[g]) * cost[g] for g in (2, 4, 6)]
    assert max(fin) - min(fin) <= max(cost)


def test_plan_rejects_more_orders_than_ctas(dgw):
    from paper_1304_5546_gb300 import DGError
    with pytest.raises(DGError):
        dgw.dg_batch_plan_ctas([1, 1, 1, 0, 0, 0, 0], [1.0] * 7, 2)


def _inradius(VX, VY, EToV):
    x, y = VX[EToV], VY[EToV]
    a = np.hypot(x[:, 1] - x[:, 0], y[:, 1] - y[:, 0])
    b = np.hypot(x[:, 2] - x[:, 1], y[:, 2] - y[:, 1])
    c = np.hypot(x[:, 0] - x[:, 2], y[:, 0] - y[:, 2])
    area = 0.5 * np.abs((x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0])
                        - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0]))
    return area / (0.5 * (a + b + c))


def test_media_cfl_step_uses_local_wave_speed(dgw):
    import oracle as O
    VX, VY, EToV = jittered_delaunay_mesh(6, seed=3)
    eps = random_permittivity(EToV.shape[0], seed=4)
    N = 4
    mesh = dgw.dg_mesh_create(VX, VY, EToV)
    op = dgw.dg_operator_setup_media(mesh, N, eps, dgw.DG_FP32, dgw.DG_SETUP_HOST_ONLY)
    op1 = dgw.dg_operator_setup(mesh, N, dgw.DG_FP32, dgw.DG_SETUP_HOST_ONLY)
    try:
        g = O.lgl_nodes(N)
        want = (2.0 / 3.0) * np.min(_inradius(VX, VY, EToV) * np.sqrt(eps)) * (g[1] - g[0])
        assert dgw.dg_cfl_dt(op) == pytest.approx(want, rel=1e-12)
        # eps = 1: the plain operator's step
        ones = dgw.dg_operator_setup_media(mesh, N, np.ones(EToV.shape[0]), dgw.DG_FP32,
                                           dgw.DG_SETUP_HOST_ONLY)
        assert dgw.dg_cfl_dt(ones) == pytest.approx(dgw.dg_cfl_dt(op1), rel=1e-14)
        dgw.dg_op_destroy(ones)
    finally:
        dgw.dg_op_destroy(op)
        dgw.dg_op_destroy(op1)
        dgw.dg_mesh_destroy(mesh)


def test_media_setup_rejects_bad_input(dgw):
    from paper_1304_5546_gb300 import DGError
    VX, VY, EToV = jittered_delaunay_mesh(3, seed=1)
    K = EToV.shape[0]
    mesh = dgw.dg_mesh_create(VX, VY, EToV)
    try:
        for bad in (np.zeros(K), -np.ones(K), np.full(K, np.nan)):
            with pytest.raises(DGError):
                dgw.dg_operator_setup_media(mesh, 3, bad, dgw.DG_FP32, dgw.DG_SETUP_HOST_ONLY)
        with pytest.raises(DGError):
            dgw.dg_operator_setup_media(mesh, 3, np.ones(K), dgw.DG_FP32,
                                        dgw.DG_SETUP_HOST_ONLY | 4)  # DG_SETUP_TC_TF32
    finally:
        dgw.dg_mesh_destroy(mesh)


def test_set_alpha_checks(dgw):
    from paper_1304_5546_gb300 import DGError
    VX, VY, EToV = jittered_delaunay_mesh(3, seed=1)
    mesh = dgw.dg_mesh_create(VX, VY, EToV)
    op = dgw.dg_operator_setup(mesh, 3, dgw.DG_FP64, dgw.DG_SETUP_HOST_ONLY)
    media = dgw.dg_operator_setup_media(mesh, 3, np.ones(EToV.shape[0]), dgw.DG_FP32,
                                        dgw.DG_SETUP_HOST_ONLY)
    try:
        dgw.dg_operator_set_alpha(op, 0.0)
        dgw.dg_operator_set_alpha(op, 0.25)
        for bad in (-0.1, 1.5, float("nan")):
            with pytest.raises(DGError):
                dgw.dg_operator_set_alpha(op, bad)
        with pytest.raises(DGError):
            dgw.dg_operator_set_alpha(media, 0.0)
    finally:
        dgw.dg_op_destroy(op)
        dgw.dg_op_destroy(media)
        dgw.dg_mesh_destroy(mesh)


def test_tune_needs_a_device_operator(dgw):
    from paper_1304_5546_gb300 import DGError
    VX, VY, EToV = jittered_delaunay_mesh(3, seed=1)
    mesh = dgw.dg_mesh_create(VX, VY, EToV)
    op = dgw.dg_operator_setup(mesh, 3, dgw.DG_FP32, dgw.DG_SETUP_HOST_ONLY)
    try:
        with pytest.raises(DGError):
            dgw.dg_operator_tune(op, 2, stream=0)
    finally:
        dgw.dg_op_destroy(op)
        dgw.dg_mesh_destroy(mesh)
