"""GPU parity of the flux parameter alpha of Eq. max2d-numflux
(dg_operator_set_alpha): the central flux (alpha = 0) and a blend (alpha =
0.5) against the oracle's maxwell_rhs with the same alpha, and the central
flux's energy conservation in FP64 (the semi-discrete operator is skew in
the mass-weighted inner product, so the energy rate vanishes up to
rounding)."""
import numpy as np
import pytest

import oracle as O
from synth import jittered_delaunay_mesh, random_fields

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


@pytest.mark.parametrize("alpha", [0.0, 0.5])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32simt"])
@pytest.mark.parametrize("N", [2, 5, 7])
def test_rhs_parity_with_alpha(P, N, prec, alpha):
    mesh = jittered_delaunay_mesh(8, seed=60 + N)
    d = O.Discretization(*mesh, N)
    q = random_fields(d.K, d.Np, seed=N + 7)
    if prec != "fp64":
        q = q.astype(np.float32).astype(np.float64)
    want = O.maxwell_rhs(d, q, alpha=alpha)
    s = P.Solver(*mesh, N=N, precision=prec)
    P.dg_operator_set_alpha(s.op, alpha)
    got = s.to_numpy(s.rhs(s.from_numpy(q)))
    P.dg_sync_check(s.op)
    s.close()
    assert _rel(got, want) <= TOL[prec], _rel(got, want)


def test_central_flux_conserves_energy(P):
    mesh = jittered_delaunay_mesh(6, seed=3)
    N = 4
    d = O.Discretization(*mesh, N)
    q = random_fields(d.K, d.Np, seed=5)
    s = P.Solver(*mesh, N=N, precision="fp64")
    P.dg_operator_set_alpha(s.op, 0.0)
    rhs = s.to_numpy(s.rhs(s.from_numpy(q)))
    P.dg_operator_set_alpha(s.op, 1.0)
    rhs_up = s.to_numpy(s.rhs(s.from_numpy(q)))
    s.close()
    scale = O.energy(d, q) * np.abs(rhs).max() / np.abs(q).max()
    assert abs(O.energy_rate(d, q, rhs)) <= 1e-12 * scale
    assert O.energy_rate(d, q, rhs_up) < -1e-6 * scale  # upwind dissipates
