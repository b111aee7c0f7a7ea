"""GPU checks of mesh partitions (dg_partition_*): P parts of one operator
stepped with one halo exchange per LSRK stage on one device.

Each part runs the single-operator stage kernel on its own elements and
reads the traces across its cuts from ghost slots, so the partitioned solve
must equal the unpartitioned one bit for bit (same kernels, same inputs per
element), for every precision and kernel variant and for any P; and it
matches the FP64 oracle within the FP32 tolerance.
"""
import numpy as np
import pytest

import oracle as O
from synth import gaussian_pulse, jittered_delaunay_mesh, random_permittivity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1304_5546_gb300 import build as B
    B.build()
    import paper_1304_5546_gb300 as P
    return P


def _run(P, n, N, precision, nparts, nsteps, seed, media=False):
    import torch
    VX, VY, EToV = jittered_delaunay_mesh(n, seed=seed)
    eps = random_permittivity(EToV.shape[0], seed=seed + 1) if media else None
    s = P.Solver(VX, VY, EToV, N=N, precision=precision, eps=eps)
    x, y = s.nodes()
    q0 = s.from_numpy(gaussian_pulse(x, y, 0.4, 0.6, 0.15))
    dt = 0.9 * s.cfl_dt()
    q, res = q0.clone(), s.new_fields()
    s.step(q, res, dt, nsteps)
    part = P.Partition(s, nparts)
    part.set_fields(q0)
    part.step(dt, nsteps)
    out = s.new_fields()
    part.get_fields(out)
    part.sync_check()
    P.dg_sync_check(s.op)
    torch.cuda.synchronize()
    return s, q, out, dt, (VX, VY, EToV), eps


CASES = [
    # (n, N, precision, parts, steps)
    (12, 5, "fp32", 2, 4),      # tensor cores, one tile per block
    (14, 3, "fp32", 3, 4),      # tensor cores, two tiles per block
    (10, 4, "fp32simt", 5, 3),  # CUDA cores
    (9, 1, "fp32", 4, 3),       # CUDA cores (default at N = 1)
    (8, 3, "fp64", 7, 3),
    (10, 7, "bf16x3", 2, 2),
    (13, 2, "fp32ept", 3, 3),   # CUDA cores, one thread per element
    (12, 5, "fp32ept", 2, 2),
]


@pytest.mark.parametrize("n,N,precision,nparts,nsteps", CASES)
def test_partitioned_equals_unpartitioned(P, n, N, precision, nparts, nsteps):
    import torch
    s, want, got, _, _, _ = _run(P, n, N, precision, nparts, nsteps, seed=n + N)
    assert torch.equal(s.view(got), s.view(want))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_partitioned_media_equals_unpartitioned(P, precision):
    import torch
    s, want, got, _, _, _ = _run(P, 11, 4, precision, 4, 3, seed=5, media=True)
    assert torch.equal(s.view(got), s.view(want))


def test_partitioned_matches_oracle(P):
    s, _, got, dt, mesh, _ = _run(P, 6, 4, "fp32", 3, 3, seed=2)
    d = O.Discretization(*mesh, 4)
    x, y = s.nodes()
    q = np.stack(gaussian_pulse(x, y, 0.4, 0.6, 0.15)).astype(np.float32).astype(np.float64)
    for k in range(3):
        q = O.lsrk_step(d, q, k * dt, dt)
    g = s.to_numpy(got).astype(np.float64)
    assert np.abs(g - q).max() / np.abs(q).max() <= 1e-5


def test_large_mesh_many_blocks(P):
    # about 20k elements in 4 parts: many blocks per part and per CTA
    import torch
    s, want, got, _, _, _ = _run(P, 100, 5, "fp32", 4, 2, seed=9)
    assert torch.equal(s.view(got), s.view(want))
