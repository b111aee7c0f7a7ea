"""GPU checks of dg_operator_tune: the FP32 kernel and element-block size
chosen by measurement on the operator's own mesh.  Every candidate (tensor
cores in each block size, CUDA cores) is timed, the fastest is kept, and
the results still match the oracle within the FP32 tolerance; operators
whose set-up fixed the kernel are left alone.  dg_operator_set_block_elems
accepts exactly the sizes the operator's kernel has."""
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
    # candidates: tensor cores in each block size (two at N <= 4), CUDA cores
    # with a thread per node, CUDA cores with a thread per element (N <= 5)
    ncand = (3 if N <= 4 else 2) + 1
    assert P.dg_launch_count(s.op) - n0 == ncand * 4
    kernel, elems = s.kernel()
    if kernel == "tensor cores":
        assert elems in ((40, 80) if N <= 4 else (40,))
    elif kernel == "element threads":
        assert elems == 32
    else:
        assert elems == {1: 64, 3: 32, 5: 24}[N]
    got = s.to_numpy(s.rhs(s.from_numpy(q)))
    P.dg_sync_check(s.op)
    s.close()
    assert _rel(got, O.maxwell_rhs(d, q)) <= 1e-5


@pytest.mark.parametrize("prec", ["fp64", "fp32simt", "tf32", "fp32ept"])
def test_tune_leaves_fixed_kernels_alone(P, prec):
    s = P.Solver(*jittered_delaunay_mesh(4, seed=1), N=3, precision=prec)
    before = s.kernel()
    assert s.tune(reps=2) == (-1.0, -1.0)
    assert s.kernel() == before
    s.close()


def test_tune_with_tensor_cores_forced_chooses_the_block_size(P):
    s = P.Solver(*jittered_delaunay_mesh(20, seed=2), N=3, precision="fp32tc")
    assert s.kernel() == ("tensor cores", 80)
    ms_tc, ms_cc = s.tune(reps=2)
    assert ms_tc > 0 and ms_cc == -1.0
    assert s.kernel()[0] == "tensor cores" and s.kernel()[1] in (40, 80)
    s.close()


@pytest.mark.parametrize("N,prec,sizes", [(3, "fp32tc", (80, 40)), (4, "fp32tc", (40, 80)),
                                          (5, "fp32tc", (40,)), (3, "fp32simt", (32,)),
                                          (2, "fp64", (16,)), (3, "bf16x3", (80,)),
                                          (2, "fp32ept", (32,))])
def test_block_elems_selection(P, N, prec, sizes):
    s = P.Solver(*jittered_delaunay_mesh(6, seed=3), N=N, precision=prec)
    assert s.kernel()[1] == sizes[0]
    for e in sizes:
        P.dg_operator_set_block_elems(s.op, e)
        assert s.kernel()[1] == e
    P.dg_operator_set_block_elems(s.op, 0)
    assert s.kernel()[1] == sizes[0]
    with pytest.raises(P.DGError) as ex:
        P.dg_operator_set_block_elems(s.op, 24)
    assert ex.value.status == P._lib.DG_ERR_ARG
    s.close()
