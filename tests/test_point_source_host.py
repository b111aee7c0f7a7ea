"""CPU: argument checks of dg_operator_set_source on a host-only operator
(the point location and the projected load are computed on the host)."""
import pytest

from synth import jittered_delaunay_mesh


@pytest.fixture(scope="module")
def P():
    from paper_1304_5546_gb300 import build as B
    B.build()
    import paper_1304_5546_gb300 as P
    return P


def test_set_source_checks(P):
    s = P.Solver(*jittered_delaunay_mesh(5, seed=2), N=3, precision="fp32", host_only=True)
    P.dg_operator_set_source(s.op, (0.5, 0.5, 10.0, 0.12, 1.0))
    P.dg_operator_set_source(s.op, None)
    for bad in [(1.5, 0.5, 10.0, 0.1, 1.0), (0.5, 0.5, 0.0, 0.1, 1.0),
                (0.5, float("nan"), 10.0, 0.1, 1.0), (0.5, 0.5, 10.0, float("inf"), 1.0)]:
        with pytest.raises(P.DGError) as ex:
            P.dg_operator_set_source(s.op, bad)
        assert ex.value.status == P._lib.DG_ERR_ARG
    assert "outside the mesh" in str(pytest.raises(
        P.DGError, P.dg_operator_set_source, s.op, (2.0, 2.0, 1.0, 0.0, 1.0)).value)
    s.close()
