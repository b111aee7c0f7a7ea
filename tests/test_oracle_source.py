"""Pins of the oracle's point source: the Ricker wavelet against its closed
forms, point location against the affine map, and the projected point load
against point evaluation of polynomials (the defining property of the L2
projection of a delta onto degree-N polynomials on the element)."""
import math

import numpy as np
import pytest

import oracle as O
from synth import jittered_delaunay_mesh


def test_ricker_closed_forms():
    f = 10.0
    t0 = 1.2 / f
    assert O.ricker(t0, f) == pytest.approx(1.0, abs=1e-15)
    z = 1.0 / (math.pi * f * math.sqrt(2.0))  # zeros at tau = +-1/(pi f sqrt 2)
    assert abs(O.ricker(t0 + z, f)) < 1e-15 and abs(O.ricker(t0 - z, f)) < 1e-15
    m = math.sqrt(1.5) / (math.pi * f)  # minima at tau = +-sqrt(3/2)/(pi f): -2 e^-3/2
    assert O.ricker(t0 + m, f) == pytest.approx(-2.0 * math.exp(-1.5), rel=1e-13)
    # zero mean: the wavelet integrates to zero over the line
    t = np.linspace(t0 - 1.0, t0 + 1.0, 200001)
    v = O.ricker(t, f)
    assert abs(np.trapezoid(v, t)) < 1e-10
    assert O.ricker(t0, f, amplitude=3.5) == pytest.approx(3.5)


@pytest.mark.parametrize("N", [1, 3, 5, 7])
def test_point_source_reproduces_point_values(N):
    VX, VY, EToV = jittered_delaunay_mesh(5, seed=9)
    d = O.Discretization(VX, VY, EToV, N)
    rng = np.random.default_rng(N)
    for _ in range(4):
        xs, ys = rng.uniform(0.05, 0.95, size=2)
        k, w = O.point_source_weights(d, xs, ys)
        # the point lies in element k: its affine image of (r, s) is (xs, ys)
        k2, r, s = O.locate_point(d, xs, ys)
        v = d.EToV[k]
        xm = 0.5 * (-(r + s) * d.VX[v[0]] + (1 + r) * d.VX[v[1]] + (1 + s) * d.VX[v[2]])
        ym = 0.5 * (-(r + s) * d.VY[v[0]] + (1 + r) * d.VY[v[1]] + (1 + s) * d.VY[v[2]])
        assert k2 == k and abs(xm - xs) < 1e-14 and abs(ym - ys) < 1e-14
        # integral over element k of w * p equals p(xs, ys) for every monomial
        # x^a y^b of degree <= N (exact quadrature: J_k w^T M p)
        for a in range(N + 1):
            for b in range(N + 1 - a):
                p = d.x[k] ** a * d.y[k] ** b
                got = d.J[k, 0] * w @ d.ref.M @ p
                assert got == pytest.approx(xs ** a * ys ** b, rel=1e-10, abs=1e-12), (a, b)


def test_point_outside_mesh_raises():
    d = O.Discretization(*jittered_delaunay_mesh(3, seed=1), 2)
    with pytest.raises(ValueError):
        O.locate_point(d, 1.5, 0.5)


def test_source_rhs_is_linear_and_local():
    d = O.Discretization(*jittered_delaunay_mesh(4, seed=2), 3)
    k, w = O.point_source_weights(d, 0.41, 0.37)
    a = O.point_source_rhs(d, k, w, 2.0)
    b = O.point_source_rhs(d, k, w, -0.5)
    assert np.array_equal(a + b, O.point_source_rhs(d, k, w, 1.5))
    nz = np.nonzero(np.abs(a).sum(axis=2))
    assert list(zip(*nz)) == [(2, k)]
