"""Pins for the oracle's LSRK(5,4) integrator: Butcher order conditions,
stage-time consistency, stability polynomial, and the CFL time-step rule."""
import math

import numpy as np

import oracle as O
from synth import square_grid_mesh


def test_order_conditions_up_to_four():
    A, b = O.butcher_form()
    c = A.sum(axis=1)
    conds = [
        (b.sum(), 1.0),
        (b @ c, 1 / 2),
        (b @ c ** 2, 1 / 3),
        (b @ A @ c, 1 / 6),
        (b @ c ** 3, 1 / 4),
        (b @ (c * (A @ c)), 1 / 8),
        (b @ A @ c ** 2, 1 / 12),
        (b @ A @ A @ c, 1 / 24),
    ]
    for got, want in conds:
        assert abs(got - want) < 1e-12
    # not fifth order: one fifth-order condition fails
    assert abs(b @ c ** 4 - 1 / 5) > 1e-6 or abs(b @ A @ A @ A @ c - 1 / 120) > 1e-6
    # explicit: strictly lower triangular
    assert np.allclose(np.triu(A), 0.0)


def test_stage_times_consistent_with_butcher_rows():
    A, _ = O.butcher_form()
    assert np.allclose(O.LSRK_C, A.sum(axis=1), atol=1e-15)
    # the printed c_2, c_3, c_5 agree; c_4 is 9.0e-5 off the row sum
    pub = O.LSRK_C_PUBLISHED
    assert np.allclose(pub[[0, 1, 2, 4]], O.LSRK_C[[0, 1, 2, 4]], atol=1e-15)
    assert abs(O.LSRK_C[3] - pub[3] - 9.0e-5) < 1e-7


def test_linear_stability_polynomial():
    # one step on y' = lam y equals R(z) = sum_k b^T A^(k-1) 1 z^k; agrees
    # with exp(z) through z^4
    A, b = O.butcher_form()
    one = np.ones(5)
    coeffs = [1.0] + [b @ np.linalg.matrix_power(A, k - 1) @ one for k in range(1, 6)]
    for k in range(5):
        assert abs(coeffs[k] - 1 / math.factorial(k)) < 1e-12
    for z in (-0.1, -0.5 + 0.3j, -1.2):
        # run the 2N-storage recurrence directly
        u, res = 1.0 + 0j, 0.0 + 0j
        for i in range(5):
            res = O.LSRK_A[i] * res + z * u
            u = u + O.LSRK_B[i] * res
        R = sum(coeffs[k] * z ** k for k in range(6))
        assert abs(u - R) < 1e-14
        assert abs(u - np.exp(z)) < 2 * abs(z) ** 5


def test_fourth_order_convergence_on_ode():
    # y' = [[0,1],[-1,0]] y + t-independent: global error ~ dt^4
    def f(u, t):
        return np.array([u[1], -u[0]])
    errs = []
    for n in (10, 20, 40):
        dt = 1.0 / n
        u = np.array([1.0, 0.0])
        for s in range(n):
            u = O.lsrk_step(None, u, s * dt, dt, rhs=f)
        errs.append(np.abs(u - np.array([math.cos(1.0), -math.sin(1.0)])).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.8)


def test_nonautonomous_uses_stage_times():
    # y' = cos(t): exact y(1) = sin(1); fourth order needs consistent c
    errs = []
    for n in (8, 16, 32):
        dt = 1.0 / n
        u = np.array([0.0])
        for s in range(n):
            u = O.lsrk_step(None, u, s * dt, dt, rhs=lambda v, t: np.array([math.cos(t)]))
        errs.append(abs(u[0] - math.sin(1.0)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.7)


def test_cfl_dt_rule_on_square_grid():
    VX, VY, EToV = square_grid_mesh(8, 8)
    d = O.Discretization(VX, VY, EToV, 4)
    h = 0.25
    inradius = h * (2 - math.sqrt(2)) / 2  # right isosceles triangle, legs h
    g = O.lgl_nodes(4)
    assert abs(O.cfl_dt(d) - (2 / 3) * inradius * (g[1] - g[0])) < 1e-15
