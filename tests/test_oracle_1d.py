"""Pins for the oracle's 1D building blocks against library quadrature,
closed forms and finite differences (not against the oracle itself)."""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from scipy import special

import oracle as O


@pytest.mark.parametrize("a,b", [(0.0, 0.0), (1.0, 1.0), (3.0, 0.0), (7.0, 0.0), (13.0, 0.0)])
def test_jacobi_orthonormal_under_library_quadrature(a, b):
    # scipy's Gauss-Jacobi rule integrates degree <= 2*20-1 exactly
    x, w = special.roots_jacobi(20, a, b)
    P = np.stack([O.jacobi_p(x, a, b, n) for n in range(9)])
    G = (P * w) @ P.T
    assert np.allclose(G, np.eye(9), atol=1e-12)


@pytest.mark.parametrize("a,b", [(0.0, 0.0), (1.0, 1.0), (5.0, 0.0)])
def test_jacobi_positive_multiple_of_library_polynomial(a, b):
    x = np.linspace(-0.97, 0.99, 17)
    for n in range(8):
        ours = O.jacobi_p(x, a, b, n)
        ref = special.eval_jacobi(n, a, b, x)
        ratio = ours / ref
        assert np.all(ratio > 0)
        assert np.allclose(ratio, ratio[0], rtol=1e-12)


def test_grad_jacobi_matches_finite_differences():
    x = np.linspace(-0.9, 0.9, 11)
    h = 1e-6
    for a, b in [(0.0, 0.0), (1.0, 1.0), (3.0, 0.0)]:
        for n in range(1, 8):
            fd = (O.jacobi_p(x + h, a, b, n) - O.jacobi_p(x - h, a, b, n)) / (2 * h)
            assert np.allclose(O.grad_jacobi_p(x, a, b, n), fd, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("a,b,m", [(0.0, 0.0, 5), (1.0, 1.0, 6), (2.0, 0.0, 4), (1.0, 1.0, 1)])
def test_gauss_jacobi_nodes_match_library(a, b, m):
    x, _ = special.roots_jacobi(m, a, b)
    assert np.allclose(O.gauss_jacobi_nodes(a, b, m), np.sort(x), atol=1e-14)


def test_lgl_nodes_are_legendre_derivative_roots():
    for N in range(1, 11):
        interior = np.sort(npleg.Legendre.basis(N).deriv().roots().real) if N > 1 else np.zeros(0)
        expect = np.concatenate([[-1.0], interior, [1.0]])
        assert np.allclose(O.lgl_nodes(N), expect, atol=1e-13)


def test_lgl_nodes_closed_forms():
    # textbook closed forms of the Gauss-Lobatto-Legendre points
    closed = {
        2: [0.0],
        3: [-1 / math.sqrt(5), 1 / math.sqrt(5)],
        4: [-math.sqrt(3 / 7), 0.0, math.sqrt(3 / 7)],
        5: sorted([s * math.sqrt(1 / 3 + t * 2 * math.sqrt(7) / 21) for s in (-1, 1) for t in (-1, 1)]),
    }
    for N, inner in closed.items():
        assert np.allclose(O.lgl_nodes(N)[1:-1], inner, atol=1e-15)


def test_vandermonde_1d_mass_is_legendre_mass():
    # (V V^T)^{-1} is the exact mass matrix of the Lagrange basis on the nodes:
    # u^T M v = integral of u v, checked for monomials with closed-form integrals
    for N in range(1, 8):
        r = O.lgl_nodes(N)
        V = O.vandermonde_1d(N, r)
        M = np.linalg.inv(V @ V.T)
        for p in range(N + 1):
            for q in range(N + 1):
                exact = (1 - (-1) ** (p + q + 1)) / (p + q + 1)
                assert abs(r ** p @ M @ r ** q - exact) < 1e-12
