"""Pins for the oracle's reference element: Warburton nodes, Dr/Ds, mass
matrix, face masks, face mass matrices and LIFT (Section "Implementation
Aspects", Eqs. dg-diff-local-to-global and dg-lift)."""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import oracle as O

ORDERS = list(range(1, 8))


def _bary(r, s):
    # barycentrics w.r.t. v1=(-1,-1), v2=(1,-1), v3=(-1,1)
    l2 = (1 + r) / 2
    l3 = (1 + s) / 2
    return np.stack([1 - l2 - l3, l2, l3], axis=1)


@pytest.mark.parametrize("N", ORDERS)
def test_nodes_count_vertices_inside(N):
    r, s = O.nodes_2d(N)
    assert r.size == (N + 1) * (N + 2) // 2
    L = _bary(r, s)
    assert np.all(L > -1e-14)
    for v in [(-1, -1), (1, -1), (-1, 1)]:
        assert np.min(np.hypot(r - v[0], s - v[1])) < 1e-14


@pytest.mark.parametrize("N", ORDERS)
def test_nodes_on_edges_are_lgl(N):
    r, s = O.nodes_2d(N)
    lgl = np.sort(npleg.Legendre.basis(N).deriv().roots().real) if N > 1 else np.zeros(0)
    lgl = np.concatenate([[-1.0], lgl, [1.0]])
    on1 = np.abs(s + 1) < 1e-12
    assert np.allclose(np.sort(r[on1]), lgl, atol=1e-13)
    on3 = np.abs(r + 1) < 1e-12
    assert np.allclose(np.sort(s[on3]), lgl, atol=1e-13)
    on2 = np.abs(r + s) < 1e-12
    assert np.allclose(np.sort(r[on2]), lgl, atol=1e-13)


@pytest.mark.parametrize("N", ORDERS)
def test_nodes_symmetric_under_triangle_symmetries(N):
    r, s = O.nodes_2d(N)
    L = _bary(r, s)
    key = {tuple(np.round(row, 11)) for row in L}
    for perm in [(0, 1, 2), (1, 2, 0), (2, 0, 1), (0, 2, 1), (2, 1, 0), (1, 0, 2)]:
        assert {tuple(np.round(row[list(perm)], 11)) for row in L} == key


@pytest.mark.parametrize("N", ORDERS)
def test_node_lattice_order(N):
    # nodes run row by row of constant s bottom-up, r increasing in a row
    r, s = O.nodes_2d(N)
    idx = 0
    for row in range(N + 1):
        rr = r[idx: idx + N + 1 - row]
        assert np.all(np.diff(rr) > 0)
        idx += N + 1 - row
    assert O.face_masks(r, s)[0].tolist() == list(range(N + 1))


def test_blending_parameter_lowers_lebesgue_constant():
    # Warburton's alpha was chosen to lower the Lebesgue constant; at N = 6, 7
    # the tabulated alpha clearly beats alpha = 0 on a fine sample.
    def lebesgue(N, alpha):
        r, s = O.nodes_2d(N, alpha)
        V = O.vandermonde_2d(N, r, s)
        m = 120
        pts = np.array([(-1 + 2 * i / m, -1 + 2 * j / m) for i in range(m + 1) for j in range(m + 1 - i)])
        P = O.vandermonde_2d(N, pts[:, 0], pts[:, 1])
        return np.abs(np.linalg.solve(V.T, P.T)).sum(axis=0).max()
    for N in (6, 7):
        assert lebesgue(N, O.WARBURTON_ALPHA[N]) < 0.97 * lebesgue(N, 0.0)


@pytest.mark.parametrize("N", ORDERS)
def test_dr_ds_differentiate_polynomials_exactly(N):
    R = O.ReferenceElement(N)
    r, s = R.r, R.s
    scale = max(np.abs(R.Dr).max(), np.abs(R.Ds).max())
    for a in range(N + 1):
        for b in range(N + 1 - a):
            u = r ** a * s ** b
            dur = a * r ** (a - 1) * s ** b if a else np.zeros_like(r)
            dus = b * r ** a * s ** (b - 1) if b else np.zeros_like(r)
            assert np.abs(R.Dr @ u - dur).max() < 1e-13 * scale * (N + 1)
            assert np.abs(R.Ds @ u - dus).max() < 1e-13 * scale * (N + 1)
    assert np.abs(R.Dr @ np.ones(R.Np)).max() < 1e-12
    assert np.abs(R.Ds @ np.ones(R.Np)).max() < 1e-12


def _ref_monomial_integral(a, b):
    # integral of r^a s^b over the reference triangle, via r = 2x-1, s = 2y-1
    # on the unit simplex and int x^p y^q = p! q! / (p+q+2)!
    tot = 0.0
    for p in range(a + 1):
        for q in range(b + 1):
            coef = math.comb(a, p) * math.comb(b, q) * 2.0 ** (p + q) * (-1.0) ** (a - p + b - q)
            tot += coef * math.factorial(p) * math.factorial(q) / math.factorial(p + q + 2)
    return 4.0 * tot


@pytest.mark.parametrize("N", ORDERS)
def test_mass_matrix_integrates_products_exactly(N):
    R = O.ReferenceElement(N)
    r, s = R.r, R.s
    assert abs(np.ones(R.Np) @ R.M @ np.ones(R.Np) - 2.0) < 1e-13
    monos = [(a, b) for a in range(N + 1) for b in range(N + 1 - a)]
    for (a1, b1) in monos:
        for (a2, b2) in monos:
            val = (r ** a1 * s ** b1) @ R.M @ (r ** a2 * s ** b2)
            assert abs(val - _ref_monomial_integral(a1 + a2, b1 + b2)) < 1e-11


def _lagrange_1d(nodes, t):
    L = np.ones((len(t), len(nodes)))
    for i in range(len(nodes)):
        for j in range(len(nodes)):
            if j != i:
                L[:, i] *= (t - nodes[j]) / (nodes[i] - nodes[j])
    return L


@pytest.mark.parametrize("N", ORDERS)
def test_lift_reproduces_face_integrals(N):
    # M LIFT g = sum over faces of int_face g l_i d(face coordinate); on face f
    # only the face's own nodes have nonzero basis functions, which restrict to
    # the 1D Lagrange basis on the face nodes.
    R = O.ReferenceElement(N)
    xq, wq = npleg.leggauss(N + 2)
    MLIFT = R.M @ R.LIFT
    for f in range(3):
        coord = R.s if f == 2 else R.r
        fn = coord[R.Fmask[f]]
        Lq = _lagrange_1d(fn, xq)
        Eface = (Lq * wq[:, None]).T @ Lq  # (Nfp, Nfp) exact 1D mass matrix
        block = MLIFT[:, f * R.Nfp:(f + 1) * R.Nfp]
        expect = np.zeros_like(block)
        expect[R.Fmask[f], :] = Eface
        assert np.abs(block - expect).max() < 1e-11


@pytest.mark.parametrize("N", ORDERS)
def test_face_masks(N):
    R = O.ReferenceElement(N)
    Fm = R.Fmask
    assert Fm.shape == (3, N + 1)
    assert np.allclose(R.s[Fm[0]], -1)
    assert np.allclose(R.r[Fm[1]] + R.s[Fm[1]], 0)
    assert np.allclose(R.r[Fm[2]], -1)
    for f in range(3):
        assert np.all(np.diff(Fm[f]) > 0)
    # face 2 runs v2 -> v3 (r decreasing)
    assert np.all(np.diff(R.r[Fm[1]]) < 0)
