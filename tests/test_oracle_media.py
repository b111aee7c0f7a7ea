"""Pins for the oracle's piecewise-constant permittivity right-hand side
(maxwell_rhs_media): Eq. tm-maxwells with a per-element eps, mu = 1, and
the upwind flux of the exact interface Riemann solution."""
import numpy as np
import pytest

import oracle as O
from synth import jittered_delaunay_mesh, random_fields, square_grid_mesh


def test_unit_permittivity_is_the_homogeneous_upwind_rhs():
    d = O.Discretization(*jittered_delaunay_mesh(5, seed=3), 4)
    q = random_fields(d.K, d.Np, seed=1)
    a = O.maxwell_rhs(d, q, alpha=1.0)
    b = O.maxwell_rhs_media(d, q, np.ones(d.K))
    assert np.abs(a - b).max() < 1e-14 * np.abs(a).max()


def test_constant_magnetic_field_is_steady_in_media():
    d = O.Discretization(*jittered_delaunay_mesh(4, seed=5), 3)
    eps = np.where(d.x.mean(1) > 0.5, 4.0, 0.25)
    q = np.zeros((3, d.K, d.Np))
    q[0], q[1] = 0.7, -1.3
    assert np.abs(O.maxwell_rhs_media(d, q, eps)).max() < 1e-11


def test_interface_flux_is_the_riemann_solution():
    # Two elements sharing one face, eps- = 1 and eps+ = 4, piecewise-constant
    # states.  Solve the interface state from the characteristics directly
    # (a 2x2 linear system: E* + Z- H* = E- + Z- H-, E* - Z+ H* = E+ - Z+ H+
    # for the normal system dHt/dt + dEz/dxi = 0, eps dEz/dt + dHt/dxi = 0)
    # and compare n.(F- - F*) with what the oracle lifts onto element 0.
    VX = np.array([0.0, 1.0, 0.0, 1.0])
    VY = np.array([0.0, 0.0, 1.0, 1.0])
    EToV = np.array([[0, 1, 3], [0, 3, 2]])
    d = O.Discretization(VX, VY, EToV, 1)
    eps = np.array([1.0, 4.0])
    Zm, Zp = 1.0, 0.5
    rng = np.random.default_rng(4)
    sM, sP = rng.normal(size=3), rng.normal(size=3)
    q = np.zeros((3, 2, d.Np))
    q[:, 0, :] = sM[:, None]
    q[:, 1, :] = sP[:, None]
    f = int(np.nonzero(d.EToE[0] == 1)[0][0])
    sl = slice(f * d.Nfp, (f + 1) * d.Nfp)
    nx, ny = d.nx[0, sl][0], d.ny[0, sl][0]
    HtM, HtP = ny * sM[0] - nx * sM[1], ny * sP[0] - nx * sP[1]
    Es, Hs = np.linalg.solve(np.array([[1.0, Zm], [1.0, -Zp]]),
                             np.array([sM[2] + Zm * HtM, sP[2] - Zp * HtP]))
    flux_Ez = HtM - Hs          # the Ez equation's flux is Ht
    flux_Ht = sM[2] - Es        # the Ht equation's flux is Ez
    expect = np.array([ny * flux_Ht, -nx * flux_Ht, flux_Ez])
    # isolate the shared face as in the homogeneous Riemann pin: a zero jump
    # with the same impedance gives zero flux, so the difference of two
    # right-hand sides is LIFT_f (Fscale flux); M LIFT_f = E_f and the face
    # mass sums to 2 (Ez row also divided by eps-)
    q_same = q.copy()
    q_same[:, 1, :] = sM[:, None]
    eps_same = np.array([1.0, 1.0])
    diff = (O.maxwell_rhs_media(d, q, eps)[:, 0, :]
            - O.maxwell_rhs_media(d, q_same, eps_same)[:, 0, :])
    R = d.ref
    got = (diff @ R.M.T)[:, R.Fmask[f]].sum(axis=1) / (2 * d.Fscale[0, sl][0])
    got[2] *= eps[0]
    assert np.allclose(got, expect, atol=1e-12)


def _operator(d, eps):
    n = 3 * d.K * d.Np
    A = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        A[:, i] = O.maxwell_rhs_media(d, e.reshape(3, d.K, d.Np), eps).reshape(-1)
    return A


@pytest.mark.parametrize("N", [2, 3])
def test_weighted_operator_is_dissipative(N):
    d = O.Discretization(*square_grid_mesh(2, 2), N)
    eps = np.array([1.0, 4.0, 0.25, 1.0, 2.0, 1.0, 0.5, 4.0])[: d.K]
    A = _operator(d, eps)
    JM = np.kron(np.diag(d.J[:, 0]), d.ref.M)
    W = np.block([[JM, 0 * JM, 0 * JM], [0 * JM, JM, 0 * JM],
                  [0 * JM, 0 * JM, np.kron(np.diag(d.J[:, 0] * eps), d.ref.M)]])
    S = W @ A
    assert np.linalg.eigvalsh(S + S.T).max() < 1e-10
    assert np.linalg.eigvals(A).real.max() < 1e-9


def test_media_energy_does_not_increase_under_lsrk():
    d = O.Discretization(*jittered_delaunay_mesh(5, seed=8), 3)
    eps = np.where(d.y.mean(1) > 0.4, 2.0, 0.5)
    q = random_fields(d.K, d.Np, seed=2)
    dt = 0.5 * O.cfl_dt(d) * np.sqrt(eps.min())
    e_prev = O.energy_media(d, q, eps)
    for n in range(10):
        q = O.lsrk_step(d, q, n * dt, dt, rhs=lambda qq, t: O.maxwell_rhs_media(d, qq, eps))
        e = O.energy_media(d, q, eps)
        assert e <= e_prev * (1 + 1e-13)
        e_prev = e
