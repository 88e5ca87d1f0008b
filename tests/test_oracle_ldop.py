"""Pins of the oracle's second-level deflation of the little Dirac operator
(Sec. 5.2: global deflation vectors by inverse iteration, prediagonalised third
level, A-DEF1 coarse solver of Table algos).  No GPU.

What fixes them, independently of the oracle's own code:
* Rayleigh-Ritz on any nd-dimensional subspace of a Hermitian matrix gives
  Ritz values theta_k >= lambda_k (Cauchy interlacing), equal to the exact
  eigenvalues when the subspace is invariant; numpy's dense eigvalsh of the
  assembled little Dirac operator gives lambda_k.
* With the complete eigenbasis, Q = A^-1, so A-DEF1's first preconditioned
  direction is the exact solution: one iteration.
* A-DEF1 must reach the dense solution A^-1 b.
"""
import numpy as np
import pytest

import synthetic as sy
from oracle.coarse import coarse_apply
from oracle.dwf import norm2
from oracle.solvers import DeflationSpace, adef1, adef2, cg, ldop_deflation_space


@pytest.fixture(scope="module")
def ldop(little_dirac_12x12x4x4):
    return little_dirac_12x12x4x4


def _apply(A, bl):
    return lambda v: coarse_apply(A, v, bl)


def test_prediagonalised_space_interlaces_and_converges(ldop):
    d, bl, phi, A, Dn, lam_exact = ldop
    nd = 8
    noise = sy.complex_normal(1210, (nd, bl.Vc, 4))
    Z, AZ, lam = ldop_deflation_space(A, bl, noise, steps=3, tol=1e-12)
    Zf, AZf = Z.reshape(nd, -1), AZ.reshape(nd, -1)
    scale = np.abs(lam_exact).max()
    assert np.abs(Zf.conj() @ Zf.T - np.eye(nd)).max() < 1e-12
    assert np.abs(Zf.conj() @ AZf.T - np.diag(lam)).max() < 1e-12 * scale
    assert np.abs(AZ - np.array([coarse_apply(A, z, bl) for z in Z])).max() < 1e-12 * scale
    assert np.all(np.diff(lam) >= 0)
    assert np.all(lam >= lam_exact[:nd] * (1 - 1e-10))          # interlacing
    # the four isolated low modes (0.18 against a bulk from 2.7) are converged
    assert np.all(np.abs(lam[:4] - lam_exact[:4]) <= 1e-5 * lam_exact[:4])
    # and they span a low subspace: the largest Ritz value lies far below the top
    assert lam[-1] < 0.6 * lam_exact[-1]


def test_adef1_with_complete_eigenbasis_is_a_direct_solve(ldop):
    d, bl, phi, A, Dn, lam_exact = ldop
    n = Dn.shape[0]
    noise = sy.complex_normal(1220, (n, bl.Vc, 4))
    Z, AZ, lam = ldop_deflation_space(A, bl, noise, steps=1, tol=1e-14)
    b = sy.coarse_gaussian(bl.Vc, 4, 1221)
    x, it = adef1(_apply(A, bl), b, Z, AZ, lam, 1e-10)
    assert it == 1
    xs = np.linalg.solve(Dn, b.ravel()).reshape(b.shape)
    assert np.sqrt(norm2(x - xs) / norm2(xs)) < 1e-10


@pytest.mark.parametrize("flexible", [True, False])
def test_adef1_reaches_dense_solution_in_fewer_iterations(ldop, flexible):
    d, bl, phi, A, Dn, lam_exact = ldop
    noise = sy.complex_normal(1230, (8, bl.Vc, 4))
    Z, AZ, lam = ldop_deflation_space(A, bl, noise, steps=3, tol=1e-10)
    b = sy.coarse_gaussian(bl.Vc, 4, 1231)
    x, it = adef1(_apply(A, bl), b, Z, AZ, lam, 1e-10, flexible=flexible)
    xs = np.linalg.solve(Dn, b.ravel()).reshape(b.shape)
    assert np.sqrt(norm2(x - xs) / norm2(xs)) < 1e-8
    _, it_cg = cg(_apply(A, bl), b, 1e-10)
    assert it < it_cg


def test_adef2_with_deflated_little_dirac_solver(ldop):
    """The outer A-DEF2 solve with the coarse solve by A-DEF1 (residual 0.04)
    reaches the CG solution; each coarse solve takes fewer iterations than the
    undeflated coarse CG on the same right-hand sides."""
    d, bl, phi, A, Dn, lam_exact = ldop
    Z, AZ, lam = ldop_deflation_space(A, bl, sy.complex_normal(1240, (8, bl.Vc, 4)), steps=3, tol=1e-8)
    b = sy.gaussian_fermion(d.lat.dims, d.Ls, 1241)
    Dd = DeflationSpace(phi, bl, A, coarse_tol=0.04, ldop=(Z, AZ, lam))
    Dc = DeflationSpace(phi, bl, A, coarse_tol=0.04)
    res = adef2(d.mdagm, b, Dd, 1e-8)
    assert res.true_residual < 2e-8
    xs, _ = cg(d.mdagm, b, 1e-12)
    assert np.sqrt(norm2(res.x - xs) / norm2(xs)) < 1e-5
    adef2(d.mdagm, b, Dc, 1e-8)
    assert np.mean(Dd.coarse_iters) < np.mean(Dc.coarse_iters)
