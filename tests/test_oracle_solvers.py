"""Pins of the oracle's Krylov solvers (no GPU)."""
import numpy as np
import pytest

import synthetic as sy
from oracle.coarse import Blocking, block_gram_schmidt, coarse_dense_bruteforce, dense_to_stencil
from oracle.dwf import DWF, inner, norm2
from oracle.solvers import DeflationSpace, adef2, cg, inverse_iteration_subspace, mirs


def _op(dims=(4, 4, 4, 4), Ls=4, mass=0.05, bc=(1.5, 0.5), eps=0.4, seed=0):
    U = sy.gauge_field(dims, eps, 300 + seed)
    return DWF(dims, Ls, 1.8, bc[0], bc[1], mass, U)


def test_cg_true_residual():
    d = _op()
    b = sy.gaussian_fermion(d.lat.dims, d.Ls, 1)
    x, it = cg(d.mdagm, b, 1e-10)
    assert np.sqrt(norm2(b - d.mdagm(x)) / norm2(b)) < 2e-10
    assert it > 5


def test_cg_free_field_plane_wave_exact_solution():
    """Free field: x = e^{ipx} (Mpc(p)^dag Mpc(p))^-1 e solves H x = e^{ipx} e."""
    from tests.test_oracle_dwf import _free_mpc_p
    dims, Ls = (4, 4, 6, 4), 4
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.03, sy.unit_gauge(dims))
    x4 = d.lat.coords[d.lat.sites[1]].astype(float)
    p = 2 * np.pi * np.array([1, 0, 2, 3]) / np.array(dims)
    e = np.random.default_rng(1).standard_normal((Ls, 4)) + 0j
    phase = np.exp(1j * x4 @ p)
    b = np.zeros(d.field_shape, dtype=np.complex128)
    b[:, :, :, 2] = phase[:, None, None] * e[None]
    Mp = _free_mpc_p(p, d.S)
    xe = np.linalg.solve(Mp.conj().T @ Mp, e.ravel()).reshape(Ls, 4)
    want = np.zeros_like(b)
    want[:, :, :, 2] = phase[:, None, None] * xe[None]
    x, _ = cg(d.mdagm, b, 1e-12)
    assert np.sqrt(norm2(x - want) / norm2(want)) < 1e-9


def test_mirs_single_iteration_closed_form_and_long_limit():
    d = _op(dims=(4, 2, 2, 2), Ls=2)
    r = sy.gaussian_fermion(d.lat.dims, d.Ls, 2)
    lam = 1.0
    Ar = d.mdagm(r) + lam * r
    x1 = mirs(d.mdagm, r, 1, lam)
    assert np.abs(x1 - (norm2(r) / inner(r, Ar).real) * r).max() < 1e-14
    # with as many iterations as the dimension, M_IRS is the exact shifted inverse
    n = int(np.prod(d.field_shape))
    xN = mirs(d.mdagm, r, n, lam)
    assert np.sqrt(norm2(d.mdagm(xN) + lam * xN - r) / norm2(r)) < 1e-9


def _tiny_deflation(coarse_tol=0.0):
    dims, Ls = (4, 2, 2, 2), 2
    d = _op(dims=dims, Ls=Ls, mass=0.1)
    bl = Blocking(d, (2, 2, 2, 2))
    phi = block_gram_schmidt(sy.gaussian_fermions(dims, Ls, 5, 3), bl)
    A = dense_to_stencil(coarse_dense_bruteforce(d.mdagm, phi, bl), bl)
    return d, bl, phi, DeflationSpace(phi, bl, A, coarse_tol=coarse_tol)


def test_projectors_block_form():
    """Sec. 2: in the basis (S-bar, S), P_R = [[1, 0], [-M_SS^-1 M_SSbar, 0]],
    P_L = [[1, -M_SbarS M_SS^-1], [0, 0]], Q H = 1 - P_R, P_L^dag = P_R."""
    d, bl, phi, D = _tiny_deflation()
    shape = d.field_shape
    n = int(np.prod(shape))
    Hm = np.zeros((n, n), dtype=np.complex128)
    Qm = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1
        Hm[:, j] = d.mdagm(e.reshape(shape)).ravel()
        Qm[:, j] = D.Q(e.reshape(shape)).ravel()
    cols = []
    for b, sites in enumerate(bl.sites_of_block):
        for k in range(phi.shape[0]):
            v = np.zeros(shape, dtype=np.complex128)
            v[sites] = phi[k, sites]
            cols.append(v.ravel())
    Phi = np.array(cols).T
    nS = Phi.shape[1]
    full, _ = np.linalg.qr(np.hstack([Phi, np.random.default_rng(0).standard_normal((n, n - nS))]))
    Psi = full[:, nS:]
    W = np.hstack([Psi, Phi])
    M = W.conj().T @ Hm @ W
    m = n - nS
    Mbb, Mbs, Msb, Mss = M[:m, :m], M[:m, m:], M[m:, :m], M[m:, m:]
    PR = np.zeros_like(M)
    PR[:m, :m] = np.eye(m)
    PR[m:, :m] = -np.linalg.solve(Mss, Msb)
    PL = np.zeros_like(M)
    PL[:m, :m] = np.eye(m)
    PL[:m, m:] = -Mbs @ np.linalg.inv(Mss)
    QH = W.conj().T @ Qm @ Hm @ W
    HQ = W.conj().T @ Hm @ Qm @ W
    assert np.abs(QH - (np.eye(n) - PR)).max() < 1e-11
    assert np.abs(HQ - (np.eye(n) - PL)).max() < 1e-11
    assert np.abs(PL.conj().T - PR).max() < 1e-11
    PLH = PL @ M
    assert np.abs(PLH - PLH.conj().T).max() < 1e-10 * np.abs(M).max()
    assert np.abs(Qm @ Hm @ Qm - Qm).max() < 1e-11 * np.abs(Qm).max()


def test_adef2_exact_Q_invariants_and_solution():
    d = _op(dims=(8, 4, 4, 4), Ls=4, mass=0.02)
    bl = Blocking(d, (4, 4, 4, 4))
    phi = block_gram_schmidt(sy.gaussian_fermions(d.lat.dims, d.Ls, 7, 4), bl)
    A = dense_to_stencil(coarse_dense_bruteforce(d.mdagm, phi, bl), bl)
    D = DeflationSpace(phi, bl, A, coarse_tol=0.0)
    b = sy.gaussian_fermion(d.lat.dims, d.Ls, 8)
    res = adef2(d.mdagm, b, D, 1e-10, track_invariants=True)
    assert res.true_residual < 2e-10
    qr, hqr = np.array(res.invariants).T
    assert qr.max() < 1e-9      # Q r_k = 0
    assert hqr.max() < 1e-9     # P_L r_k = r_k
    xs, _ = cg(d.mdagm, b, 1e-12)
    assert np.sqrt(norm2(res.x - xs) / norm2(xs)) < 1e-7


@pytest.fixture(scope="module")
def two_level():
    d = _op(dims=(8, 8, 4, 4), Ls=4, mass=0.01)
    bl = Blocking(d, (4, 4, 4, 4))
    phi = inverse_iteration_subspace(d.mdagm, sy.gaussian_fermions(d.lat.dims, d.Ls, 9, 6), bl,
                                     steps=2, tol=1e-3)
    A = dense_to_stencil(coarse_dense_bruteforce(d.mdagm, phi, bl), bl)
    b = sy.gaussian_fermion(d.lat.dims, d.Ls, 10)
    hist = []
    cg(d.mdagm, b, 1e-8, history=hist)
    xs, _ = cg(d.mdagm, b, 1e-12)
    return d, bl, phi, A, b, len(hist), xs


@pytest.mark.parametrize("flexible", [True, False])
def test_adef2_inexact_coarse_solve_converges(two_level, flexible):
    """Table optimised: coarse residual 0.04 inside the solver, M_IRS(7, 1.0)."""
    d, bl, phi, A, b, cg_iters, xs = two_level
    D = DeflationSpace(phi, bl, A, coarse_tol=0.04)
    res = adef2(d.mdagm, b, D, 1e-8, flexible=flexible)
    assert res.true_residual < 2e-8
    assert res.iterations < cg_iters
    assert np.sqrt(norm2(res.x - xs) / norm2(xs)) < 1e-5


def test_inverse_iteration_enriches_low_modes():
    d = _op(dims=(8, 4, 4, 4), Ls=4, mass=0.01)
    bl = Blocking(d, (4, 4, 4, 4))
    noise = sy.gaussian_fermions(d.lat.dims, d.Ls, 11, 3)
    phi = inverse_iteration_subspace(d.mdagm, noise, bl, steps=2, tol=1e-3)
    for sites in bl.sites_of_block:
        X = phi[:, sites].reshape(3, -1)
        assert np.abs(np.conj(X) @ X.T - np.eye(3)).max() < 1e-13
    rq_phi = [inner(v, d.mdagm(v)).real / norm2(v) for v in phi]
    rq_noise = [inner(v, d.mdagm(v)).real / norm2(v) for v in noise]
    assert max(rq_phi) < 0.05 * min(rq_noise)


def _dense_H(d):
    """H as a dense matrix, one oracle apply per unit vector."""
    shape = d.field_shape
    n = int(np.prod(shape))
    Hm = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[j] = 1.0
        Hm[:, j] = d.mdagm(e.reshape(shape)).ravel()
        e[j] = 0.0
    return Hm


def _block_qr(V, bl, shape):
    """Per block, the Q factor of numpy's QR of the block pieces with the
    diagonal of R made real positive (the unique such factorisation)."""
    out = np.zeros_like(V)
    W = V.reshape((V.shape[0],) + shape)
    O = out.reshape((V.shape[0],) + shape)
    for sites in bl.sites_of_block:
        X = W[:, sites].reshape(V.shape[0], -1).T
        Q, R = np.linalg.qr(X)
        ph = np.diag(R) / np.abs(np.diag(R))
        O[:, sites] = (Q * ph).T.reshape((V.shape[0], len(sites)) + shape[1:])
    return out


@pytest.mark.parametrize("shift", [0.0, 0.3])
def test_inverse_iteration_subspace_is_dense_inverse_iteration(shift):
    """Pin: two steps of phi <- blockQR((H + shift)^-1 phi) with H assembled
    densely, numpy's linear solve and numpy's QR per block (4x4x2x2 lattice,
    Ls 2, 2^4 blocks).  A dropped shift or sign, a skipped orthonormalisation or
    a wrong block assignment all fail."""
    dims, Ls = (4, 4, 2, 2), 2
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.1, sy.gauge_field(dims, 0.4, 330))
    bl = Blocking(d, (2, 2, 2, 2))
    noise = sy.gaussian_fermions(dims, Ls, 331, 3)
    Hm = _dense_H(d) + shift * np.eye(int(np.prod(d.field_shape)))
    V = noise.reshape(3, -1)
    for _ in range(2):
        V = np.linalg.solve(Hm, V.T).T
        V = _block_qr(V, bl, d.field_shape)
    got = inverse_iteration_subspace(d.mdagm, noise, bl, steps=2, shift=shift, tol=1e-14)
    assert np.abs(got.reshape(3, -1) - V).max() < 1e-9
    if shift:
        other = inverse_iteration_subspace(d.mdagm, noise, bl, steps=2, shift=-shift / 2, tol=1e-14)
        assert np.abs(other.reshape(3, -1) - V).max() > 1e-3


def test_cg_kappa_on_a_diagonal_operator():
    """The Lanczos tridiagonal of CG's coefficients recovers lambda_max /
    lambda_min of a diagonal operator with known spectrum."""
    from tests.gpu_util import cg_kappa
    lam = np.linspace(0.01, 5.0, 400)
    b = sy.complex_normal(332, (400,))
    x, k = cg_kappa(lambda v: lam * v, b, 1e-13)
    assert abs(k - 500.0) < 1e-6 * 500
    assert np.abs(x - b / lam).max() < 1e-9
