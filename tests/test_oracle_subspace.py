"""Pins of the oracle's rational-filter subspace generation (Sec. 4.2, Eq.
ratfilt, Table FineSubspaceParams).  No GPU.

What fixes them, independently of the oracle's own code:
* the partial fractions against the product prod_i 1/(x + sigma_i) at
  sample points (closed form);
* multi-shift solutions against numpy's dense solves of every shifted
  system, and with a single shift the textbook CG, iterate by iterate;
* the filter against the eigendecomposition of a dense Hermitian matrix
  (numpy's eigh);
* the support and chirality of the wall noise (gamma_5 eigenvalues);
* the filtered subspace of a domain wall operator concentrating on its low
  end of the spectrum (Rayleigh quotients far below those of the noise).
"""
import numpy as np
import pytest

import synthetic as sy
from oracle.coarse import Blocking
from oracle.dwf import DWF, gamma_matrices
from oracle.solvers import cg
from oracle.subspace import (multishift_cg, promote, rational_filter, rational_filter_shifts, rational_subspace,
                             surface_truncate, two_pass_subspace, wall_noise)


def _hpd(n, seed, lo=1e-3, hi=10.0):
    U, _ = np.linalg.qr(sy.complex_normal(seed, (n, n)))
    ev = np.geomspace(lo, hi, n)
    return (U * ev) @ U.conj().T, ev, U


@pytest.mark.parametrize("lam,eps", [(0.0003, 0.0001), (0.5, 0.25), (1e-2, 1e-2)])
def test_partial_fractions(lam, eps):
    sig, c = rational_filter_shifts(lam, eps)
    assert sig == pytest.approx([lam, lam + eps, lam + 2 * eps, lam + 3 * eps])
    for x in [0.0, 1e-4, 0.01, 1.0, 37.0]:
        prod = 1.0 / np.prod([x + s for s in sig])
        terms = [ci / (x + si) for ci, si in zip(c, sig)]
        # the weights grow like eps^-3, so the sum cancels: its rounding error is
        # bounded by a few ulps of the largest term (the filter's high-mode
        # response is then tiny in absolute terms, far below its low-mode one)
        assert abs(sum(terms) - prod) <= 1e-15 * max(abs(t) for t in terms) * 8


def test_multishift_solves_every_shifted_system():
    H, ev, U = _hpd(60, 1700)
    b = sy.complex_normal(1701, (60,))
    shifts = [0.3, 0.0, 1e-2, 2.0]
    xs, it = multishift_cg(lambda v: H @ v, b, shifts, 1e-12)
    for s, x in zip(shifts, xs):
        want = np.linalg.solve(H + s * np.eye(60), b)
        assert np.linalg.norm(x - want) <= 1e-8 * np.linalg.norm(want)
        assert np.linalg.norm(b - (H @ x + s * x)) <= 1e-10 * np.linalg.norm(b)
    # the base system (the smallest shift) runs exactly the textbook CG
    _, itc = cg(lambda v: H @ v, b, 1e-12)
    assert it == itc


def test_single_shift_is_textbook_cg():
    H, ev, U = _hpd(40, 1702, lo=0.05)
    b = sy.complex_normal(1703, (40,))
    for n in [1, 3, 10]:
        xs, it = multishift_cg(lambda v: H @ v, b, [0.0], 0.0, maxiter=n)
        xc, itc = cg(lambda v: H @ v, b, 0.0, maxiter=n)
        assert it == itc == n
        assert np.abs(xs[0] - xc).max() < 1e-12 * np.abs(xc).max()


def test_filter_against_eigendecomposition():
    H, ev, U = _hpd(50, 1704, lo=1e-4, hi=5.0)
    eta = sy.complex_normal(1705, (50,))
    lam, eps = 3e-4, 1e-4
    phi = rational_filter(lambda v: H @ v, eta, lam, eps, 1e-13)
    resp = 1.0 / np.prod([ev + lam + i * eps for i in range(4)], axis=0)
    want = U @ (resp * (U.conj().T @ eta))
    assert np.linalg.norm(phi - want) <= 1e-7 * np.linalg.norm(want)
    # a fourth-order low-pass filter: x^4 times the response tends to 1
    assert abs(resp[-1] * ev[-1] ** 4 - 1) < 6 * (lam + 3 * eps) / ev[-1]


def test_wall_noise_support_and_chirality():
    n4, Ls = 10, 6
    eta = wall_noise(n4, Ls, 3, 1706)
    assert eta.shape == (3, n4, Ls, 4, 3)
    assert np.all(eta[:, :, 1:Ls - 1] == 0)
    _, g5 = gamma_matrices()
    # s = 0 holds gamma_5 = -1 components only, s = Ls - 1 gamma_5 = +1 only
    assert np.allclose(np.einsum("ab,kxbc->kxac", g5, eta[:, :, 0]), -eta[:, :, 0])
    assert np.allclose(np.einsum("ab,kxbc->kxac", g5, eta[:, :, Ls - 1]), eta[:, :, Ls - 1])
    xi = sy.complex_normal(1706, (3, n4, 4, 3))
    assert np.allclose(eta[:, :, 0] + eta[:, :, Ls - 1], xi)


def test_surface_truncation():
    phi = sy.complex_normal(1707, (2, 5, 8, 4, 3))
    t = surface_truncate(phi, 2)
    assert np.array_equal(t[:, :, :2], phi[:, :, :2]) and np.array_equal(t[:, :, 6:], phi[:, :, 6:])
    assert np.all(t[:, :, 2:6] == 0)
    assert np.array_equal(surface_truncate(phi, 4), phi)


def test_rational_subspace_concentrates_on_low_modes():
    """Domain wall operator 8x4x4x4, Ls 4: the filtered vectors' Rayleigh
    quotients lie far below those of the wall noise and of Gaussian vectors."""
    dims, Ls = (8, 4, 4, 4), 4
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.02, sy.gauge_field(dims, 0.4, 1708))
    bl = Blocking(d, (4, 4, 4, 4))
    phi = rational_subspace(d.mdagm, bl, 4, 1709, lam=0.05, eps=0.02, tol=1e-6)
    def rq(v):
        return np.vdot(v, d.mdagm(v)).real / np.vdot(v, v).real
    q_phi = max(rq(v) for v in phi)
    q_noise = min(rq(v) for v in wall_noise(d.lat.V // 2, Ls, 4, 1709))
    q_gauss = min(rq(v) for v in sy.gaussian_fermions(dims, Ls, 1710, 4))
    assert q_phi < 0.1 * q_noise and q_phi < 0.1 * q_gauss


def test_promote_places_the_surfaces():
    phi = sy.complex_normal(1711, (2, 5, 4, 4, 3))
    out = promote(phi, 10)
    assert out.shape == (2, 5, 10, 4, 3)
    assert np.array_equal(out[:, :, :2], phi[:, :, :2])
    assert np.array_equal(out[:, :, 8:], phi[:, :, 2:])
    assert np.all(out[:, :, 2:8] == 0)
    odd = sy.complex_normal(1712, (5, 3, 4, 3))
    o2 = promote(odd, 7)          # Ls1 = 3: slices 0, 1 near the first wall, 2 at the last
    assert np.array_equal(o2[:, :2], odd[:, :2]) and np.array_equal(o2[:, 6], odd[:, 2])
    assert np.all(o2[:, 2:6] == 0)
    assert np.array_equal(promote(phi, 4), phi)
    with pytest.raises(ValueError):
        promote(phi, 3)


@pytest.fixture(scope="module")
def dwf8():
    dims, Ls = (8, 4, 4, 4), 6
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.02, sy.gauge_field(dims, 0.4, 1713))
    return d, Blocking(d, (4, 4, 4, 4))


def test_two_pass_without_refinement_at_full_ls_is_the_single_pass():
    dims = (8, 4, 4, 4)
    d = DWF(dims, 4, 1.8, 1.5, 0.5, 0.02, sy.gauge_field(dims, 0.4, 1713))
    bl = Blocking(d, (4, 4, 4, 4))
    a = two_pass_subspace(d, bl, 2, 1714, d.Ls, d.mass, 0.05, 0.02, 1e-8)
    b = rational_subspace(d.mdagm, bl, 2, 1714, 0.05, 0.02, tol=1e-8)
    assert np.abs(a - b).max() < 1e-12


def test_two_pass_refined_subspace(dwf8):
    """First pass at Ls 4 with a heavier mass, promotion to Ls 6, one deflated
    shifted inversion per vector: the vectors concentrate on the low end
    (Rayleigh quotients well below those of Gaussian vectors) and on the walls."""
    d, bl = dwf8
    phi = two_pass_subspace(d, bl, 2, 1715, 4, 0.05, 0.05, 0.02, 1e-6, lam2=1e-3, tol2=1e-3, mirs_iter=4)
    def rq(v):
        return np.vdot(v, d.mdagm(v)).real / np.vdot(v, v).real
    q_phi = max(rq(v) for v in phi)
    q_gauss = min(rq(v) for v in sy.gaussian_fermions(d.lat.dims, d.Ls, 1716, 2))
    assert q_phi < 0.1 * q_gauss
    w = np.sqrt((np.abs(phi) ** 2).sum(axis=(1, 3, 4)))   # (nvec, Ls) weight per s-slice
    assert np.all(w[:, [0, -1]].sum(axis=1) > w[:, 2:4].sum(axis=1))


def test_second_pass_coarse_operator_is_shifted_by_lam2():
    """The reading behind the second pass: for block-orthonormal vectors the
    coarse operator of H + lam2 is that of H plus lam2 on the diagonal blocks
    (P^dag P = 1), which is how the second pass builds it."""
    from oracle.coarse import block_gram_schmidt, coarse_dense_bruteforce
    dims, Ls, lam2 = (8, 4, 4, 4), 4, 1e-3
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.02, sy.gauge_field(dims, 0.4, 1717))
    bl = Blocking(d, (4, 4, 4, 4))
    basis = block_gram_schmidt(sy.gaussian_fermions(dims, Ls, 1718, 3), bl)
    A = coarse_dense_bruteforce(d.mdagm, basis, bl)
    As = coarse_dense_bruteforce(lambda v: d.mdagm(v) + lam2 * v, basis, bl)
    eye = np.einsum("ab,jk->ajbk", np.eye(bl.Vc), np.eye(3))
    assert np.abs(As - (A + lam2 * eye)).max() < 1e-12 * np.abs(A).max()


def test_promotion_keeps_block_orthonormality():
    """Promotion moves whole s-slices without dropping any, so a block-orthonormal
    Ls1 subspace stays block-orthonormal in Ls (Gram-Schmidt leaves it unchanged)."""
    from oracle.coarse import block_gram_schmidt
    dims = (8, 4, 4, 4)
    d1 = DWF(dims, 4, 1.8, 1.5, 0.5, 0.05, sy.gauge_field(dims, 0.4, 1719))
    d = DWF(dims, 8, 1.8, 1.5, 0.5, 0.01, d1.U)
    phi1 = block_gram_schmidt(sy.gaussian_fermions(dims, 4, 1720, 3), Blocking(d1, (4, 4, 4, 4)))
    v = promote(phi1, 8)
    assert np.abs(block_gram_schmidt(v, Blocking(d, (4, 4, 4, 4))) - v).max() < 1e-13
