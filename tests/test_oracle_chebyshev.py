"""Pins of the oracle's high-mode preconditioner for the A-DEF1 coarse solver
(Sec. 5.2, "Truncated little Dirac operator as preconditioner"; Table
hierarchy: a Chebyshev approximation of order 16 to 1/x on [0.5, 45] applied
to the 0- and 1-hop truncation Q_trunc of the little Dirac operator).  No GPU.

What fixes them, independently of the oracle's own code:
* the residual polynomial 1 - x p(x) of the order-n Chebyshev approximation is
  T_n((theta - x)/delta) / T_n(theta/delta), evaluated here with numpy's
  Chebyshev series (a different evaluation than the oracle's recurrence);
* on a Hermitian matrix with spectrum in [lo, hi] that gives
  |r - M p(M) r| <= |r| / T_n(theta/delta), with T_n(s) = cosh(n acosh s);
* the truncation keeps the 9 offsets of taxicab length <= 1 and zeroes the
  couplings between blocks two or more hops apart, where the hop count comes
  from the blocks' coordinates; a Hermitian stencil stays Hermitian;
* A-DEF1 with the preconditioner reaches numpy's dense solution.
"""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as C

import synthetic as sy
from oracle.coarse import Blocking, coarse_apply, dense_to_stencil, stencil_to_dense
from oracle.dwf import DWF, norm2
from oracle.solvers import adef1, cg, chebyshev_inverse, ldop_deflation_space, qtrunc_chebyshev, truncate_stencil


def _scalar_p(x, order, lo, hi):
    """p(x) from the oracle, applied to a diagonal matrix."""
    return chebyshev_inverse(lambda v: x * v, np.ones_like(x), order, lo, hi)


def _residual_closed_form(x, order, lo, hi):
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    Tn = C.Chebyshev.basis(order)
    return Tn((theta - x) / delta) / Tn(theta / delta)


@pytest.mark.parametrize("order", [1, 2, 3, 7, 16])
@pytest.mark.parametrize("lo,hi", [(0.5, 45.0), (0.01, 2.0)])
def test_residual_polynomial_is_scaled_chebyshev(order, lo, hi):
    x = np.concatenate([np.linspace(-1.0, 1.2 * hi, 301), [lo, hi]])
    p = _scalar_p(x, order, lo, hi)
    want = _residual_closed_form(x, order, lo, hi)
    assert np.abs((1 - x * p) - want).max() < 1e-12 * max(1.0, np.abs(want).max())


def test_order_one_is_the_midpoint_reciprocal_and_order_two_is_linear():
    x = np.linspace(0.1, 5.0, 7)
    lo, hi = 0.5, 4.5
    assert np.allclose(_scalar_p(x, 1, lo, hi), 1 / 2.5, rtol=0, atol=1e-15)
    p2 = _scalar_p(x, 2, lo, hi)
    assert np.abs(np.diff(p2, 2)).max() < 1e-13       # degree one
    # 1 - x p(x) = T_2(...) / T_2(sigma) vanishes at the Chebyshev nodes of T_2
    theta, delta = 2.5, 2.0
    nodes = theta - delta * np.cos(np.pi / 4 * np.array([1, 3]))
    assert np.abs(1 - nodes * _scalar_p(nodes, 2, lo, hi)).max() < 1e-13


def test_paper_parameters_positive_and_bounded():
    """Order 16 on [0.5, 45]: p > 0 on (0, 45] (a positive definite
    preconditioner), |1 - x p(x)| <= 1/T_16(sigma) on [0.5, 45], and
    0 <= 1 - x p(x) < 1 below 0.5 (modes under the infra-red edge are damped
    less, never amplified)."""
    lo, hi, n = 0.5, 45.0, 16
    x = np.linspace(1e-4, hi, 20001)
    p = _scalar_p(x, n, lo, hi)
    assert np.all(p > 0)
    sigma = (hi + lo) / (hi - lo)
    bound = 1 / np.cosh(n * np.arccosh(sigma))
    inside = x >= lo
    assert np.abs(1 - x[inside] * p[inside]).max() <= bound * (1 + 1e-9)
    below = (1 - x * p)[~inside]
    assert np.all(below >= 0) and np.all(below < 1)


def test_matrix_bound_on_hermitian_spectrum():
    n, lo, hi, order = 40, 0.3, 12.0, 9
    U, _ = np.linalg.qr(sy.complex_normal(1300, (n, n)))
    ev = np.linspace(lo, hi, n)
    H = (U * ev) @ U.conj().T
    r = sy.complex_normal(1301, (n,))
    y = chebyshev_inverse(lambda v: H @ v, r, order, lo, hi)
    sigma = (hi + lo) / (hi - lo)
    res = np.linalg.norm(r - H @ y) / np.linalg.norm(r)
    assert res <= 1 / np.cosh(order * np.arccosh(sigma)) * (1 + 1e-9)
    # same result as the polynomial applied through the eigenbasis
    pe = _scalar_p(ev, order, lo, hi)
    assert np.abs(y - (U * pe) @ (U.conj().T @ r)).max() < 1e-12 * np.abs(y).max()


def test_chebyshev_argument_errors():
    r = np.ones(3)
    for order, lo, hi in [(0, 0.5, 45.0), (4, 0.0, 1.0), (4, 2.0, 1.0)]:
        with pytest.raises(ValueError):
            chebyshev_inverse(lambda v: v, r, order, lo, hi)


@pytest.fixture(scope="module")
def full_stencil():
    """Random Hermitian 81-point stencil on coarse grid 3^4 (no aliased
    offsets), Nvec 2."""
    dims = (12, 12, 12, 12)
    bl = Blocking(DWF(dims, 2, 1.8, 1.0, 0.0, 0.1, sy.unit_gauge(dims)), (4, 4, 4, 4))
    A0 = sy.complex_normal(1310, (bl.Vc, 81, 2, 2))
    D = stencil_to_dense(A0, bl)
    H = D + D.conj().transpose(2, 3, 0, 1)
    return bl, dense_to_stencil(H, bl), H


def test_truncation_keeps_nearest_neighbour_blocks(full_stencil):
    bl, A, H = full_stencil
    T = truncate_stencil(A)
    kept = np.nonzero(np.abs(T).reshape(bl.Vc, 81, -1).max(axis=(0, 2)))[0]
    assert len(kept) == 9
    # hop distance between blocks from their coordinates (extent 3: 0 or 1 per axis)
    bc = bl.block_coords
    hops = (bc[:, None, :] != bc[None, :, :]).sum(axis=2)
    Td = stencil_to_dense(T, bl)
    near = np.broadcast_to((hops <= 1)[:, None, :, None], Td.shape)
    assert np.array_equal(Td[near], H[near])
    assert np.all(Td[~near] == 0)
    Tn = Td.reshape(bl.Vc * 2, -1)
    assert np.abs(Tn - Tn.conj().T).max() == 0
    # truncating at four hops keeps everything
    assert np.array_equal(truncate_stencil(A, 4), A)


@pytest.fixture(scope="module")
def ldop(little_dirac_12x12x4x4):
    d, bl, phi, A, Dn, lam = little_dirac_12x12x4x4
    return bl, A, Dn


def test_preconditioner_is_hermitian_positive_definite(ldop):
    bl, A, Dn = ldop
    n = Dn.shape[0]
    Tn = stencil_to_dense(truncate_stencil(A), bl).reshape(n, n)
    hi = 1.1 * np.linalg.eigvalsh(Tn)[-1]
    M = qtrunc_chebyshev(A, bl, 16, 0.5, hi)
    Md = np.stack([M(e.reshape(bl.Vc, 4)).ravel() for e in np.eye(n, dtype=np.complex128)], axis=1)
    assert np.abs(Md - Md.conj().T).max() < 1e-12 * np.abs(Md).max()
    assert np.linalg.eigvalsh(Md).min() > 0
    # the explicit infra-red shift acts on Q_trunc before the polynomial
    Ms = qtrunc_chebyshev(A, bl, 5, 0.5, hi + 1.0, shift=1.0)
    r = sy.coarse_gaussian(bl.Vc, 4, 1320)
    want = chebyshev_inverse(lambda v: (Tn @ v.ravel() + v.ravel()).reshape(v.shape), r, 5, 0.5, hi + 1.0)
    assert np.abs(Ms(r) - want).max() < 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("flexible", [True, False])
def test_adef1_with_chebyshev_qtrunc_converges_faster(ldop, flexible):
    """Table hierarchy's coarse solver: A-DEF1 with second-level deflation and
    the order-16 Chebyshev of Q_trunc reaches the dense solution in fewer
    iterations than with M = 1 (16 on this operator)."""
    bl, A, Dn = ldop
    n = Dn.shape[0]
    Z, AZ, lam = ldop_deflation_space(A, bl, sy.complex_normal(1230, (8, bl.Vc, 4)), steps=3, tol=1e-10)
    b = sy.coarse_gaussian(bl.Vc, 4, 1231)
    xs = np.linalg.solve(Dn, b.ravel()).reshape(b.shape)

    def apply_A(v):
        return coarse_apply(A, v, bl)

    x1, it1 = adef1(apply_A, b, Z, AZ, lam, 1e-10, flexible=flexible)
    Tn = stencil_to_dense(truncate_stencil(A), bl).reshape(n, n)
    M = qtrunc_chebyshev(A, bl, 16, 0.5, 1.1 * np.linalg.eigvalsh(Tn)[-1])
    x, it = adef1(apply_A, b, Z, AZ, lam, 1e-10, flexible=flexible, M=M)
    assert np.sqrt(norm2(x - xs) / norm2(xs)) < 1e-8
    assert it < it1 / 2


def test_empty_deflation_space_is_preconditioned_cg(ldop):
    """With no deflation vectors A-DEF1 is CG preconditioned by M: the dense
    solution in fewer iterations than plain CG, and with M = 1 exactly CG's
    iterates."""
    bl, A, Dn = ldop
    n = Dn.shape[0]
    b = sy.coarse_gaussian(bl.Vc, 4, 1330)
    xs = np.linalg.solve(Dn, b.ravel()).reshape(b.shape)

    def apply_A(v):
        return coarse_apply(A, v, bl)

    Z0 = np.zeros((0, bl.Vc, 4), dtype=np.complex128)
    Tn = stencil_to_dense(truncate_stencil(A), bl).reshape(n, n)
    M = qtrunc_chebyshev(A, bl, 16, 0.05, 1.1 * np.linalg.eigvalsh(Tn)[-1])
    x, it = adef1(apply_A, b, Z0, Z0, np.zeros(0), 1e-10, M=M)
    assert np.sqrt(norm2(x - xs) / norm2(xs)) < 1e-8
    x1, it1 = adef1(apply_A, b, Z0, Z0, np.zeros(0), 1e-10, flexible=False)
    xc, itc = cg(apply_A, b, 1e-10)
    assert it1 == itc and np.abs(x1 - xc).max() < 1e-10 * np.abs(xc).max()
    assert it < itc
