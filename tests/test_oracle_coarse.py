"""Pins of the oracle's blocked subspace and little Dirac operator (no GPU)."""
import numpy as np
import pytest

import synthetic as sy
from oracle.coarse import (Blocking, block_gram_schmidt, canonical_offsets, coarse_apply,
                           coarse_dense_bruteforce, coarse_fourier, dense_to_stencil,
                           prolong, restrict, stencil_offsets, stencil_to_dense)
from oracle.dwf import DWF


def _setup(dims, Ls, block, nvec, seed=0, bc=(1.5, 0.5), mass=0.05, eps=0.5):
    U = sy.gauge_field(dims, eps, 100 + seed)
    d = DWF(dims, Ls, 1.8, bc[0], bc[1], mass, U)
    bl = Blocking(d, block)
    phi = block_gram_schmidt(sy.gaussian_fermions(dims, Ls, 200 + seed, nvec), bl)
    return d, bl, phi


def test_stencil_hop_counts(golden):
    offs = stencil_offsets()
    assert offs.shape == (81, 4)
    assert len({tuple(o) for o in offs}) == 81
    assert tuple(offs[40]) == (0, 0, 0, 0)
    hops = np.abs(offs).sum(axis=1)
    cum = [int((hops <= h).sum()) for h in range(5)]
    assert cum == golden["coarse_terms_by_hop_cumulative"]["value"]
    assert 81 - 1 == golden["coarse_stencil_neighbours"]["value"]
    assert cum[1] == golden["truncated_coarse_terms"]["value"]


def test_block_gram_schmidt_orthonormal_and_span():
    dims, Ls, block, nvec = (8, 4, 4, 4), 4, (4, 4, 4, 4), 5
    U = sy.gauge_field(dims, 0.5, 1)
    d = DWF(dims, Ls, 1.8, 1.0, 0.0, 0.05, U)
    bl = Blocking(d, block)
    raw = sy.gaussian_fermions(dims, Ls, 2, nvec)
    phi = block_gram_schmidt(raw, bl)
    for sites in bl.sites_of_block:
        X = phi[:, sites].reshape(nvec, -1)
        G = np.conj(X) @ X.T
        assert np.abs(G - np.eye(nvec)).max() < 1e-14
        Y = raw[:, sites].reshape(nvec, -1)
        # span unchanged: the original vectors are reproduced by their projections
        proj = (Y @ np.conj(X).T) @ X
        assert np.abs(proj - Y).max() < 1e-12 * np.abs(Y).max()
        # triangular: phi_k lies in span(raw_0..raw_k)
        for k in range(nvec):
            coef = np.linalg.lstsq(Y[:k + 1].T, X[k], rcond=None)[0]
            assert np.abs(Y[:k + 1].T @ coef - X[k]).max() < 1e-12


def test_restrict_prolong_adjoint():
    d, bl, phi = _setup((8, 8, 4, 4), 4, (4, 4, 4, 4), 3)
    v = sy.gaussian_fermion(d.lat.dims, d.Ls, 9)
    c = sy.coarse_gaussian(bl.Vc, 3, 10)
    assert np.vdot(c, restrict(phi, v, bl)) == pytest.approx(np.vdot(prolong(phi, c, bl), v), rel=1e-13)
    assert np.abs(restrict(phi, prolong(phi, c, bl), bl) - c).max() < 1e-13


@pytest.mark.parametrize("dims", [(8, 8, 4, 4), (16, 4, 4, 4), (12, 4, 4, 4)])
def test_stencil_apply_equals_RHP(dims):
    """The 81-point stencil apply of A reproduces R H P c on every coarse lattice,
    including aliased extents (1, 2) and extent >= 3."""
    d, bl, phi = _setup(dims, 4, (4, 4, 4, 4), 3)
    Ad = coarse_dense_bruteforce(d.mdagm, phi, bl)
    A = dense_to_stencil(Ad, bl)
    c = sy.coarse_gaussian(bl.Vc, 3, 11)
    want = restrict(phi, d.mdagm(prolong(phi, c, bl)), bl)
    assert np.abs(coarse_apply(A, c, bl) - want).max() < 1e-12 * np.abs(want).max()
    assert np.abs(stencil_to_dense(A, bl) - Ad).max() < 1e-13 * np.abs(Ad).max()
    # Hermitian positive definite
    n = bl.Vc * 3
    M = Ad.reshape(n, n)
    assert np.abs(M - M.conj().T).max() < 1e-12 * np.abs(M).max()
    assert np.linalg.eigvalsh(M).min() > 0


def test_coupling_vanishes_beyond_one_block_hop():
    """Sec. 5.1: blocks of 4^4 couple only to blocks one hop away per direction."""
    d, bl, phi = _setup((16, 4, 4, 4), 4, (4, 4, 4, 4), 2)
    Ad = coarse_dense_bruteforce(d.mdagm, phi, bl)
    scale = np.abs(Ad).max()
    for a in range(bl.Vc):
        for b in range(bl.Vc):
            sep = abs(bl.block_coords[a][0] - bl.block_coords[b][0])
            sep = min(sep, 4 - sep)
            if sep >= 2:
                assert np.abs(Ad[a, :, b, :]).max() < 1e-14 * scale
            else:
                assert np.abs(Ad[a, :, b, :]).max() > 1e-6 * scale


def test_stencil_hermitian_pairs_unaliased():
    """A^{a, a+l} = (A^{a+l, a})^dag in stencil form when no extent aliases."""
    d, bl, phi = _setup((12, 12, 4, 4), 2, (4, 4, 4, 4), 2)
    assert bl.coarse_dims == (3, 3, 1, 1)
    A = dense_to_stencil(coarse_dense_bruteforce(d.mdagm, phi, bl), bl)
    offs = stencil_offsets()
    keep = [canonical_offsets(bl.coarse_dims, mu) for mu in range(4)]
    for l in range(81):
        if not all(offs[l, mu] in keep[mu] for mu in range(4)):
            assert np.abs(A[:, l]).max() == 0.0
            continue
        lm = 80 - l
        for a in range(bl.Vc):
            b = bl.neighbour_block(a, offs[l])
            assert np.abs(A[a, l] - A[b, lm].conj().T).max() < 1e-12 * np.abs(A).max()


@pytest.mark.parametrize("dims,block", [((12, 12, 4, 4), (4, 4, 4, 4)),
                                        ((8, 12, 4, 4), (4, 4, 4, 4)),
                                        ((12, 4, 12, 8), (4, 4, 4, 4))])
def test_fourier_trick_equals_bruteforce(dims, block):
    d, bl, phi = _setup(dims, 2, block, 2, seed=3)
    Ab = dense_to_stencil(coarse_dense_bruteforce(d.mdagm, phi, bl), bl)
    Af = coarse_fourier(d.mdagm, phi, bl)
    assert np.abs(Af - Ab).max() < 1e-11 * np.abs(Ab).max()


def test_fourier_trick_full_81_point_stencil():
    """All four coarse extents >= 3: the 81 momenta of Sec. 5.1.1."""
    d, bl, phi = _setup((12, 12, 12, 12), 2, (4, 4, 4, 4), 1, seed=4, bc=(1.0, 0.0))
    assert bl.coarse_dims == (3, 3, 3, 3)
    Af = coarse_fourier(d.mdagm, phi, bl)
    # compare a few brute-force columns: A[a, l, :, 0] for the block b = a + delta_l
    offs = stencil_offsets()
    for b in (0, 17, 40, 80):
        v = np.zeros(phi.shape[1:], dtype=np.complex128)
        sites = bl.sites_of_block[b]
        v[sites] = phi[0, sites]
        col = restrict(phi, d.mdagm(v), bl)      # <phi_j^a | H | phi_0^b> for all a
        for l in range(81):
            a = bl.neighbour_block(b, -offs[l])  # a + delta_l = b
            assert abs(Af[a, l, 0, 0] - col[a, 0]) < 1e-11 * np.abs(Af).max()
