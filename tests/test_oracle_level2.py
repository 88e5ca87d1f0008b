"""Pins of the oracle's blocked second coarsening (three-level HDCG; the
construction of Sec. 2 applied to the little Dirac operator).  No GPU.

What fixes them, independently of the oracle's own code:
* the level-2 blocking against a coordinate walk of the coarse lattice;
* orthonormal block pieces, the same span as the start vectors, R2 = P2^dag;
* the level-2 stencil against the dense Galerkin product P2^dag A P2 formed
  from explicit matrices (numpy), which also shows that nothing couples
  blocks two or more hops apart;
* Galerkin bounds: P2 has orthonormal columns, so the spectrum of A2 lies
  inside [lambda_min(A), lambda_max(A)] (Rayleigh quotients), and A2 is
  Hermitian positive definite;
* the deflated level-1 solve meets numpy's dense solution with the A-DEF2
  invariant Q2 r_k = 0 (exact Q2), in fewer iterations than CG;
* the three-level solve of a domain wall problem meets CG's solution.
"""
import itertools

import numpy as np
import pytest

import synthetic as sy
from oracle.coarse import (Blocking, block_gram_schmidt, coarse_apply, coarse_dense_bruteforce, dense_to_stencil,
                           prolong, restrict, stencil_offsets, stencil_to_dense)
from oracle.dwf import DWF, norm2
from oracle.level2 import CoarseBlocking
from oracle.solvers import DeflationSpace, adef2, cg, inverse_iteration_subspace


def _decaying_hpd(lat, n, seed, lam_min=0.02, decay=0.15):
    """Seeded HPD 81-point stencil on the coarse lattice `lat` (a
    CoarseBlocking with unit blocks): couplings falling by `decay` per hop
    (Table frobnorm), K on offset l and K^dag on -l, diagonal shifted so that
    the lowest eigenvalue is lam_min."""
    K = sy.complex_normal(seed, (lat.Vc, 81, n, n)) / np.sqrt(n)
    offs = stencil_offsets()
    hops = np.abs(offs).sum(axis=1)
    A = np.zeros_like(K)
    sites = np.arange(lat.Vc)
    for l in range(81):
        if l == 40:
            continue
        b = lat.neighbour_block(sites, offs[l])      # a translation: a permutation of the sites
        k = K[:, l] * decay ** hops[l]
        A[:, l] += k
        A[b, 80 - l] += k.conj().transpose(0, 2, 1)
    D = stencil_to_dense(A, lat).reshape(lat.Vc * n, -1)
    A[:, 40] += (lam_min - np.linalg.eigvalsh(D)[0]) * np.eye(n)
    return dense_to_stencil(stencil_to_dense(A, lat), lat)


GEOMS = {
    # level-2 lattice 3^4: no aliasing
    "l1_6x6x6x6_b2": ((6, 6, 6, 6), (2, 2, 2, 2)),
    # level-2 lattice (2, 2, 1, 1): extents 2 and 1 alias
    "l1_4x4x2x2_b2": ((4, 4, 2, 2), (2, 2, 2, 2)),
    # uneven blocks, level-2 lattice (3, 1, 2, 2)
    "l1_6x2x4x4_b212": ((6, 2, 4, 4), (2, 2, 2, 2)),
}


@pytest.fixture(scope="module", params=list(GEOMS))
def level2(request):
    dims, block = GEOMS[request.param]
    lat = CoarseBlocking(dims, (1, 1, 1, 1))
    n1, n2 = 2, 2
    A1 = _decaying_hpd(lat, n1, 1500)
    cb = CoarseBlocking(dims, block)
    phi2 = block_gram_schmidt(sy.complex_normal(1501, (n2, lat.Vc, n1)), cb)
    A2 = dense_to_stencil(coarse_dense_bruteforce(lambda v: coarse_apply(A1, v, lat), phi2, cb), cb)
    return lat, cb, n1, n2, A1, phi2, A2


def test_blocking_against_coordinate_walk():
    dims, block = (6, 2, 4, 4), (3, 2, 2, 1)
    cb = CoarseBlocking(dims, block)
    assert cb.coarse_dims == (2, 1, 2, 4) and cb.Vc == 16
    seen = np.zeros(int(np.prod(dims)), dtype=int)
    for t, z, y, x in itertools.product(range(dims[3]), range(dims[2]), range(dims[1]), range(dims[0])):
        a = x + dims[0] * (y + dims[1] * (z + dims[2] * t))
        bx, by, bz, bt = x // block[0], y // block[1], z // block[2], t // block[3]
        b = bx + 2 * (by + 1 * (bz + 2 * bt))
        assert cb.block_of_site[a] == b
        assert a in cb.sites_of_block[b]
        seen[a] += 1
    assert np.all(seen == 1)
    for b in range(cb.Vc):
        assert len(cb.sites_of_block[b]) == np.prod(block)
        for delta in itertools.product((-1, 0, 1), repeat=4):
            c = (cb.block_coords[b] + np.array(delta)) % np.array(cb.coarse_dims)
            assert cb.neighbour_block(b, delta) == c[0] + 2 * (c[1] + 1 * (c[2] + 2 * c[3]))


def test_block_orthonormal_same_span_and_adjoint(level2):
    lat, cb, n1, n2, A1, phi2, A2 = level2
    raw = sy.complex_normal(1501, (n2, lat.Vc, n1))
    for sites in cb.sites_of_block:
        X = phi2[:, sites].reshape(n2, -1)
        assert np.abs(X.conj() @ X.T - np.eye(n2)).max() < 1e-13
        Y = raw[:, sites].reshape(n2, -1)
        # the raw pieces lie in the span of the orthonormal ones
        assert np.abs(Y - (Y @ X.conj().T) @ X).max() < 1e-12 * np.abs(Y).max()
    c = sy.complex_normal(1502, (cb.Vc, n2))
    v = sy.complex_normal(1503, (lat.Vc, n1))
    assert abs(np.vdot(c, restrict(phi2, v, cb)) - np.vdot(prolong(phi2, c, cb), v)) < 1e-12 * np.abs(c).sum()
    assert np.abs(restrict(phi2, prolong(phi2, c, cb), cb) - c).max() < 1e-13


def test_stencil_equals_dense_galerkin_product(level2):
    lat, cb, n1, n2, A1, phi2, A2 = level2
    N1, N2 = lat.Vc * n1, cb.Vc * n2
    D1 = stencil_to_dense(A1, lat).reshape(N1, N1)
    P = np.zeros((N1, N2), dtype=np.complex128)
    for j in range(N2):
        e = np.zeros(N2, dtype=np.complex128)
        e[j] = 1.0
        P[:, j] = prolong(phi2, e.reshape(cb.Vc, n2), cb).ravel()
    assert np.abs(P.conj().T @ P - np.eye(N2)).max() < 1e-13
    G = P.conj().T @ D1 @ P
    D2 = stencil_to_dense(A2, cb).reshape(N2, N2)
    assert np.abs(D2 - G).max() < 1e-12 * np.abs(G).max()
    # nothing couples level-2 blocks two or more blocks apart along any
    # direction (periodic distance): the 81-point stencil holds all of G
    bc, L = cb.block_coords, np.array(cb.coarse_dims)
    d = np.abs(bc[:, None, :] - bc[None, :, :])
    dist = np.minimum(d, L - d).max(axis=2)
    far = np.repeat(np.repeat(dist >= 2, n2, axis=0), n2, axis=1)
    assert np.abs(G[far]).max(initial=0.0) < 1e-14 * np.abs(G).max()
    # the stencil apply is the Galerkin product
    c = sy.complex_normal(1504, (cb.Vc, n2))
    want = G @ c.ravel()
    assert np.abs(coarse_apply(A2, c, cb).ravel() - want).max() < 1e-12 * np.abs(want).max()


def test_hermitian_positive_and_galerkin_bounds(level2):
    lat, cb, n1, n2, A1, phi2, A2 = level2
    N1, N2 = lat.Vc * n1, cb.Vc * n2
    D1 = stencil_to_dense(A1, lat).reshape(N1, N1)
    D2 = stencil_to_dense(A2, cb).reshape(N2, N2)
    assert np.abs(D2 - D2.conj().T).max() < 1e-13 * np.abs(D2).max()
    e1, e2 = np.linalg.eigvalsh(D1), np.linalg.eigvalsh(D2)
    assert e2[0] > 0
    assert e2[0] >= e1[0] * (1 - 1e-12) and e2[-1] <= e1[-1] * (1 + 1e-12)


def test_deflated_level1_solve():
    """A-DEF2 on the level-1 operator with the level-2 space from inverse
    iteration: exact Q2 keeps Q2 r_k = 0, the solve meets numpy's dense
    solution, and needs fewer iterations than CG."""
    lat = CoarseBlocking((6, 6, 6, 6), (1, 1, 1, 1))
    n1, n2 = 2, 2
    A1 = _decaying_hpd(lat, n1, 1510, lam_min=0.005)
    cb = CoarseBlocking(lat.lattice_dims, (2, 2, 2, 2))

    def apply_A1(v):
        return coarse_apply(A1, v, lat)

    phi2 = inverse_iteration_subspace(apply_A1, sy.complex_normal(1511, (n2, lat.Vc, n1)), cb, steps=2, tol=1e-4)
    A2 = dense_to_stencil(coarse_dense_bruteforce(apply_A1, phi2, cb), cb)
    b = sy.complex_normal(1512, (lat.Vc, n1))
    D1 = stencil_to_dense(A1, lat).reshape(lat.Vc * n1, -1)
    xs = np.linalg.solve(D1, b.ravel()).reshape(b.shape)
    res = adef2(apply_A1, b, DeflationSpace(phi2, cb, A2), 1e-10, M=lambda v: v, track_invariants=True)
    assert res.true_residual < 2e-10
    assert np.sqrt(norm2(res.x - xs) / norm2(xs)) < 1e-7
    qr, _ = np.array(res.invariants).T
    assert qr.max() < 1e-9
    _, it_cg = cg(apply_A1, b, 1e-10)
    assert res.iterations < it_cg


def test_three_level_solve_meets_cg_solution():
    """Domain wall operator 8x8x4x4, Ls 4 (coarse lattice 2x2x1x1, Nvec 6),
    a level-2 blocking (1, 2, 1, 1) with Nvec 3, the level-1 solve A-DEF2 with
    Q2 to 1e-4: HDCG with three levels meets CG's solution."""
    U = sy.gauge_field((8, 8, 4, 4), 0.4, 1520)
    d = DWF((8, 8, 4, 4), 4, 1.8, 1.5, 0.5, 0.05, U)
    bl = Blocking(d, (4, 4, 4, 4))
    phi = block_gram_schmidt(sy.gaussian_fermions(d.lat.dims, d.Ls, 1521, 6), bl)
    A1 = dense_to_stencil(coarse_dense_bruteforce(d.mdagm, phi, bl), bl)

    def apply_A1(v):
        return coarse_apply(A1, v, bl)

    cb = CoarseBlocking(bl.coarse_dims, (1, 2, 1, 1))
    phi2 = inverse_iteration_subspace(apply_A1, sy.complex_normal(1522, (3, bl.Vc, 6)), cb, steps=2, tol=1e-6)
    A2 = dense_to_stencil(coarse_dense_bruteforce(apply_A1, phi2, cb), cb)
    D3 = DeflationSpace(phi, bl, A1, coarse_tol=1e-4, level2=DeflationSpace(phi2, cb, A2))
    b = sy.gaussian_fermion(d.lat.dims, d.Ls, 1523)
    res = adef2(d.mdagm, b, D3, 1e-8, mirs_iter=3)
    assert res.true_residual < 2e-8
    xs, _ = cg(d.mdagm, b, 1e-12)
    assert np.sqrt(norm2(res.x - xs) / norm2(xs)) < 1e-5
    assert len(D3.coarse_iters) > 0
