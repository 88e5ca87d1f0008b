"""FP64 oracle: blocked subspace, restriction/prolongation and the little Dirac operator.

TEST INFRASTRUCTURE (see ``oracle/__init__``): never imported by the library.

Sec. 2 cuts each subspace vector phi_k into 4D blocks b (all of the fifth
dimension inside one block, Sec. 5.1), orthonormalises the block pieces
phi_k^b by Gram-Schmidt, and defines the little Dirac operator

    A^{ab}_{jk} = <phi_j^a | H | phi_k^b>.

With blocks of at least 4 sites per dimension, H (taxicab range 4) couples a
block only to blocks at most one hop away in each direction: 80 neighbours
plus itself (Sec. 5.1).  The canonical stencil layout is
``A[a][l][j][k] = <phi_j^a | H | phi_k^{a + delta_l}>`` with
``l = (dx+1) + 3 (dy+1) + 9 (dz+1) + 27 (dt+1)``, delta in {-1, 0, 1}^4.

Coarse extents of 1 or 2 alias offsets (+1 and -1 name the same block).
Reading used here: along a dimension of coarse extent 2 only delta in {0, +1}
is stored, along extent 1 only delta = 0; the other entries are zero, so the
stencil apply sums each distinct coupling exactly once.

Parity: pinned by tests/test_oracle_coarse.py (orthonormality and span of the
block Gram-Schmidt, R = P^dag and R P = 1, stencil apply equal to R H P,
Hermiticity and positivity of A, zero couplings beyond one block hop,
Fourier trick equal to brute force, hop counts 1/9/33/65/81).
"""
from __future__ import annotations

import itertools

import numpy as np

from .dwf import DWF


def stencil_offsets() -> np.ndarray:
    """(81, 4) offsets delta_l, l = (dx+1) + 3(dy+1) + 9(dz+1) + 27(dt+1)."""
    offs = np.zeros((81, 4), dtype=np.int64)
    for l in range(81):
        r = l
        for mu in range(4):
            offs[l, mu] = r % 3 - 1
            r //= 3
    return offs


def canonical_offsets(coarse_dims, mu: int):
    """Distinct offsets stored along dimension mu (see module docstring)."""
    L = coarse_dims[mu]
    if L >= 3:
        return [-1, 0, 1]
    if L == 2:
        return [0, 1]
    return [0]


class Blocking:
    """Partition of the odd-checkerboard sites into 4D blocks."""

    def __init__(self, dwf: DWF, block):
        self.dwf = dwf
        self.block = tuple(int(b) for b in block)
        dims = dwf.lat.dims
        if any(d % b for d, b in zip(dims, self.block)):
            raise ValueError("block extents must divide the lattice extents")
        self.coarse_dims = tuple(d // b for d, b in zip(dims, self.block))
        self.Vc = int(np.prod(self.coarse_dims))
        odd = dwf.lat.sites[1]
        bc = dwf.lat.coords[odd] // np.array(self.block)
        self.block_coords_of_site = bc
        Lcx, Lcy, Lcz, _ = self.coarse_dims
        self.block_of_site = bc[:, 0] + Lcx * (bc[:, 1] + Lcy * (bc[:, 2] + Lcz * bc[:, 3]))
        self.sites_of_block = [np.nonzero(self.block_of_site == b)[0] for b in range(self.Vc)]
        lexc = np.arange(self.Vc)
        self.block_coords = np.stack([lexc % Lcx, (lexc // Lcx) % Lcy,
                                      (lexc // (Lcx * Lcy)) % Lcz,
                                      lexc // (Lcx * Lcy * Lcz)], axis=1)

    def coarse_lex(self, c):
        c = np.asarray(c) % np.array(self.coarse_dims)
        Lcx, Lcy, Lcz, _ = self.coarse_dims
        return c[..., 0] + Lcx * (c[..., 1] + Lcy * (c[..., 2] + Lcz * c[..., 3]))

    def neighbour_block(self, a, delta):
        return self.coarse_lex(self.block_coords[a] + np.asarray(delta))


# ----------------------------------------------------------------------------
# block Gram-Schmidt, restriction, prolongation (Sec. 2)
# ----------------------------------------------------------------------------

def block_gram_schmidt(phi, blocking: Blocking):
    """Orthonormalise the block pieces phi_k^b within every block.

    Modified Gram-Schmidt over k = 0..Nvec-1, each vector orthogonalised
    against the earlier ones twice, then normalised.  ``phi`` has shape
    (Nvec, V/2, Ls, 4, 3); a new array is returned.
    """
    out = np.array(phi, dtype=np.complex128, copy=True)
    nvec = out.shape[0]
    for sites in blocking.sites_of_block:
        X = out[:, sites].reshape(nvec, -1)
        for k in range(nvec):
            for _ in range(2):
                for j in range(k):
                    X[k] -= np.vdot(X[j], X[k]) * X[j]
            X[k] /= np.linalg.norm(X[k])
        out[:, sites] = X.reshape((nvec, len(sites)) + out.shape[2:])
    return out


def restrict(phi, v, blocking: Blocking):
    """c[b, k] = <phi_k^b, v> = sum_{x in b} conj(phi_k(x)) . v(x); shape (Vc, Nvec)."""
    nvec = phi.shape[0]
    c = np.zeros((blocking.Vc, nvec), dtype=np.complex128)
    for b, sites in enumerate(blocking.sites_of_block):
        X = phi[:, sites].reshape(nvec, -1)
        c[b] = np.conj(X) @ v[sites].ravel()
    return c


def prolong(phi, c, blocking: Blocking):
    """v(x) = sum_k c[b(x), k] phi_k(x)."""
    return np.einsum("nk,kn...->n...", c[blocking.block_of_site], phi)


# ----------------------------------------------------------------------------
# the little Dirac operator (Sec. 2, Sec. 5.1, Sec. 5.1.1)
# ----------------------------------------------------------------------------

def coarse_dense_bruteforce(apply_H, phi, blocking: Blocking):
    """A_dense[a, j, b, k] = <phi_j^a | H | phi_k^b> by one H per (b, k)."""
    nvec = phi.shape[0]
    Vc = blocking.Vc
    A = np.zeros((Vc, nvec, Vc, nvec), dtype=np.complex128)
    for b, sites in enumerate(blocking.sites_of_block):
        for k in range(nvec):
            v = np.zeros(phi.shape[1:], dtype=np.complex128)
            v[sites] = phi[k, sites]
            A[:, :, b, k] = restrict(phi, apply_H(v), blocking)
    return A


def dense_to_stencil(A_dense, blocking: Blocking):
    """Canonical [Vc][81][N][N] stencil from the dense matrix (aliasing rule above)."""
    Vc, nvec = A_dense.shape[0], A_dense.shape[1]
    offs = stencil_offsets()
    keep = [canonical_offsets(blocking.coarse_dims, mu) for mu in range(4)]
    A = np.zeros((Vc, 81, nvec, nvec), dtype=np.complex128)
    for l in range(81):
        if not all(offs[l, mu] in keep[mu] for mu in range(4)):
            continue
        for a in range(Vc):
            b = blocking.neighbour_block(a, offs[l])
            A[a, l] = A_dense[a, :, b, :]
    return A


def stencil_to_dense(A, blocking: Blocking):
    Vc, nvec = A.shape[0], A.shape[2]
    offs = stencil_offsets()
    D = np.zeros((Vc, nvec, Vc, nvec), dtype=np.complex128)
    for a in range(Vc):
        for l in range(81):
            b = blocking.neighbour_block(a, offs[l])
            D[a, :, b, :] += A[a, l]
    return D


def coarse_fourier(apply_H, phi, blocking: Blocking):
    """Little Dirac operator by the Fourier trick of Sec. 5.1.1.

    For each subspace vector k and each low momentum p^s (one unit or less
    per direction), apply H to phi~_k(p) = sum_b exp(i p.x_b) phi_k^b,
    project onto every phi_j^b and multiply by exp(-i p.x_b).  This gives
    F[b, s, j, k] = sum_l M_sl A[b, l, j, k] with M_sl = exp(i p^s . delta^l);
    A follows from M^-1.  Momentum reading: p_mu = 2 pi n_mu / Lc_mu (periodic
    on the coarse torus).  Along a dimension of coarse extent L < 3 only the
    ``canonical_offsets`` exist and n runs over 0..L-1, so the number of
    H applications is Nvec times the number of distinct offsets (81 when every
    coarse extent is at least 3).
    """
    nvec = phi.shape[0]
    cd = blocking.coarse_dims
    keep = [canonical_offsets(cd, mu) for mu in range(4)]
    moms = []
    for mu in range(4):
        moms.append([-1, 0, 1] if cd[mu] >= 3 else list(range(cd[mu])))
    deltas = list(itertools.product(*keep))
    momenta = list(itertools.product(*moms))
    nS = len(momenta)
    assert nS == len(deltas)
    Lc = np.array(cd, dtype=np.float64)
    M = np.zeros((nS, nS), dtype=np.complex128)
    for s, n in enumerate(momenta):
        for l, d in enumerate(deltas):
            M[s, l] = np.exp(1j * 2 * np.pi * np.sum(np.array(n) * np.array(d) / Lc))
    F = np.zeros((blocking.Vc, nS, nvec, nvec), dtype=np.complex128)
    xb = blocking.block_coords.astype(np.float64)
    for s, n in enumerate(momenta):
        phase_b = np.exp(1j * 2 * np.pi * (xb @ (np.array(n) / Lc)))
        ph_site = phase_b[blocking.block_of_site]
        for k in range(nvec):
            v = phi[k] * ph_site[:, None, None, None]
            proj = restrict(phi, apply_H(v), blocking)
            F[:, s, :, k] = np.conj(phase_b)[:, None] * proj
    Acomp = np.einsum("ls,bsjk->bljk", np.linalg.inv(M), F)
    offs = stencil_offsets()
    A = np.zeros((blocking.Vc, 81, nvec, nvec), dtype=np.complex128)
    for li, d in enumerate(deltas):
        l = int(np.nonzero((offs == np.array(d)).all(axis=1))[0][0])
        A[:, l] = Acomp[:, li]
    return A


def coarse_apply(A, x, blocking: Blocking):
    """y[a] = sum_l A[a, l] x[a + delta_l]; x has shape (Vc, Nvec)."""
    offs = stencil_offsets()
    y = np.zeros_like(x, dtype=np.complex128)
    for l in range(81):
        nb = blocking.neighbour_block(np.arange(blocking.Vc), offs[l])
        y += np.einsum("ajk,ak->aj", A[:, l], x[nb])
    return y
