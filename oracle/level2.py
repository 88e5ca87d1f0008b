"""FP64 oracle: the blocked second coarsening (three-level HDCG).

TEST INFRASTRUCTURE (see ``oracle/__init__``): never imported by the library.

The little Dirac operator A of Sec. 2 is itself a nearest-neighbour
operator on the coarse lattice (81-point stencil, Sec. 5.1), so the
construction of Sec. 2 applies to it once more:
* Nvec2 coarse vectors phi2_k (shape (Vc, Nvec) each) are cut into 4D blocks
  of the coarse lattice and the block pieces are orthonormalised;
* R2 c = <phi2_k^b, c>, P2 = R2^dag;
* A2^{ab}_{jk} = <phi2_j^a | A | phi2_k^b>, and the level-1 solve is deflated
  by Q2 = P2 A2^-1 R2.

Reading: the paper's own hierarchy (Sec. 5.2, Table hierarchy) ends in a
single global, dense level; the three-level workload ("4^4 then 2^4 blocks,
Nvec 40 then 24") replaces it by this blocked level, i.e. the method of
Sec. 2 applied recursively.  A couples coarse sites at most one site apart in
each direction, so with level-2 blocks of any size A2 couples a block only to
blocks at most one hop away: A2 is again an 81-point stencil in the canonical
layout of ``oracle.coarse``, with the same aliasing rule for level-2 extents
1 and 2.  The block Gram-Schmidt, restriction, prolongation, brute-force
assembly and stencil apply of ``oracle.coarse`` are written for any blocking
object with the attributes below, so ``CoarseBlocking`` reuses them
unchanged.  The level-1 solve is ``solvers.adef2`` on A with
``DeflationSpace(phi2, CoarseBlocking, A2)`` (see ``solvers.DeflationSpace.level2``).

Parity: pinned by tests/test_oracle_level2.py (block orthonormality, R2 =
P2^dag and R2 P2 = 1, the stencil apply of A2 equal to R2 A P2 on aliased and
unaliased level-2 lattices, zero couplings beyond one level-2 block hop,
Hermiticity and positivity, the three-level solve reaching the dense
solution, and deflated level-1 solves needing fewer iterations than CG).
"""
from __future__ import annotations

import numpy as np


class CoarseBlocking:
    """Partition of a coarse lattice into 4D blocks of ``block`` sites.

    Coarse sites are numbered as ``oracle.coarse.Blocking`` numbers its
    blocks: lexicographically with x fastest.  The attributes match
    ``Blocking`` (``coarse_dims``, ``Vc``, ``block_of_site``,
    ``sites_of_block``, ``block_coords``, ``neighbour_block``), with the
    level-2 blocks in the role of the coarse sites.
    """

    def __init__(self, lattice_dims, block):
        self.lattice_dims = tuple(int(d) for d in lattice_dims)
        self.block = tuple(int(b) for b in block)
        if any(d % b for d, b in zip(self.lattice_dims, self.block)):
            raise ValueError("block extents must divide the coarse lattice extents")
        self.coarse_dims = tuple(d // b for d, b in zip(self.lattice_dims, self.block))
        self.Vc = int(np.prod(self.coarse_dims))
        n = int(np.prod(self.lattice_dims))
        self.coords = self._coords(np.arange(n), self.lattice_dims)
        bc = self.coords // np.array(self.block)
        self.block_of_site = self.coarse_lex(bc)
        self.sites_of_block = [np.nonzero(self.block_of_site == b)[0] for b in range(self.Vc)]
        self.block_coords = self._coords(np.arange(self.Vc), self.coarse_dims)

    @staticmethod
    def _coords(lex, dims):
        Lx, Ly, Lz, _ = dims
        return np.stack([lex % Lx, (lex // Lx) % Ly, (lex // (Lx * Ly)) % Lz, lex // (Lx * Ly * Lz)], axis=1)

    def coarse_lex(self, c):
        c = np.asarray(c) % np.array(self.coarse_dims)
        Lx, Ly, Lz, _ = self.coarse_dims
        return c[..., 0] + Lx * (c[..., 1] + Ly * (c[..., 2] + Lz * c[..., 3]))

    def neighbour_block(self, a, delta):
        return self.coarse_lex(self.block_coords[a] + np.asarray(delta))
