"""FP64 CPU oracle for the HDCG hot path (arXiv 1402.2585).

TEST INFRASTRUCTURE.  This package is the plain, slow, obviously correct
definition that the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline`` leg and
``--impl reference``) may import it.  The library never does, and it shares
no code with the CUDA path: both sides only share the seeded input
generators in ``synthetic/``.

Modules
-------
``dwf``      lattice indexing, gamma matrices, Wilson hop, Moebius/Shamir
             s-direction operators, the Schur-complement operator Mpc, its
             adjoint and H = Mpc^dag Mpc (Sec. 4, Eq. for the Hermitian
             red-black operator).
``coarse``   blocks, block Gram-Schmidt, restriction / prolongation, the
             little Dirac operator by brute force and by the Fourier trick,
             the coarse stencil apply (Sec. 2, Sec. 5.1, Sec. 5.1.1).
``solvers``  CG, the infra-red shifted smoother M_IRS, inverse-iteration
             subspace, A-DEF2 with flexible beta (Figs. pcg / pcg_general,
             Table algos, Sec. 4.3); second-level global deflation and A-DEF1
             with the Chebyshev preconditioner on Q_trunc (Sec. 5.2).
``pcg_family`` the generalised preconditioned CG of Fig. pcg_general with the
             rows of Table algos (PREC, AD, DEF1, DEF2, A-DEF1, A-DEF2, BNN,
             V(1,1)) and the frozen CG polynomial M_IRSpoly (Sec. 4.5).
``codec``    reduced-precision spinor codecs: 16-bit truncation and the 8-bit
             format with a half-precision prefactor (Sec. 6.5).
``subspace`` subspace generation by the rational low-pass filter: multi-shift
             CG, wall-placed noise, surface truncation (Sec. 4.2).
``level2``   blocks of the coarse lattice: the blocked second coarsening of
             a three-level hierarchy (Sec. 2 applied to the little Dirac
             operator).

Parity status of each function is stated in its docstring; every function
here is pinned by a ``-m "not gpu"`` test except where marked
"parity unpinned".
"""
