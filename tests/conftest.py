import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def golden():
    import json
    with open(os.path.join(ROOT, "tests", "golden", "paper_facts.json")) as f:
        return json.load(f)


@pytest.fixture(scope="session")
def little_dirac_12x12x4x4():
    """Little Dirac operator of a 12x12x4x4, Ls 4 Mobius lattice: coarse grid
    3x3x1x1, Nvec 4 from inverse iteration (dimension 36, spectrum 0.18 .. 6.5
    with four isolated low modes).  Built once: the brute-force assembly takes
    about 40 s.  Returns (dwf, blocking, phi, stencil, dense, eigenvalues)."""
    import numpy as np

    import synthetic as sy
    from oracle.coarse import Blocking, coarse_dense_bruteforce, dense_to_stencil, stencil_to_dense
    from oracle.dwf import DWF
    from oracle.solvers import inverse_iteration_subspace

    dims, Ls = (12, 12, 4, 4), 4
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.01, sy.gauge_field(dims, 0.4, 1200))
    bl = Blocking(d, (4, 4, 4, 4))
    phi = inverse_iteration_subspace(d.mdagm, sy.gaussian_fermions(dims, Ls, 1201, 4), bl, steps=2, tol=1e-4)
    A = dense_to_stencil(coarse_dense_bruteforce(d.mdagm, phi, bl), bl)
    n = bl.Vc * 4
    Dn = stencil_to_dense(A, bl).reshape(n, n)
    return d, bl, phi, A, Dn, np.linalg.eigvalsh(Dn)


@pytest.fixture(scope="session")
def two_level_8x8x4x4():
    """A two-level problem shared by several oracle pins: the 8x8x4x4, Ls 4
    Moebius operator (m = 0.05, links with eps 0.4), Nvec 6 from two steps of
    inverse iteration, its little Dirac operator, a Gaussian source and the CG
    solution to 1e-12 with the CG iteration count to 1e-8.
    Returns (dwf, blocking, phi, stencil, b, x_cg, cg_iterations_1e-8)."""
    import numpy as np

    import synthetic as sy
    from oracle.coarse import Blocking, coarse_dense_bruteforce, dense_to_stencil
    from oracle.dwf import DWF
    from oracle.solvers import cg, inverse_iteration_subspace

    dims, Ls = (8, 8, 4, 4), 4
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.05, sy.gauge_field(dims, 0.4, 1900))
    bl = Blocking(d, (4, 4, 4, 4))
    phi = inverse_iteration_subspace(d.mdagm, sy.gaussian_fermions(dims, Ls, 1901, 6), bl, steps=2, tol=1e-3)
    A = dense_to_stencil(coarse_dense_bruteforce(d.mdagm, phi, bl), bl)
    b = sy.gaussian_fermion(dims, Ls, 1902)
    hist = []
    xs, _ = cg(d.mdagm, b, 1e-12, history=hist)
    it8 = next(i + 1 for i, h in enumerate(hist) if h <= 1e-8)
    return d, bl, phi, A, b, xs, it8
