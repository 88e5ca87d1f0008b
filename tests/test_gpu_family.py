"""The preconditioner family of Table algos on the GPU (Sec. 4.5, Fig.
pcg_general, Table preconditioner) against the FP64 oracle's generalised PCG.

Both sides use the same subspace and little Dirac operator (the oracle's,
uploaded), an exact coarse solve (the GPU's coarse CG to 1e-13) and the same
linear smoother M_IRSpoly (6 iterations, shift 1, frozen on b), so every
method runs the same recurrences in FP64: the iteration counts agree to one
and the solutions meet the oracle's CG solution to 1e-6 (the solves run to
1e-9; kappa is about 72 at m = 0.3).  The nonlinear M_IRS and the Chebyshev
smoother are checked with A-DEF2 (flexible beta) against the solution.
"""
import numpy as np
import pytest

import synthetic as sy
from oracle.coarse import Blocking, coarse_dense_bruteforce, dense_to_stencil
from oracle.dwf import DWF, norm2
from oracle.pcg_family import METHODS, MirsPoly, generalised_pcg
from oracle.solvers import DeflationSpace, cg, inverse_iteration_subspace
from paper_1402_2585_gb300 import F64, Hdcg
from paper_1402_2585_gb300.binding import (ALG_ADEF2_FAMILY, FAMILY, SMOOTHER_CHEBYSHEV, SMOOTHER_MIRS,
                                           SMOOTHER_MIRSPOLY)
from tests.gpu_util import rel, torch_or_skip

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def problem():
    torch = torch_or_skip()
    dims, Ls = (8, 4, 4, 4), 4
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.3, sy.gauge_field(dims, 0.4, 1800))
    bl = Blocking(d, (4, 4, 4, 4))
    phi = inverse_iteration_subspace(d.mdagm, sy.gaussian_fermions(dims, Ls, 1801, 4), bl, steps=1, tol=1e-2)
    A = dense_to_stencil(coarse_dense_bruteforce(d.mdagm, phi, bl), bl)
    defl = DeflationSpace(phi, bl, A, coarse_tol=0.0)
    b = sy.gaussian_fermion(dims, Ls, 1802)
    xs, _ = cg(d.mdagm, b, 1e-13)
    h = Hdcg(dims, Ls, stream=torch.cuda.current_stream().cuda_stream)
    h.set_dwf(1.8, 1.5, 0.5, 0.3)
    h.set_gauge(torch.from_numpy(d.U).cuda())
    h.set_subspace((4, 4, 4, 4), torch.from_numpy(phi).cuda(), prec=F64, already_orthonormal=True)
    h.set_coarse(A, prec=F64)
    return torch, d, defl, b, xs, h


def _gpu(problem, alg, **kw):
    torch, d, defl, b, xs, h = problem
    prm = Hdcg.default_params(algorithm=alg, outer_prec=F64, coarse_tol=1e-13, coarse_maxiter=100000,
                              maxiter=2000, flexible=0, smoother=SMOOTHER_MIRSPOLY, mirs_iter=6, mirs_shift=1.0)
    for k, v in kw.items():
        setattr(prm, k, v)
    x = np.zeros_like(b)
    st = h.solve(b, x, TOL, prm)
    return x, st


@pytest.mark.parametrize("name", METHODS)
def test_method_matches_oracle(problem, name):
    torch, d, defl, b, xs, h = problem
    M = MirsPoly(d.mdagm, b, n_iter=6, shift=1.0)
    xo, it_o = generalised_pcg(name, d.mdagm, b, defl, M, TOL, maxiter=2000)
    xg, st = _gpu(problem, FAMILY[name])
    assert st.status == 0, name
    assert abs(st.iterations - it_o) <= 1, (name, st.iterations, it_o)
    assert rel(xg, xs) < 1e-6, name
    assert rel(xg, xo) < 1e-6, name


def test_def2_adef2_bnn_take_the_same_iterations(problem):
    """Sec. 4.5's equivalence on the GPU: with exact Q and a linear smoother,
    DEF2, A-DEF2 and BNN from the DEF2 start run the same recurrences."""
    its = {name: _gpu(problem, FAMILY[name])[1].iterations for name in ("DEF2", "A-DEF2", "BNN-DEF2-start")}
    assert max(its.values()) - min(its.values()) <= 1, its


def test_adef2_with_mirs_and_chebyshev_smoothers(problem):
    torch, d, defl, b, xs, h = problem
    x, st = _gpu(problem, ALG_ADEF2_FAMILY, smoother=SMOOTHER_MIRS, mirs_iter=7, flexible=1)
    assert st.status == 0 and rel(x, xs) < 1e-6
    # Chebyshev on [lo, hi] with hi above lambda_max(H) (power iteration)
    v = sy.gaussian_fermion(d.lat.dims, d.Ls, 1810)
    for _ in range(60):
        v = d.mdagm(v)
        v /= np.sqrt(norm2(v))
    lmax = float(np.vdot(v, d.mdagm(v)).real)
    x, st = _gpu(problem, ALG_ADEF2_FAMILY, smoother=SMOOTHER_CHEBYSHEV, cheb_order=8, cheb_lo=0.05 * lmax,
                 cheb_hi=1.1 * lmax)
    assert st.status == 0 and rel(x, xs) < 1e-6
    assert st.true_residual < 1e-7


def test_family_rejects_bad_parameters(problem):
    from paper_1402_2585_gb300 import HdcgError
    with pytest.raises(HdcgError):
        _gpu(problem, ALG_ADEF2_FAMILY, smoother=SMOOTHER_CHEBYSHEV, cheb_order=8, cheb_lo=2.0, cheb_hi=1.0)
    with pytest.raises(HdcgError):
        _gpu(problem, ALG_ADEF2_FAMILY, smoother=7)
