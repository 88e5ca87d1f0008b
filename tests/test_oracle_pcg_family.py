"""Pins of the generalised preconditioned CG and its family (Sec. 4.5, Fig.
pcg_general, Tables precs and algos).  No GPU.

What fixes them, independently of the oracle's own code:
* every method reaches the solution of the textbook CG (oracle cg at 1e-12);
* the equivalence stated in Sec. 4.5 (after Tang et al.): with exact Q and a
  fixed linear smoother, DEF2, A-DEF2 and BNN from the DEF2 start vector
  produce the same iterates, and DEF1's V_end the same solution;
* Hermiticity of the BNN and V(1,1) preconditioners (Table precs), checked as
  <u, M1 v> = <M1 u, v> on random vectors;
* M_IRSpoly reproduces M_IRS on its reference vector, and is a fixed linear,
  Hermitian operator.
"""
import numpy as np
import pytest

import synthetic as sy
from oracle.coarse import Blocking, coarse_dense_bruteforce, dense_to_stencil
from oracle.dwf import DWF, norm2
from oracle.pcg_family import METHODS, ChebyshevSmoother, MirsPoly, generalised_pcg, method
from oracle.solvers import DeflationSpace, cg, inverse_iteration_subspace, mirs


@pytest.fixture(scope="module")
def problem():
    dims, Ls = (8, 4, 4, 4), 4
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.3, sy.gauge_field(dims, 0.4, 1800))
    bl = Blocking(d, (4, 4, 4, 4))
    phi = inverse_iteration_subspace(d.mdagm, sy.gaussian_fermions(dims, Ls, 1801, 4), bl, steps=1, tol=1e-2)
    A = dense_to_stencil(coarse_dense_bruteforce(d.mdagm, phi, bl), bl)
    defl = DeflationSpace(phi, bl, A, coarse_tol=0.0)
    b = sy.gaussian_fermion(dims, Ls, 1802)
    M = MirsPoly(d.mdagm, b, n_iter=6, shift=1.0)
    xs, _ = cg(d.mdagm, b, 1e-12)
    return d, defl, b, M, xs


@pytest.mark.parametrize("name", METHODS)
def test_every_method_reaches_the_solution(problem, name):
    d, defl, b, M, xs = problem
    x, it = generalised_pcg(name, d.mdagm, b, defl, M, 1e-8, maxiter=2000)
    assert np.sqrt(norm2(x - xs) / norm2(xs)) < 1e-5, (name, it)


def test_def2_adef2_bnn_iterates_agree(problem):
    d, defl, b, M, xs = problem
    runs = {}
    for name in ("DEF2", "A-DEF2", "BNN-DEF2-start"):
        hist = []
        _, it = generalised_pcg(name, d.mdagm, b, defl, M, 1e-10, history=hist)
        runs[name] = (it, hist)
    # equal in exact arithmetic; rounding separates the recursions slowly, so
    # the counts may differ by an iteration or two and the late iterates by
    # more than the early ones
    its = {k: v[0] for k, v in runs.items()}
    assert max(its.values()) - min(its.values()) <= 2, its
    ref = runs["DEF2"][1]
    for name in ("A-DEF2", "BNN-DEF2-start"):
        for k, (a, c) in enumerate(zip(ref[:15], runs[name][1][:15])):
            assert np.sqrt(norm2(a - c) / norm2(xs)) < 1e-9, (name, k)
    # DEF1 reaches the same solution through its V_end = Q b + P_R x
    x1, _ = generalised_pcg("DEF1", d.mdagm, b, defl, M, 1e-10)
    assert np.sqrt(norm2(x1 - ref[-1]) / norm2(xs)) < 1e-7


@pytest.mark.parametrize("name", ["BNN", "V11", "AD", "PREC"])
def test_hermitian_preconditioners(problem, name):
    d, defl, b, M, xs = problem
    M1 = method(name, d.mdagm, defl, M)[1]
    u = sy.gaussian_fermion(d.lat.dims, d.Ls, 1803)
    v = sy.gaussian_fermion(d.lat.dims, d.Ls, 1804)
    a, c = np.vdot(u, M1(v)), np.vdot(M1(u), v)
    assert abs(a - c) < 1e-10 * abs(a)


def test_mirs_poly_replays_and_is_linear_hermitian(problem):
    d, defl, b, M, xs = problem
    assert np.abs(M(b) - mirs(d.mdagm, b, 6, 1.0)).max() < 1e-12 * np.abs(M(b)).max()
    u = sy.gaussian_fermion(d.lat.dims, d.Ls, 1805)
    v = sy.gaussian_fermion(d.lat.dims, d.Ls, 1806)
    lin = M(2.0 * u - 0.5j * v) - (2.0 * M(u) - 0.5j * M(v))
    assert np.abs(lin).max() < 1e-12 * np.abs(M(u)).max()
    a, c = np.vdot(u, M(v)), np.vdot(M(u), v)
    assert abs(a - c) < 1e-12 * abs(a)
    # M_IRS itself is not linear: a CG polynomial adapts to its right-hand side
    assert np.abs(mirs(d.mdagm, u + v, 6, 1.0) - mirs(d.mdagm, u, 6, 1.0) - mirs(d.mdagm, v, 6, 1.0)).max() > 1e-6


def test_mssdef_is_def2_without_a_smoother(problem):
    """MssDef (the little Dirac operator alone) iterates as DEF2 with M = 1,
    by the same equivalence with exact Q, and reaches the solution in more
    iterations than with the smoother."""
    d, defl, b, M, xs = problem
    ident = lambda v: v
    h1, h2 = [], []
    x1, it1 = generalised_pcg("MssDef", d.mdagm, b, defl, M, 1e-10, maxiter=3000, history=h1)
    x2, it2 = generalised_pcg("DEF2", d.mdagm, b, defl, ident, 1e-10, maxiter=3000, history=h2)
    assert abs(it1 - it2) <= 2
    for k, (a, c) in enumerate(zip(h1[:15], h2[:15])):
        assert np.sqrt(norm2(a - c) / norm2(xs)) < 1e-9, k
    _, it_smoothed = generalised_pcg("A-DEF2", d.mdagm, b, defl, M, 1e-10, maxiter=3000)
    assert it_smoothed < it1


def _lambda_max(d, seed, iters=30):
    v = sy.gaussian_fermion(d.lat.dims, d.Ls, seed)
    lam = 0.0
    for _ in range(iters):
        v = v / np.sqrt(norm2(v))
        w = d.mdagm(v)
        lam = float(np.vdot(v, w).real)
        v = w
    return lam


def test_chebyshev_smoother(problem):
    """The Chebyshev option of Table preconditioner (order 8 on [hi/90, hi],
    hi above the spectrum): linear and Hermitian, and A-DEF2 with it reaches
    the CG solution."""
    d, defl, b, M, xs = problem
    hi = 1.2 * _lambda_max(d, 1807)
    C = ChebyshevSmoother(d.mdagm, 8, hi / 90, hi)
    u = sy.gaussian_fermion(d.lat.dims, d.Ls, 1808)
    v = sy.gaussian_fermion(d.lat.dims, d.Ls, 1809)
    lin = C(2.0 * u - 0.5j * v) - (2.0 * C(u) - 0.5j * C(v))
    assert np.abs(lin).max() < 1e-12 * np.abs(C(u)).max()
    a, c = np.vdot(u, C(v)), np.vdot(C(u), v)
    assert abs(a - c) < 1e-12 * abs(a)
    assert np.vdot(u, C(u)).real > 0
    x, it = generalised_pcg("A-DEF2", d.mdagm, b, defl, C, 1e-8, maxiter=2000)
    assert np.sqrt(norm2(x - xs) / norm2(xs)) < 1e-5, it


def test_prec_with_identity_is_textbook_cg(problem):
    """With M = 1 the generalised PCG of Fig. pcg_general reduces to the
    textbook CG: the same residual norms iteration by iteration (recomputed
    from its iterates) and the same iteration count."""
    d, defl, b, M, xs = problem
    hist_x, hist_r = [], []
    x1, it1 = generalised_pcg("PREC", d.mdagm, b, defl, lambda v: v, 1e-8, flexible=False, history=hist_x)
    x2, it2 = cg(d.mdagm, b, 1e-8, history=hist_r)
    assert abs(it1 - it2) <= 1
    bn = np.sqrt(norm2(b))
    for k, (xk, rk) in enumerate(zip(hist_x[:30], hist_r[:30])):
        tr = np.sqrt(norm2(b - d.mdagm(xk))) / bn
        assert abs(tr - rk) <= 1e-6 * rk, k
    assert np.sqrt(norm2(x1 - x2) / norm2(x2)) < 1e-8


def _steps(name, H, Q, M, r):
    """M1 r as the sequence of smoothing and coarse-correction steps."""
    if name == "V11":                       # pre-smooth, coarse-correct, post-smooth
        z = M(r)
        z = z + Q(r - H(z))
        return z + M(r - H(z))
    if name == "BNN":                       # z = M (r - H Q r), then coarse-correct
        z = M(r - H(Q(r)))
        return z + Q(r - H(z))
    if name == "A-DEF1":                    # coarse-correct, then smooth the rest
        q = Q(r)
        return q + M(r - H(q))
    if name == "A-DEF2":                    # smooth, then coarse-correct
        z = M(r)
        return z + Q(r - H(z))
    if name == "AD":
        return M(r) + Q(r)
    if name == "MssDef":                    # coarse correction of r itself
        return r + Q(r - H(r))
    raise ValueError(name)


@pytest.mark.parametrize("name", ["V11", "BNN", "A-DEF1", "A-DEF2", "AD", "MssDef"])
def test_preconditioners_as_smoothing_and_coarse_steps(problem, name):
    """Each M_1 of Tables precs and algos, written with P_L = 1 - H Q and
    P_R = 1 - Q H, equals its form as smoothing and coarse-correction steps
    (V(1,1): the symmetric two-grid cycle)."""
    d, defl, b, M, xs = problem
    M1 = method(name, d.mdagm, defl, M)[1]
    r = sy.gaussian_fermion(d.lat.dims, d.Ls, 1810)
    want = M1(r)
    got = _steps(name, d.mdagm, defl.Q, M, r)
    assert np.abs(got - want).max() < 1e-10 * np.abs(want).max()
