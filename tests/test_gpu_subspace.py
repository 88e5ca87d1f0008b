"""Parity of the GPU subspace generation of Sec. 4.2 with the FP64 oracle:
the rational low-pass filter (wall noise, multi-shift CG over the four shifts
lambda + i eps, the partial-fraction sum, the surface truncation, block
Gram-Schmidt), the promotion of a reduced-Ls subspace, and the second pass.

The block Gram-Schmidt of a fixed set of vectors is unique (positive
diagonal), and both sides draw the same noise from the shared counter-based
generator, so the subspaces are compared element by element.  Both sides
solve to relative residual 1e-11 (FP64) or 1e-7 (FP32); the filtered vectors
then agree to about kappa(H + lambda) times that, kappa <= 1e3 here, so the
bars are 1e-7 (FP64) and 2e-3 (FP32).
"""
import numpy as np
import pytest

import synthetic as sy
from oracle.coarse import Blocking, block_gram_schmidt
from oracle.dwf import DWF
from oracle.subspace import promote, rational_subspace, two_pass_subspace
from paper_1402_2585_gb300 import F16, F32, F64, Hdcg
from paper_1402_2585_gb300.binding import SUBSPACE_CONTINUE, SUBSPACE_RATIONAL
from tests.gpu_util import rel, torch_or_skip

pytestmark = pytest.mark.gpu

DIMS = (8, 4, 4, 4)
BLOCK = (4, 4, 4, 4)
M5, B, C = 1.8, 1.5, 0.5


def _handle(torch, U, Ls, mass):
    h = Hdcg(DIMS, Ls, stream=torch.cuda.current_stream().cuda_stream)
    h.set_dwf(M5, B, C, mass)
    h.set_gauge(torch.from_numpy(U).cuda())
    return h


def _get(h, Ls, nvec):
    out = np.zeros((nvec, sy.volume(DIMS) // 2, Ls, 4, 3), dtype=np.complex128)
    h.get_subspace(out)
    return out


@pytest.mark.parametrize("prec,tol,bar", [(F64, 1e-11, 1e-7), (F32, 1e-7, 2e-3)])
@pytest.mark.parametrize("depth", [0, 1])
def test_rational_subspace_matches_oracle(prec, tol, bar, depth):
    torch = torch_or_skip()
    Ls, nvec, mass, seed = 4, 3, 0.02, 1801
    U = sy.gauge_field(DIMS, 0.4, 1800)
    d = DWF(DIMS, Ls, M5, B, C, mass, U)
    bl = Blocking(d, BLOCK)
    ref = rational_subspace(d.mdagm, bl, nvec, seed, lam=0.05, eps=0.02, tol=1e-12, depth=depth)
    h = _handle(torch, U, Ls, mass)
    h.build_subspace(BLOCK, nvec, prec=prec, inv_tol=tol, inv_maxiter=5000, seed=seed,
                     method=SUBSPACE_RATIONAL, filter_lambda=0.05, filter_eps=0.02, filter_order=4,
                     surface_depth=depth)
    got = _get(h, Ls, nvec)
    assert rel(got, ref) < bar
    if depth:
        assert np.all(got[:, :, depth:Ls - depth] == 0)


def test_rational_subspace_f16_storage():
    """A 16-bit subspace is filtered in FP32 and rounded once: block-orthonormal
    to 16-bit accuracy and within the rounding of the FP32 result."""
    torch = torch_or_skip()
    Ls, nvec, mass, seed = 4, 3, 0.02, 1802
    U = sy.gauge_field(DIMS, 0.4, 1803)
    d = DWF(DIMS, Ls, M5, B, C, mass, U)
    bl = Blocking(d, BLOCK)
    ref = rational_subspace(d.mdagm, bl, nvec, seed, lam=0.05, eps=0.02, tol=1e-12)
    h = _handle(torch, U, Ls, mass)
    h.build_subspace(BLOCK, nvec, prec=F16, inv_tol=1e-7, inv_maxiter=5000, seed=seed,
                     method=SUBSPACE_RATIONAL, filter_lambda=0.05, filter_eps=0.02, filter_order=4)
    got = _get(h, Ls, nvec)
    assert rel(got, ref) < 5e-3


def test_promotion_matches_oracle():
    """A reduced-Ls (Ls1 = 4, its own mass) rational subspace promoted to Ls = 8:
    the oracle's placement followed by block Gram-Schmidt, to FP64 rounding."""
    torch = torch_or_skip()
    Ls, Ls1, nvec, seed = 8, 4, 2, 1804
    U = sy.gauge_field(DIMS, 0.4, 1805)
    h1 = _handle(torch, U, Ls1, 0.05)
    h1.build_subspace(BLOCK, nvec, prec=F64, inv_tol=1e-11, inv_maxiter=5000, seed=seed,
                      method=SUBSPACE_RATIONAL, filter_lambda=0.05, filter_eps=0.02)
    phi1 = _get(h1, Ls1, nvec)
    h = _handle(torch, U, Ls, 0.01)
    h.promote_subspace(h1, prec=F64)
    d = DWF(DIMS, Ls, M5, B, C, 0.01, U)
    ref = block_gram_schmidt(promote(phi1, Ls), Blocking(d, BLOCK))
    assert rel(_get(h, Ls, nvec), ref) < 1e-12


def test_two_pass_subspace_matches_oracle():
    """First pass on Ls1 = 4 with mass 0.05, promotion to Ls = 8, one solve of
    (H + lam2) per vector to 1e-10, surface depth 2: the oracle's two-stage
    generation (its A-DEF2 second pass solved to 1e-10 too)."""
    torch = torch_or_skip()
    Ls, Ls1, nvec, seed, mass = 8, 4, 2, 1806, 0.01
    U = sy.gauge_field(DIMS, 0.4, 1807)
    d = DWF(DIMS, Ls, M5, B, C, mass, U)
    bl = Blocking(d, BLOCK)
    ref = two_pass_subspace(d, bl, nvec, seed, Ls1, 0.05, 0.05, 0.02, 1e-12, lam2=1e-2, tol2=1e-11, depth=2)
    h1 = _handle(torch, U, Ls1, 0.05)
    h1.build_subspace(BLOCK, nvec, prec=F64, inv_tol=1e-12, inv_maxiter=5000, seed=seed,
                      method=SUBSPACE_RATIONAL, filter_lambda=0.05, filter_eps=0.02)
    h = _handle(torch, U, Ls, mass)
    h.promote_subspace(h1, prec=F64)
    h.build_subspace(BLOCK, nvec, prec=F64, inv_steps=1, inv_shift=1e-2, inv_tol=1e-11, inv_maxiter=20000,
                     method=SUBSPACE_CONTINUE, surface_depth=2)
    assert rel(_get(h, Ls, nvec), ref) < 1e-6


def test_rational_filter_rejects_bad_parameters():
    torch = torch_or_skip()
    U = sy.gauge_field(DIMS, 0.4, 1808)
    h = _handle(torch, U, 4, 0.02)
    for kw in [dict(filter_order=0), dict(filter_order=9), dict(filter_eps=0.0), dict(filter_lambda=-1.0),
               dict(surface_depth=-1)]:
        args = dict(filter_lambda=0.05, filter_eps=0.02, filter_order=4, surface_depth=0)
        args.update(kw)
        with pytest.raises(RuntimeError):
            h.build_subspace(BLOCK, 2, prec=F32, seed=1, method=SUBSPACE_RATIONAL, **args)
    h2 = _handle(torch, U, 8, 0.02)
    with pytest.raises(RuntimeError):      # src without a subspace
        h.promote_subspace(h2)
    h2.build_subspace(BLOCK, 2, prec=F32, seed=1, method=SUBSPACE_RATIONAL, filter_lambda=0.05, filter_eps=0.02)
    with pytest.raises(RuntimeError):      # Ls1 = 8 > Ls = 4
        h.promote_subspace(h2)
