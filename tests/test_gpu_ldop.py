"""Second-level deflation of the little Dirac operator on the GPU (Sec. 5.2)
against the FP64 oracle, through the C ABI.

Both sides start from the same Gaussian vectors (splitmix64 stream, canonical
order), apply three steps of inverse iteration and the Rayleigh-Ritz
prediagonalisation to the same operator (rounded on the host to the storage
precision and uploaded with hdcg_set_coarse).  The GPU's vectors are FP32 and
its inner CG stops at 1e-6, so the converged low Ritz values agree to 1e-5
relative and the rest to 1e-3; all must interlace with the dense eigenvalues.
The A-DEF1 coarse solve is checked by its true residual (oracle stencil apply)
and against plain CG's iteration count; with a complete eigenbasis it is a
direct solve (one iteration).
"""
import numpy as np
import pytest

import synthetic as sy
from oracle.coarse import (Blocking, block_gram_schmidt, coarse_apply, coarse_dense_bruteforce, dense_to_stencil,
                           stencil_offsets, stencil_to_dense)
from oracle.dwf import DWF, norm2
from oracle.solvers import cg, ldop_deflation_space
from paper_1402_2585_gb300 import ALG_ADEF2, F16, F32, F64, Hdcg
from tests.gpu_util import rel, torch_or_skip

pytestmark = pytest.mark.gpu


def _round(A, prec):
    if prec == F16:
        return A.real.astype(np.float16).astype(np.float64) + 1j * A.imag.astype(np.float16).astype(np.float64)
    return A.astype(np.complex64).astype(np.complex128)


def _hpd_stencil(bl, n, seed, lam_min=0.01):
    """Seeded Hermitian positive definite 81-point stencil on a coarse grid with
    every extent >= 3: random couplings K and K^dag on opposite offsets, the
    diagonal shifted so that the lowest eigenvalue is lam_min."""
    K = sy.complex_normal(seed, (bl.Vc, 81, n, n)) * 0.02
    A = np.zeros_like(K)
    offs = stencil_offsets()
    for a in range(bl.Vc):
        for l in range(81):
            if l == 40:
                continue
            b = bl.neighbour_block(a, offs[l])
            A[a, l] += K[a, l]
            A[b, 80 - l] += K[a, l].conj().T
    Dn = stencil_to_dense(A, bl).reshape(bl.Vc * n, -1)
    shift = lam_min - np.linalg.eigvalsh(Dn)[0]
    A[:, 40] += shift * np.eye(n)
    return A


def _handle(dims, Ls, nvec, prec, A):
    torch = torch_or_skip()
    d = DWF(dims, Ls, 1.8, 1.0, 0.0, 0.05, sy.unit_gauge(dims))
    bl = Blocking(d, (4, 4, 4, 4))
    h = Hdcg(dims, Ls, stream=torch.cuda.current_stream().cuda_stream)
    h.set_dwf(1.8, 1.0, 0.0, 0.05)
    h.set_gauge(torch.from_numpy(d.U).cuda())
    phi = sy.gaussian_fermions(dims, Ls, 1300, nvec)
    h.set_subspace((4, 4, 4, 4), torch.from_numpy(phi).cuda(), prec=F32, already_orthonormal=True)
    if A is None:
        return torch, d, bl, h
    h.set_coarse(torch.from_numpy(A).cuda(), prec)
    return torch, d, bl, h


@pytest.fixture(scope="module")
def synthetic_op():
    dims, Ls, n = (12, 12, 12, 12), 2, 8
    d = DWF(dims, Ls, 1.8, 1.0, 0.0, 0.05, sy.unit_gauge(dims))
    bl = Blocking(d, (4, 4, 4, 4))
    return dims, Ls, n, _hpd_stencil(bl, n, 1310)


def _cvec(torch, X):
    return torch.view_as_real(torch.from_numpy(np.ascontiguousarray(X))).cuda().contiguous()


@pytest.mark.parametrize("prec", [F32, F16])
def test_ritz_values_match_oracle(synthetic_op, prec):
    dims, Ls, n, A0 = synthetic_op
    A = _round(A0, prec)
    torch, d, bl, h = _handle(dims, Ls, n, prec, A)
    nd, seed = 40, 1320          # three batches of the inner CG, the last one ragged
    h.build_coarse_deflation(nd, inv_steps=3, tol=1e-6, seed=seed)
    lam, Z = h.get_coarse_deflation(nd, vectors=True, shape=(nd, bl.Vc, n))
    noise = sy.complex_normal(seed, (nd, bl.Vc, n))
    _, _, lam_o = ldop_deflation_space(A, bl, noise, steps=3, tol=1e-10)
    lam_exact = np.linalg.eigvalsh(stencil_to_dense(A, bl).reshape(bl.Vc * n, -1))[:nd]
    assert np.all(np.abs(lam[:5] - lam_o[:5]) <= 1e-5 * lam_o[:5])
    assert np.all(np.abs(lam - lam_o) <= 1e-3 * lam_o)
    assert np.all(lam >= lam_exact * (1 - 1e-5))
    # the vectors are orthonormal and prediagonalise A
    Zf = Z.reshape(nd, -1)
    assert np.abs(Zf.conj() @ Zf.T - np.eye(nd)).max() < 1e-5
    AZ = np.array([coarse_apply(A, z, bl) for z in Z]).reshape(nd, -1)
    G = Zf.conj() @ AZ.T
    assert np.abs(G - np.diag(lam)).max() < 1e-5 * lam[-1]


@pytest.mark.parametrize("prec", [F32, F16])
def test_adef1_coarse_solve(synthetic_op, prec):
    """Three right-hand sides: A-DEF1 reaches the tolerance in the true
    residual and needs fewer iterations than plain CG on the same system."""
    dims, Ls, n, A0 = synthetic_op
    A = _round(A0, prec)
    torch, d, bl, h = _handle(dims, Ls, n, prec, A)
    B = sy.complex_normal(1330, (3, bl.Vc, n))
    bt = _cvec(torch, B)
    xt = torch.zeros_like(bt)
    it_cg = h.coarse_solve(bt, xt, 3, 1e-5)
    h.build_coarse_deflation(40, inv_steps=3, tol=1e-6, seed=1331)
    xt.zero_()
    it_d = h.coarse_solve(bt, xt, 3, 1e-5)
    X = torch.view_as_complex(xt.cpu()).numpy()
    for r in range(3):
        res = np.sqrt(norm2(B[r] - coarse_apply(A, X[r], bl)) / norm2(B[r]))
        assert res < 3e-5, f"rhs {r}: {res}"
    assert it_d < it_cg


def test_complete_eigenbasis_is_a_direct_solve():
    """A little Dirac operator of a 12x12x4x4, Ls 4 Mobius lattice (36 unknowns)
    with all 36 deflation vectors: Q = A^-1 and A-DEF1 stops after one iteration."""
    dims, Ls, n = (12, 12, 4, 4), 4, 4
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.01, sy.gauge_field(dims, 0.4, 1340))
    bl = Blocking(d, (4, 4, 4, 4))
    phi = block_gram_schmidt(sy.gaussian_fermions(dims, Ls, 1341, n), bl)
    A = _round(dense_to_stencil(coarse_dense_bruteforce(d.mdagm, phi, bl), bl), F32)
    torch, d2, bl2, h = _handle(dims, Ls, n, F32, A)
    h.build_coarse_deflation(bl.Vc * n, inv_steps=1, tol=1e-7, seed=1342)
    b = sy.complex_normal(1343, (1, bl.Vc, n))
    bt = _cvec(torch, b)
    xt = torch.zeros_like(bt)
    it = h.coarse_solve(bt, xt, 1, 1e-4)
    assert it == 1
    x = torch.view_as_complex(xt.cpu()).numpy()[0]
    xs = np.linalg.solve(stencil_to_dense(A, bl).reshape(bl.Vc * n, -1), b[0].ravel()).reshape(b[0].shape)
    assert rel(x, xs) < 1e-4


@pytest.mark.parametrize("coarse,nrhs", [(F32, 1), (F16, 1), (F16, 4)])
def test_hdcg_solve_with_deflated_coarse_solver(coarse, nrhs):
    """HDCG (A-DEF2 outside, A-DEF1 on the little Dirac operator) meets the
    true residual and agrees with the oracle's CG solution."""
    torch = torch_or_skip()
    dims, Ls = (8, 8, 4, 4), 4
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.01, sy.gauge_field(dims, 0.4, 800))
    bl = Blocking(d, (4, 4, 4, 4))
    from oracle.solvers import inverse_iteration_subspace
    phi = inverse_iteration_subspace(d.mdagm, sy.gaussian_fermions(dims, Ls, 801, 6), bl, steps=2, tol=1e-3)
    h = Hdcg(dims, Ls, stream=torch.cuda.current_stream().cuda_stream)
    h.set_dwf(d.M5, d.b, d.c, d.mass)
    h.set_gauge(torch.from_numpy(d.U).cuda())
    h.set_subspace((4, 4, 4, 4), torch.from_numpy(phi).cuda(), prec=F32, already_orthonormal=True)
    h.build_coarse(coarse)
    h.build_coarse_deflation(8, inv_steps=3, tol=1e-6, seed=1350)
    B = sy.gaussian_fermions(dims, Ls, 1351, nrhs)
    bt = torch.from_numpy(B).cuda()
    x = torch.zeros_like(bt)
    st = h.solve(bt, x, 1e-8, Hdcg.default_params(algorithm=ALG_ADEF2), nrhs=nrhs)
    assert st.status == 0
    X = x.cpu().numpy()
    for k in range(nrhs):
        assert np.sqrt(norm2(B[k] - d.mdagm(X[k])) / norm2(B[k])) <= 1.05e-8
        xk, _ = cg(d.mdagm, B[k], 1e-12)
        assert rel(X[k], xk) < 1e-5
