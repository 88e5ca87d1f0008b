"""Parity of the CUDA coarse level (through the C ABI) with the FP64 oracle:
block orthonormalisation, restriction, prolongation, the little Dirac operator
and its stencil apply.  Both sides use the same oracle-built subspace (uploaded
to the library), since the subspace itself is unique only up to block unitaries.

Tolerances: FP64 1e-11 (relative to the largest entry / L2 norm); FP32 1e-5
(sums over ~10^4 FP32 products); FP16 subspace storage 5e-3.
"""
import numpy as np
import pytest

import synthetic as sy
from oracle.coarse import (Blocking, block_gram_schmidt, coarse_apply, coarse_dense_bruteforce,
                           dense_to_stencil, prolong, restrict)
from oracle.dwf import DWF
from paper_1402_2585_gb300 import F16, F32, F64, Hdcg
from tests.gpu_util import from_gpu, rel, to_gpu, torch_or_skip

pytestmark = pytest.mark.gpu

TOL = {F64: 1e-11, F32: 1e-5, F16: 5e-3}

GEOMS = {
    # coarse (2,1,1,1): aliased extents
    "aliased_8x4x4x4_ls4": dict(dims=(8, 4, 4, 4), Ls=4, nvec=3, bc=(1.5, 0.5)),
    # coarse (3,3,1,2): extent 3 and 2 mixed, Shamir, Ls 8
    "mixed_12x12x4x8_ls8": dict(dims=(12, 12, 4, 8), Ls=8, nvec=4, bc=(1.0, 0.0)),
    # coarse (4,1,1,1): couplings beyond one hop vanish
    "long_16x4x4x4_ls4": dict(dims=(16, 4, 4, 4), Ls=4, nvec=2, bc=(1.5, 0.5)),
}


def _setup(geom, sub_prec, seed=0):
    torch = torch_or_skip()
    g = GEOMS[geom]
    dims, Ls = g["dims"], g["Ls"]
    U = sy.gauge_field(dims, 0.4, 700 + seed)
    d = DWF(dims, Ls, 1.8, g["bc"][0], g["bc"][1], 0.02, U)
    bl = Blocking(d, (4, 4, 4, 4))
    raw = sy.gaussian_fermions(dims, Ls, 710 + seed, g["nvec"])
    phi = block_gram_schmidt(raw, bl)
    h = Hdcg(dims, Ls, stream=torch.cuda.current_stream().cuda_stream)
    h.set_dwf(1.8, g["bc"][0], g["bc"][1], 0.02)
    h.set_gauge(torch.from_numpy(U).cuda())
    return torch, d, bl, raw, phi, h


@pytest.mark.parametrize("sub_prec", [F64, F32])
def test_block_orthonormalisation_matches_gram_schmidt(sub_prec):
    """The Q factor of the block QR (positive diagonal) is unique: CholQR2 on the
    GPU must reproduce the oracle's Gram-Schmidt."""
    torch, d, bl, raw, phi, h = _setup("aliased_8x4x4x4_ls4", sub_prec)
    h.set_subspace((4, 4, 4, 4), torch.from_numpy(raw).cuda(), prec=sub_prec, already_orthonormal=False)
    out = np.zeros_like(raw)
    h.get_subspace(out)
    assert rel(out, phi) < TOL[sub_prec] * 10


@pytest.mark.parametrize("geom", list(GEOMS))
@pytest.mark.parametrize("sub_prec", [F64, F32, F16])
def test_restrict_prolong(geom, sub_prec):
    torch, d, bl, raw, phi, h = _setup(geom, sub_prec)
    h.set_subspace((4, 4, 4, 4), torch.from_numpy(phi).cuda(), prec=sub_prec, already_orthonormal=True)
    v = sy.gaussian_fermion(d.lat.dims, d.Ls, 720)
    c = torch.zeros((bl.Vc, phi.shape[0], 2), dtype=torch.float64, device="cuda")
    h.restrict(to_gpu(v, F64), F64, c)
    assert rel(from_gpu(c), restrict(phi, v, bl)) < TOL[sub_prec]
    cv = sy.coarse_gaussian(bl.Vc, phi.shape[0], 721)
    out = torch.zeros(to_gpu(v, F32).shape, dtype=torch.float32, device="cuda")
    h.prolong(to_gpu(cv, F64), out, F32)
    assert rel(from_gpu(out), prolong(phi, cv, bl)) < max(TOL[sub_prec], 1e-6)


@pytest.mark.parametrize("geom", list(GEOMS))
@pytest.mark.parametrize("prec", [F64, F32])
def test_little_dirac_operator(geom, prec):
    """A from the Fourier trick on the GPU equals the oracle's brute force
    <phi_j^a | H | phi_k^b>; the stencil apply equals the oracle's."""
    torch, d, bl, raw, phi, h = _setup(geom, prec)
    h.set_subspace((4, 4, 4, 4), torch.from_numpy(phi).cuda(), prec=prec, already_orthonormal=True)
    h.build_coarse(prec)
    n = phi.shape[0]
    A = np.zeros((bl.Vc, 81, n, n), dtype=np.complex128)
    h.get_coarse(A)
    Ao = dense_to_stencil(coarse_dense_bruteforce(d.mdagm, phi, bl), bl)
    scale = np.abs(Ao).max()
    assert np.abs(A - Ao).max() < TOL[prec] * scale
    x = sy.coarse_gaussian(bl.Vc, n, 730)
    y = torch.zeros((bl.Vc, n, 2), dtype=torch.float64, device="cuda")
    h.coarse_apply(to_gpu(x, F64), y)
    assert rel(from_gpu(y), coarse_apply(Ao, x, bl)) < TOL[prec] * 10


def test_subspace_noise_is_the_published_generator():
    """With no inverse-iteration step the GPU subspace is block-GS of its Gaussian
    start vectors, which must be splitmix64 + Box-Muller in canonical order."""
    torch, d, bl, raw, phi, h = _setup("aliased_8x4x4x4_ls4", F64)
    seed = 12345
    h.build_subspace((4, 4, 4, 4), 3, F64, inv_steps=0, seed=seed)
    out = np.zeros((3,) + d.field_shape, dtype=np.complex128)
    h.get_subspace(out)
    noise = sy.complex_normal(seed, (3,) + d.field_shape)
    assert rel(out, block_gram_schmidt(noise, bl)) < 1e-11


def test_inverse_iteration_subspace_properties():
    torch, d, bl, raw, phi, h = _setup("aliased_8x4x4x4_ls4", F32)
    h.build_subspace((4, 4, 4, 4), 3, F32, inv_steps=2, inv_tol=1e-3, seed=99)
    out = np.zeros((3,) + d.field_shape, dtype=np.complex128)
    h.get_subspace(out)
    for sites in bl.sites_of_block:
        X = out[:, sites].reshape(3, -1)
        assert np.abs(np.conj(X) @ X.T - np.eye(3)).max() < 1e-5
    rq = [np.vdot(v, d.mdagm(v)).real / np.vdot(v, v).real for v in out]
    rq0 = [np.vdot(v, d.mdagm(v)).real / np.vdot(v, v).real for v in raw]
    assert max(rq) < 0.05 * min(rq0)
