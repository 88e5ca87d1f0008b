"""The little Dirac operator applied to several right-hand sides at once
(hdcg_coarse_apply_multi): FP16 operators on the tensor cores (tcgen05), FP32
operators on the tensor cores as FP16 hi + lo parts, FP64 operators on the
CUDA cores, against the FP64 oracle's stencil apply
y_a = sum_l A[a][l] x_{a+delta_l} (Sec. 5.1).

The operator is a seeded random stencil rounded to the storage precision on
the host (numpy) and uploaded with hdcg_set_coarse, so both sides apply the
same matrix.  What remains on the GPU is the rounding of X (FP32, then an
FP16 hi + lo pair after a power-of-two scale per right-hand side, about 2^-22
relative to the largest entry) and FP32 accumulation over 81 Nvec products:
relative L2 error per right-hand side below 1e-5 (measured ~1e-7 in the CPU
emulation of the kernel's arithmetic).  FP64 operators: 1e-12.
"""
import numpy as np
import pytest

import synthetic as sy
from oracle.coarse import Blocking, canonical_offsets, coarse_apply, stencil_offsets
from oracle.dwf import DWF
from paper_1402_2585_gb300 import F16, F32, F64, Hdcg, HdcgError
from tests.gpu_util import rel, torch_or_skip

pytestmark = pytest.mark.gpu

GEOMS = {
    # coarse (3,1,1,1): odd number of coarse sites, aliased extents
    "odd_12x4x4x4_ls4": dict(dims=(12, 4, 4, 4), Ls=4),
    # coarse (3,3,3,3): all 81 offsets distinct, Vc = 81
    "full_12x12x12x12_ls2": dict(dims=(12, 12, 12, 12), Ls=2),
}


def _round(A, prec):
    if prec == F16:
        return A.real.astype(np.float16).astype(np.float64) + 1j * A.imag.astype(np.float16).astype(np.float64)
    if prec == F32:
        return A.astype(np.complex64).astype(np.complex128)
    return A


def _random_stencil(bl, nvec, seed, prec):
    """Seeded complex Gaussian stencil, zero on the offsets a coarse extent <= 2
    does not store, rounded to the storage precision."""
    A = sy.complex_normal(seed, (bl.Vc, 81, nvec, nvec)) / np.sqrt(81 * nvec)
    offs = stencil_offsets()
    keep = [canonical_offsets(bl.coarse_dims, mu) for mu in range(4)]
    for l in range(81):
        if not all(offs[l, mu] in keep[mu] for mu in range(4)):
            A[:, l] = 0
    return _round(A, prec)


def _handle(geom, nvec, prec, seed=0):
    torch = torch_or_skip()
    g = GEOMS[geom]
    dims, Ls = g["dims"], g["Ls"]
    d = DWF(dims, Ls, 1.8, 1.0, 0.0, 0.05, sy.unit_gauge(dims))
    bl = Blocking(d, (4, 4, 4, 4))
    h = Hdcg(dims, Ls, stream=torch.cuda.current_stream().cuda_stream)
    h.set_dwf(1.8, 1.0, 0.0, 0.05)
    h.set_gauge(torch.from_numpy(d.U).cuda())
    # the subspace only fixes the blocking and Nvec here
    phi = sy.gaussian_fermions(dims, Ls, 900 + seed, nvec)
    h.set_subspace((4, 4, 4, 4), torch.from_numpy(phi).cuda(), prec=F64 if prec == F64 else F32,
                   already_orthonormal=True)
    A = _random_stencil(bl, nvec, 910 + seed, prec)
    h.set_coarse(torch.from_numpy(A).cuda(), prec)
    return torch, bl, h, A


def _multi(torch, h, X):
    xt = torch.view_as_real(torch.from_numpy(np.ascontiguousarray(X))).cuda().contiguous()
    yt = torch.zeros_like(xt)
    h.coarse_apply_multi(xt, yt, X.shape[0])
    return torch.view_as_complex(yt.cpu()).numpy()


@pytest.mark.parametrize("geom", list(GEOMS))
@pytest.mark.parametrize("nvec", [32, 40, 6])
@pytest.mark.parametrize("R", [1, 3, 12, 16])
def test_tensor_core_multi_apply(geom, nvec, R):
    """Two coarse sites per M = 128 MMA (Nvec 32, 6) and one site (Nvec 40);
    padded K (Nvec 6, 40); ragged site pair (Vc odd); N = 8 Rp from 16 to 128."""
    torch, bl, h, A = _handle(geom, nvec, F16)
    X = sy.complex_normal(920 + R, (R, bl.Vc, nvec))
    Y = _multi(torch, h, X)
    for r in range(R):
        assert rel(Y[r], coarse_apply(A, X[r], bl)) < 1e-5, f"rhs {r}"


def test_tensor_core_per_rhs_scaling():
    """Right-hand sides 30 orders of magnitude apart in one launch: each is
    scaled by its own power of two before the FP16 split, so every one keeps
    its relative accuracy; a zero right-hand side gives exactly zero."""
    torch, bl, h, A = _handle("full_12x12x12x12_ls2", 32, F16)
    X = sy.complex_normal(930, (4, bl.Vc, 32))
    X[0] *= 1e-25
    X[1] *= 1e20
    X[3] = 0
    Y = _multi(torch, h, X)
    for r in range(3):
        assert rel(Y[r], coarse_apply(A, X[r], bl)) < 1e-5, f"rhs {r}"
    assert np.all(Y[3] == 0)


@pytest.mark.parametrize("prec,tol", [(F32, 1e-5), (F64, 1e-12)])
def test_fp32_split_and_fp64_multi_apply(prec, tol):
    torch, bl, h, A = _handle("full_12x12x12x12_ls2", 24, prec)
    X = sy.complex_normal(940, (5, bl.Vc, 24))
    Y = _multi(torch, h, X)
    for r in range(5):
        assert rel(Y[r], coarse_apply(A, X[r], bl)) < tol, f"rhs {r}"


@pytest.mark.parametrize("R", [1, 16])
def test_fp32_operator_with_hop_dependent_magnitudes(R):
    """Couplings falling with the block hop distance like the paper's Table
    frobnorm (627, 6.2, 0.08, 7e-4, 3e-5 for 0..4 hops): the per-site scale
    keeps the small far blocks in FP16's normal range, and the hi + lo split
    keeps the FP32 operator's accuracy.  x lives on one coarse site, so the
    sites two or more hops away see only the small blocks; their error is
    measured against the output's overall size (the operator's own scale)."""
    torch, bl, h, A = _handle("full_12x12x12x12_ls2", 32, F32)
    offs = np.array([[(l // 3 ** mu) % 3 - 1 for mu in range(4)] for l in range(81)])
    hops = np.abs(offs).sum(axis=1)
    frob = np.array([627.0, 6.2, 0.08, 7e-4, 3e-5])
    A = (A * (frob[hops] / frob[0])[None, :, None, None]).astype(np.complex64).astype(np.complex128)
    h.set_coarse(torch.from_numpy(A).cuda(), F32)
    X = np.zeros((R, bl.Vc, 32), dtype=np.complex128)
    X[:, 40] = sy.complex_normal(961, (R, 32))
    Y = _multi(torch, h, X)
    for r in range(R):
        want = coarse_apply(A, X[r], bl)
        assert rel(Y[r], want) < 1e-5
        far = [a for a in range(bl.Vc) if np.abs(offs[a] - offs[40]).sum() >= 2]
        err = np.abs(Y[r][far] - want[far]).max() / np.abs(want).max()
        assert err < 1e-6, err


@pytest.mark.parametrize("prec", [F16, F32, F64])
def test_set_coarse_roundtrip_and_single_apply(prec):
    """hdcg_set_coarse stores exactly the rounded operator (get_coarse gives it
    back bit for bit); the single-vector apply agrees with the oracle too."""
    torch, bl, h, A = _handle("odd_12x4x4x4_ls4", 8, prec)
    out = np.zeros_like(A)
    h.get_coarse(out)
    assert np.array_equal(out, A)
    x = sy.coarse_gaussian(bl.Vc, 8, 950)
    xt = torch.view_as_real(torch.from_numpy(x)).cuda().contiguous()
    yt = torch.zeros_like(xt)
    h.coarse_apply(xt, yt)
    y = torch.view_as_complex(yt.cpu()).numpy()
    assert rel(y, coarse_apply(A, x, bl)) < (1e-12 if prec == F64 else 1e-5)


def test_set_coarse_and_multi_apply_errors():
    torch = torch_or_skip()
    h = Hdcg((8, 8, 4, 4), 4, stream=torch.cuda.current_stream().cuda_stream)
    A = torch.zeros((4, 81, 2, 2, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(HdcgError) as e:
        h.set_coarse(A, F16)
    assert e.value.code == -7           # no subspace yet
    torch_, bl, h2, A2 = _handle("odd_12x4x4x4_ls4", 8, F16)
    x = torch.zeros((17, bl.Vc, 8, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(HdcgError) as e:
        h2.coarse_apply_multi(x, torch.zeros_like(x), 17)
    assert e.value.code == -1           # at most 16 right-hand sides


@pytest.mark.parametrize("nvec,prec", [(40, F32), (24, F16), (64, F16)])
def test_persistent_shapes_give_identical_results(nvec, prec):
    """One and two persistent CTAs per SM (ring depths 192 KB and 96 KB) run the
    same MMAs in the same order: bit-identical outputs, both equal to the
    oracle's apply; the autotuned default gives the same bits again."""
    torch, bl, h, A = _handle("full_12x12x12x12_ls2", nvec, prec)
    X = sy.complex_normal(940 + nvec, (12, bl.Vc, nvec))
    out = {}
    for shape in (1, 2, 0):
        h.set_coarse_tc_shape(shape)
        out[shape] = _multi(torch, h, X)
    assert np.array_equal(out[1], out[2]) and np.array_equal(out[0], out[2])
    for r in range(12):
        assert rel(out[2][r], coarse_apply(A, X[r], bl)) < 1e-5, f"rhs {r}"
    with pytest.raises(HdcgError):
        h.set_coarse_tc_shape(3)
