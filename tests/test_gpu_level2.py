"""The blocked second coarsening (three-level HDCG) through the C ABI, against
the FP64 oracle (oracle/level2.py, oracle/coarse.py, oracle/solvers.py).

The level-1 operator is the little Dirac operator of a small domain wall
problem, built on the GPU (inverse-iteration subspace, Fourier assembly,
stored FP32) and read back exactly with hdcg_get_coarse, so the oracle works
on the very matrix the GPU holds.  The level-2 vectors are uploaded
(hdcg_set_subspace, level 2) where the oracle must use the same ones, or
generated on the GPU where a property test says so.

Bars: A2 = P2^dag A P2 is contracted in FP64 from FP32 inputs on both sides,
so it agrees to FP64 rounding (1e-11 relative).  R2, P2 and the level-1
vectors are FP32 on the GPU: 1e-6.  The level-1 operator runs on the tensor
cores as FP16 hi + lo parts (about 2^-22 relative per product), so a level-1
solution to tol agrees with numpy's dense solution within
kappa(A) (tol + 5e-7), kappa from numpy's eigenvalues.
"""
import numpy as np
import pytest

import synthetic as sy
from oracle.coarse import (Blocking, block_gram_schmidt, coarse_apply, coarse_dense_bruteforce, dense_to_stencil,
                           prolong, restrict, stencil_to_dense)
from oracle.dwf import DWF, norm2
from oracle.level2 import CoarseBlocking
from oracle.solvers import cg
from paper_1402_2585_gb300 import ALG_ADEF2, F16, F32, F64, Hdcg
from tests.gpu_util import from_gpu, rel, to_gpu, torch_or_skip, cg_kappa

pytestmark = pytest.mark.gpu

# fine lattice, Ls, fine blocks -> coarse lattice; level-2 blocks -> level-2 lattice
GEOMS = {
    # coarse (6, 6, 4, 4): no aliasing at level 1; level 2 (3, 3, 2, 2): extents 2 alias
    "c6x6x4x4_l2_2222": dict(dims=(24, 24, 16, 16), Ls=4, block=(4, 4, 4, 4), block2=(2, 2, 2, 2)),
    # coarse (4, 4, 2, 2): level-1 extents 2 alias; level 2 (2, 4, 2, 1): an extent of 1
    "c4x4x2x2_l2_2112": dict(dims=(16, 16, 8, 8), Ls=4, block=(4, 4, 4, 4), block2=(2, 1, 1, 2)),
}
N1, N2 = 4, 3


def _handle(torch, d):
    h = Hdcg(d.lat.dims, d.Ls, stream=torch.cuda.current_stream().cuda_stream)
    h.set_dwf(d.M5, d.b, d.c, d.mass)
    h.set_gauge(torch.from_numpy(d.U).cuda())
    return h


@pytest.fixture(scope="module", params=list(GEOMS))
def setup(request):
    torch = torch_or_skip()
    g = GEOMS[request.param]
    dims, Ls = g["dims"], g["Ls"]
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.01, sy.gauge_field(dims, 0.4, 3099))
    bl = Blocking(d, g["block"])
    lat = CoarseBlocking(bl.coarse_dims, (1, 1, 1, 1))
    cb = CoarseBlocking(bl.coarse_dims, g["block2"])
    h = _handle(torch, d)
    h.build_subspace(g["block"], N1, F32, inv_steps=2, inv_tol=1e-3, seed=3102)
    h.build_coarse(F32)
    A1 = np.zeros((lat.Vc, 81, N1, N1), dtype=np.complex128)
    h.get_coarse(A1)
    raw2 = sy.complex_normal(3101, (N2, lat.Vc, N1))
    phi2 = block_gram_schmidt(raw2, cb).astype(np.complex64).astype(np.complex128)
    h.set_subspace(g["block2"], phi2, prec=F32, already_orthonormal=True, level=2)

    def apply_A1(v):
        return coarse_apply(A1, v, lat)

    A2 = dense_to_stencil(coarse_dense_bruteforce(apply_A1, phi2, cb), cb)
    yield torch, h, d, g, lat, cb, A1, raw2, phi2, A2, apply_A1
    h.close()


def test_level2_operator_is_the_galerkin_product(setup):
    torch, h, d, g, lat, cb, A1, raw2, phi2, A2, apply_A1 = setup
    h.build_coarse(F32, level=2)
    got = np.zeros((cb.Vc, 81, N2, N2), dtype=np.complex128)
    h.get_coarse(got, level=2)
    assert rel(got, A2) < 1e-11


def test_restrict_and_prolong_level2(setup):
    torch, h, d, g, lat, cb, A1, raw2, phi2, A2, apply_A1 = setup
    R = 3
    x = sy.complex_normal(3103, (R, lat.Vc, N1))
    c2 = torch.zeros((R, cb.Vc, N2, 2), dtype=torch.float64, device="cuda")
    h.restrict_coarse(to_gpu(x, F64), c2, R)
    want = np.stack([restrict(phi2, x[r], cb) for r in range(R)])
    assert rel(from_gpu(c2), want) < 1e-6
    cc = sy.complex_normal(3104, (R, cb.Vc, N2))
    y = torch.zeros((R, lat.Vc, N1, 2), dtype=torch.float64, device="cuda")
    h.prolong_coarse(to_gpu(cc, F64), y, R)
    want = np.stack([prolong(phi2, cc[r], cb) for r in range(R)])
    assert rel(from_gpu(y), want) < 1e-6


def test_level2_block_orthonormalisation_is_the_gram_schmidt_q(setup):
    """CholQR2 on the GPU and modified Gram-Schmidt in the oracle give the same
    unique Q (positive diagonal R) of every level-2 block."""
    torch, h, d, g, lat, cb, A1, raw2, phi2, A2, apply_A1 = setup
    torch_h = _handle(torch, d)
    torch_h.build_subspace(g["block"], N1, F32, inv_steps=0, seed=3102)
    torch_h.set_coarse(A1, prec=F32)
    torch_h.set_subspace(g["block2"], raw2, prec=F32, already_orthonormal=False, level=2)
    got = np.zeros_like(raw2)
    torch_h.get_subspace(got, level=2)
    want = block_gram_schmidt(raw2, cb)
    assert rel(got, want) < 1e-5
    for sites in cb.sites_of_block:
        X = got[:, sites].reshape(N2, -1)
        assert np.abs(X.conj() @ X.T - np.eye(N2)).max() < 1e-6
    torch_h.close()


@pytest.mark.parametrize("inv_prec,tol", [(F64, 1e-6), (F32, 1e-5)])
def test_q2_is_p2_a2_inverse_r2(setup, inv_prec, tol):
    """With a tolerance the start vector already meets, the level-1 solve
    returns its A-DEF2 start x0 = Q2 b = P2 A2^-1 R2 b: the dense level-2
    inverse against numpy's solve of the oracle's A2."""
    torch, h, d, g, lat, cb, A1, raw2, phi2, A2, apply_A1 = setup
    h.build_coarse(inv_prec, level=2)
    R = 2
    b = sy.complex_normal(3105, (R, lat.Vc, N1))
    x = torch.zeros((R, lat.Vc, N1, 2), dtype=torch.float64, device="cuda")
    its = h.coarse_solve(to_gpu(b, F64), x, R, 1e30)
    assert its == 0
    D2 = stencil_to_dense(A2, cb).reshape(cb.Vc * N2, -1)
    want = np.stack([prolong(phi2, np.linalg.solve(D2, restrict(phi2, b[r], cb).ravel()).reshape(cb.Vc, N2), cb)
                     for r in range(R)])
    assert rel(from_gpu(x), want) < tol


def test_level1_adef2_solve(setup):
    """A-DEF2 with Q2 (level-2 vectors from inverse iteration on A) meets numpy's
    dense solution in fewer iterations than the plain coarse CG."""
    torch, h, d, g, lat, cb, A1, raw2, phi2, A2, apply_A1 = setup
    R, tol = 3, 1e-7
    b = sy.complex_normal(3106, (R, lat.Vc, N1))
    D1 = stencil_to_dense(A1, lat).reshape(lat.Vc * N1, -1)
    ev = np.linalg.eigvalsh(0.5 * (D1 + D1.conj().T))
    kappa = ev[-1] / ev[0]
    xs = np.stack([np.linalg.solve(D1, b[r].ravel()).reshape(lat.Vc, N1) for r in range(R)])
    # plain coarse CG first: a fresh level-1 operator drops the level-2 operator
    h.set_coarse(A1, prec=F32)
    x = torch.zeros((R, lat.Vc, N1, 2), dtype=torch.float64, device="cuda")
    it_cg = h.coarse_solve(to_gpu(b, F64), x, R, tol)
    assert rel(from_gpu(x), xs) < kappa * (tol + 5e-7)
    h.build_subspace(g["block2"], N2, F32, inv_steps=2, inv_tol=1e-5, seed=3108, level=2)
    h.build_coarse(F32, level=2)
    x = torch.zeros((R, lat.Vc, N1, 2), dtype=torch.float64, device="cuda")
    it = h.coarse_solve(to_gpu(b, F64), x, R, tol)
    assert rel(from_gpu(x), xs) < kappa * (tol + 5e-7)
    assert it < it_cg


def test_level2_subspace_by_inverse_iteration(setup):
    """hdcg_build_subspace at level 2: block-orthonormal vectors whose Rayleigh
    quotients lie far below those of the Gaussian start vectors."""
    torch, h, d, g, lat, cb, A1, raw2, phi2, A2, apply_A1 = setup
    h.set_coarse(A1, prec=F32)
    h.build_subspace(g["block2"], N2, F32, inv_steps=3, inv_tol=1e-6, seed=3107, level=2)
    got = np.zeros((N2, lat.Vc, N1), dtype=np.complex128)
    h.get_subspace(got, level=2)
    for sites in cb.sites_of_block:
        X = got[:, sites].reshape(N2, -1)
        assert np.abs(X.conj() @ X.T - np.eye(N2)).max() < 1e-5

    def rq(v):
        return float(np.vdot(v, apply_A1(v)).real / norm2(v))

    noise = sy.complex_normal(3107, (N2, lat.Vc, N1))
    assert max(rq(v) for v in got) < 0.5 * min(rq(v) for v in noise)
    # the vectors are the generator's stream followed by (A)^-1 steps: a fresh
    # build with the same seed reproduces them
    h.build_subspace(g["block2"], N2, F32, inv_steps=3, inv_tol=1e-6, seed=3107, level=2)
    again = np.zeros_like(got)
    h.get_subspace(again, level=2)
    assert np.array_equal(again, got)


_SOLUTIONS = {}


def _oracle_solution(d, b):
    """The oracle's CG solution (to 1e-13) and kappa, computed once per module."""
    key = (d.lat.dims, d.Ls)
    if key not in _SOLUTIONS:
        _SOLUTIONS[key] = cg_kappa(d.mdagm, b, 1e-13)
    return _SOLUTIONS[key]




@pytest.mark.parametrize("coarse_prec", [F32, F16])
def test_three_level_hdcg_meets_the_oracle_solution(coarse_prec):
    """HDCG with three levels on a domain wall problem (16x8x8x8, Ls 4 Moebius,
    m 0.01): the fine subspace and its FP32 or FP16 little Dirac operator, a
    level-2 subspace from inverse iteration on it, FP32 outer and FP16 sloppy
    operator.
    The solution agrees with the oracle's CG solution to 1e-6: the GPU solves
    to min(1e-8, 0.5e-6 / kappa), kappa from the Lanczos tridiagonal of the
    oracle's CG, so |x - x*| / |x*| <= kappa |r| / |b| <= 0.5e-6."""
    torch = torch_or_skip()
    dims, Ls = (16, 8, 8, 8), 4
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.01, sy.gauge_field(dims, 0.4, 3200))
    b = sy.gaussian_fermion(dims, Ls, 3201)
    xs, kappa = _oracle_solution(d, b)
    tol = min(1e-8, 0.5e-6 / kappa)
    h = _handle(torch, d)
    h.build_subspace((4, 4, 4, 4), 8, F16, inv_steps=2, inv_tol=1e-3, seed=3202)
    h.build_coarse(coarse_prec)
    h.build_subspace((2, 1, 1, 1), 4, F32, inv_steps=2, inv_tol=1e-4, seed=3203, level=2)
    h.build_coarse(F32, level=2)
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    st = h.solve(bt, x, tol, Hdcg.default_params(algorithm=ALG_ADEF2, outer_prec=F32, sloppy_prec=F16))
    assert st.status == 0
    xg = x.cpu().numpy()
    assert np.sqrt(norm2(b - d.mdagm(xg)) / norm2(b)) <= 1.05 * tol
    assert rel(xg, xs) <= 1e-6
    h.close()


# ---------------------------------------------------------------------------
# the high-mode preconditioner of Sec. 5.2: Chebyshev polynomial of Q_trunc
# ---------------------------------------------------------------------------

def test_qtrunc_chebyshev_against_the_oracle(setup):
    """hdcg_coarse_precondition against the oracle's qtrunc_chebyshev (the
    truncated stencil, the same interval [lo, hi], order 16): FP32 vectors and
    15 products with Q_trunc: 1e-5.  The interval the library estimated bounds
    the spectrum of Q_trunc (numpy's eigenvalues of the oracle's truncation)."""
    from oracle.solvers import qtrunc_chebyshev, truncate_stencil
    torch, h, d, g, lat, cb, A1, raw2, phi2, A2, apply_A1 = setup
    h.set_coarse(A1, prec=F32)
    lo, hi = h.set_coarse_preconditioner(16)
    T = stencil_to_dense(truncate_stencil(A1, 1), lat).reshape(lat.Vc * N1, -1)
    ev = np.linalg.eigvalsh(0.5 * (T + T.conj().T))
    assert ev[-1] < hi < 1.3 * ev[-1] and lo == pytest.approx(hi / 90)
    M = qtrunc_chebyshev(A1, lat, 16, lo, hi)
    R = 3
    x = sy.complex_normal(3110, (R, lat.Vc, N1))
    y = torch.zeros((R, lat.Vc, N1, 2), dtype=torch.float64, device="cuda")
    h.coarse_precondition(to_gpu(x, F64), y, R)
    want = np.stack([M(x[r]) for r in range(R)])
    assert rel(from_gpu(y), want) < 1e-5
    h.set_coarse_preconditioner(0)


def test_level1_solve_with_the_qtrunc_smoother(setup):
    """The level-1 A-DEF2 solve smoothed by M = p(Q_trunc): it meets numpy's
    dense solution (kappa-bound as above) in no more iterations than with
    M = 1."""
    torch, h, d, g, lat, cb, A1, raw2, phi2, A2, apply_A1 = setup
    R, tol = 2, 1e-7
    b = sy.complex_normal(3111, (R, lat.Vc, N1))
    D1 = stencil_to_dense(A1, lat).reshape(lat.Vc * N1, -1)
    ev = np.linalg.eigvalsh(0.5 * (D1 + D1.conj().T))
    kappa = ev[-1] / ev[0]
    xs = np.stack([np.linalg.solve(D1, b[r].ravel()).reshape(lat.Vc, N1) for r in range(R)])
    h.set_coarse(A1, prec=F32)
    h.build_subspace(g["block2"], N2, F32, inv_steps=2, inv_tol=1e-5, seed=3112, level=2)
    h.build_coarse(F32, level=2)
    x = torch.zeros((R, lat.Vc, N1, 2), dtype=torch.float64, device="cuda")
    it1 = h.coarse_solve(to_gpu(b, F64), x, R, tol)
    h.set_coarse_preconditioner(16)
    x = torch.zeros((R, lat.Vc, N1, 2), dtype=torch.float64, device="cuda")
    itm = h.coarse_solve(to_gpu(b, F64), x, R, tol)
    assert rel(from_gpu(x), xs) < kappa * (tol + 5e-7)
    assert itm <= it1
    h.set_coarse_preconditioner(0)
