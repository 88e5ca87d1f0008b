"""Solves through the C ABI, checked by the FP64 oracle.

The oracle recomputes every true residual |b - H x| / |b| in FP64 from the
GPU's solution, and compares the solution with its own CG solution x* (to
1e-13).  Solution agreement is held to relative L2 1e-6: each solve runs to
the residual min(1e-8, 0.5e-6 / kappa), kappa = lambda_max / lambda_min of H
from the Lanczos tridiagonal of the oracle's CG (about 460 on the 8x8x4x4
lattice, 2.8e4 on the 8^4 x 8 workload), so |x - x*| / |x*| <= kappa |r| / |b|
<= 0.5e-6.
"""
import numpy as np
import pytest

import synthetic as sy
from oracle.coarse import Blocking
from oracle.dwf import DWF, norm2
from oracle.solvers import cg, inverse_iteration_subspace
from paper_1402_2585_gb300 import ALG_ADEF2, ALG_CG, F16, F32, F64, Hdcg, HdcgError
from tests.gpu_util import cg_kappa, kappa_tol, rel, torch_or_skip

pytestmark = pytest.mark.gpu


def _true_res(d, b, x):
    return float(np.sqrt(norm2(b - d.mdagm(x)) / norm2(b)))


def _handle(d, torch, apbc=False):
    h = Hdcg(d.lat.dims, d.Ls, antiperiodic_t=apbc, stream=torch.cuda.current_stream().cuda_stream)
    h.set_dwf(d.M5, d.b, d.c, d.mass)
    h.set_gauge(torch.from_numpy(d.U).cuda())
    return h


@pytest.fixture(scope="module")
def small():
    torch = torch_or_skip()
    dims, Ls = (8, 8, 4, 4), 4
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.01, sy.gauge_field(dims, 0.4, 800))
    bl = Blocking(d, (4, 4, 4, 4))
    phi = inverse_iteration_subspace(d.mdagm, sy.gaussian_fermions(dims, Ls, 801, 6), bl, steps=2, tol=1e-3)
    b = sy.gaussian_fermion(dims, Ls, 802)
    xs, kappa = cg_kappa(d.mdagm, b, 1e-13)
    assert 100 < kappa < 1e4
    _KAPPA[id(d)] = kappa
    return torch, d, bl, phi, b, xs


_KAPPA = {}


def _tol(small, outer):
    """min(1e-8, 0.5e-6 / kappa), and 1e-10 at most for an FP64 outer solve."""
    return min(kappa_tol(_KAPPA[id(small[1])]), 1e-10 if outer == F64 else 1.0)


@pytest.mark.parametrize("outer", [F64, F32])
def test_plain_cg(small, outer):
    torch, d, bl, phi, b, xs = small
    tol = _tol(small, outer)
    h = _handle(d, torch)
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    st = h.solve(bt, x, tol, Hdcg.default_params(algorithm=ALG_CG, outer_prec=outer, maxiter=20000))
    assert st.status == 0
    xg = x.cpu().numpy()
    assert _true_res(d, b, xg) <= 1.05 * tol
    assert st.true_residual <= tol
    assert rel(xg, xs) < 1e-6
    if outer == F32:
        assert st.reliable_updates >= 2


@pytest.mark.parametrize("outer,sloppy,prec_sub,coarse", [
    (F64, F64, F64, F64),
    (F32, F32, F32, F32),
    (F32, F16, F32, F32),
    (F32, F16, F16, F32),
    (F32, F16, F16, F16),
])
def test_adef2_with_oracle_subspace(small, outer, sloppy, prec_sub, coarse):
    torch, d, bl, phi, b, xs = small
    tol = _tol(small, outer)
    h = _handle(d, torch)
    h.set_subspace((4, 4, 4, 4), torch.from_numpy(phi).cuda(), prec=prec_sub, already_orthonormal=True)
    h.build_coarse(coarse)
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    st = h.solve(bt, x, tol, Hdcg.default_params(algorithm=ALG_ADEF2, outer_prec=outer, sloppy_prec=sloppy))
    assert st.status == 0
    xg = x.cpu().numpy()
    assert _true_res(d, b, xg) <= 1.05 * tol
    assert rel(xg, xs) < 1e-6
    # fewer outer iterations than plain CG (oracle CG count at the same tolerance)
    hist = []
    cg(d.mdagm, b, tol, history=hist)
    assert st.iterations < len(hist)


def test_host_buffers_equal_device_buffers(small):
    torch, d, bl, phi, b, xs = small
    h = _handle(d, torch)
    prm = Hdcg.default_params(algorithm=ALG_CG, outer_prec=F64)
    bt = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bt)
    h.solve(bt, xd, 1e-9, prm)
    xh = np.zeros_like(b)
    h.solve(b, xh, 1e-9, prm)
    assert np.array_equal(xd.cpu().numpy(), xh)


def test_zero_source_and_errors(small):
    torch, d, bl, phi, b, xs = small
    h = _handle(d, torch)
    z = torch.zeros(d.field_shape, dtype=torch.complex128, device="cuda")
    x = torch.ones_like(z)
    st = h.solve(z, x, 1e-8, Hdcg.default_params(algorithm=ALG_CG))
    assert st.status == 0 and float(x.abs().max()) == 0.0
    with pytest.raises(HdcgError) as e:
        h.solve(z + 1, x, 1e-8, Hdcg.default_params(algorithm=ALG_ADEF2))
    assert e.value.code == -7          # no subspace / coarse operator
    with pytest.raises(HdcgError):
        h.solve(z, x, -1.0, Hdcg.default_params(algorithm=ALG_CG))


def test_two_level_workload_8x8x8x8_ls8_fp64():
    """The plain-FP64 workload: 8^4 x 8 Shamir, M5 1.8, m 0.01, eps 0.3, 4^4
    blocks, Nvec 8 by inverse iteration.  HDCG and plain CG reach the oracle's
    solution to 1e-6 (solved to 0.5e-6 / kappa, kappa about 2.8e4); the oracle
    certifies both true residuals."""
    torch = torch_or_skip()
    w = sy.WORKLOADS["cfg1_8x8x8x8_ls8_shamir"]
    d = DWF(w.dims, w.Ls, w.M5, w.b, w.c, w.mass, sy.gauge_field(w.dims, w.eps, w.gauge_seed))
    h = _handle(d, torch)
    h.build_subspace(w.block, w.nvec, F64, inv_steps=3, inv_tol=1e-4, seed=w.subspace_seed)
    h.build_coarse(F64)
    b = sy.gaussian_fermion(w.dims, w.Ls, w.source_seed)
    xs, kappa = cg_kappa(d.mdagm, b, 1e-13)
    tol = min(w.tol, kappa_tol(kappa))
    bt = torch.from_numpy(b).cuda()
    x1, x2 = torch.zeros_like(bt), torch.zeros_like(bt)
    s1 = h.solve(bt, x1, tol, Hdcg.default_params(algorithm=ALG_ADEF2, outer_prec=F64, sloppy_prec=F64))
    s2 = h.solve(bt, x2, tol, Hdcg.default_params(algorithm=ALG_CG, outer_prec=F64, maxiter=50000))
    a, c = x1.cpu().numpy(), x2.cpu().numpy()
    assert s1.status == 0 and s2.status == 0
    assert _true_res(d, b, a) <= 1.05 * tol
    assert _true_res(d, b, c) <= 1.05 * tol
    assert rel(a, xs) < 1e-6
    assert rel(c, xs) < 1e-6
    assert s1.iterations < s2.iterations


def _sources(d, n, seed):
    """n right-hand sides of uneven difficulty: Gaussian ones and point sources."""
    out = []
    for k in range(n):
        if k % 3 == 2:
            b = np.zeros(d.field_shape, dtype=np.complex128)
            b[(7 * k) % d.field_shape[0], 0, k % 4, k % 3] = 1.0
            b[(7 * k) % d.field_shape[0], d.Ls - 1, (k + 2) % 4, k % 3] = 1.0
        else:
            b = sy.gaussian_fermion(d.lat.dims, d.Ls, seed + k)
        out.append(b)
    return np.stack(out)


@pytest.mark.parametrize("alg,outer,sloppy,nrhs,coarse", [
    (ALG_ADEF2, F32, F32, 4, F32),
    (ALG_ADEF2, F32, F16, 5, F32),
    (ALG_ADEF2, F32, F16, 5, F16),
    (ALG_ADEF2, F32, F32, 16, F16),
    (ALG_CG, F32, F32, 3, F32),
    (ALG_ADEF2, F64, F64, 2, F64),
])
def test_batched_solve(small, alg, outer, sloppy, nrhs, coarse):
    """Lockstep solve of several right-hand sides with uneven convergence: each
    solution meets its true residual (oracle) and agrees with the oracle's CG.
    An FP16 little Dirac operator runs the coarse CG on the tensor cores."""
    torch, d, bl, phi, b0, xs0 = small
    h = _handle(d, torch)
    if alg == ALG_ADEF2:
        h.set_subspace((4, 4, 4, 4), torch.from_numpy(phi).cuda(), prec=F64 if outer == F64 else F32,
                       already_orthonormal=True)
        h.build_coarse(coarse)
    tol = _tol(small, outer)
    B = _sources(d, nrhs, 820)
    bt = torch.from_numpy(B).cuda()
    x = torch.zeros_like(bt)
    st = h.solve(bt, x, tol, Hdcg.default_params(algorithm=alg, outer_prec=outer, sloppy_prec=sloppy,
                                                  maxiter=20000), nrhs=nrhs)
    assert st.status == 0
    X = x.cpu().numpy()
    for k in range(nrhs):
        assert _true_res(d, B[k], X[k]) <= 1.05 * tol, f"rhs {k}"
        xk, _ = cg(d.mdagm, B[k], 1e-13)
        assert rel(X[k], xk) < 1e-6, f"rhs {k}"


def test_batched_equals_sequential_and_chunks(small):
    """batch=1 and batch=0 reach the same solutions; 17 right-hand sides run as
    a batch of 16 plus one."""
    torch, d, bl, phi, b0, xs0 = small
    h = _handle(d, torch)
    h.set_subspace((4, 4, 4, 4), torch.from_numpy(phi).cuda(), prec=F32, already_orthonormal=True)
    h.build_coarse(F32)
    B = _sources(d, 17, 840)
    bt = torch.from_numpy(B).cuda()
    xb, xq = torch.zeros_like(bt), torch.zeros_like(bt)
    tol = _tol(small, F32)
    sb = h.solve(bt, xb, tol, Hdcg.default_params(batch=1), nrhs=17)
    sq = h.solve(bt, xq, tol, Hdcg.default_params(batch=0), nrhs=17)
    assert sb.status == 0 and sq.status == 0
    Xb, Xq = xb.cpu().numpy(), xq.cpu().numpy()
    for k in range(17):
        assert _true_res(d, B[k], Xb[k]) <= 1.05 * tol
        assert rel(Xb[k], Xq[k]) < 1e-6
