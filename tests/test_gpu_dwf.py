"""Parity of the CUDA fine operator (through the C ABI) with the FP64 oracle.

Tolerances (relative L2 over the whole output): FP64 1e-12, and 1e-12 too for
the double-float operator (about 48 significant bits, 2^-48 ~ 3.6e-15 per
rounding); FP32 1e-6 and
FP16 storage 3e-3 (the operator-apply bars of the specification); BF16 with
round-to-nearest 2e-2 and with truncation 4e-2 (8-bit mantissa: ~4e-3 per
rounding, about eight roundings of input, links and intermediates).
"""
import numpy as np
import pytest

import synthetic as sy
from oracle.dwf import DWF, norm2
from paper_1402_2585_gb300 import BF16, BF16T, DF64, F16, F32, F64, Hdcg, HdcgError
from tests.gpu_util import from_gpu, rel, to_gpu, torch_or_skip

pytestmark = pytest.mark.gpu

TOL = {F64: 1e-12, DF64: 1e-12, F32: 1e-6, F16: 3e-3, BF16: 2e-2, BF16T: 4e-2}

CASES = {
    "shamir_4x4x4x4_ls4": dict(dims=(4, 4, 4, 4), Ls=4, b=1.0, c=0.0, m=0.01, eps=0.3, apbc=False),
    "mobius_8x4x4x6_ls8_apbc": dict(dims=(8, 4, 4, 6), Ls=8, b=1.5, c=0.5, m=0.002, eps=0.4, apbc=True),
    "mobius_4x6x4x4_ls16": dict(dims=(4, 6, 4, 4), Ls=16, b=1.5, c=0.5, m=0.02, eps=0.45, apbc=False),
    "shamir_2x2x2x2_ls2": dict(dims=(2, 2, 2, 2), Ls=2, b=1.0, c=0.0, m=0.1, eps=0.5, apbc=False),
    "mobius_2x2x4x2_ls32": dict(dims=(2, 2, 4, 2), Ls=32, b=2.0, c=1.0, m=0.05, eps=0.5, apbc=True),
}


def _setup(case, seed=0):
    torch = torch_or_skip()
    p = CASES[case]
    U = sy.gauge_field(p["dims"], p["eps"], 500 + seed)
    d = DWF(p["dims"], p["Ls"], 1.8, p["b"], p["c"], p["m"], U, antiperiodic_t=p["apbc"])
    h = Hdcg(p["dims"], p["Ls"], antiperiodic_t=p["apbc"], stream=torch.cuda.current_stream().cuda_stream)
    h.set_dwf(1.8, p["b"], p["c"], p["m"])
    h.set_gauge(torch.from_numpy(U).cuda())
    return torch, d, h


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [F64, DF64, F32, F16, BF16, BF16T])
def test_mpc_and_mdagm_parity(case, prec):
    torch, d, h = _setup(case)
    psi = sy.gaussian_fermion(d.lat.dims, d.Ls, 600)
    x = to_gpu(psi, prec)
    y = torch.empty_like(x)
    for dagger, ref in ((False, d.mpc), (True, d.mpc_dag)):
        h.apply_mpc(x, y, dagger=dagger, prec=prec)
        err = rel(from_gpu(y), ref(psi))
        assert err < TOL[prec], f"Mpc{'^dag' if dagger else ''} {case} prec {prec}: {err:.3e}"
    pHp = h.apply_mdagm(x, y, prec=prec, want_pHp=True)
    want = d.mdagm(psi)
    err = rel(from_gpu(y), want)
    assert err < TOL[prec], f"H {case} prec {prec}: {err:.3e}"
    assert pHp == pytest.approx(norm2(d.mpc(psi)), rel=max(TOL[prec], 1e-12))


@pytest.mark.parametrize("prec", [F32, DF64])
def test_mdagm_full_size_16x16x16x16_ls16(prec):
    """The two-level workload's lattice (16^4 x 16, Shamir, m = 0.005) in FP32
    (the outer operator) and double-float (the true-residual operator)."""
    w = sy.WORKLOADS["cfg2_16x16x16x16_ls16_shamir"]
    torch = torch_or_skip()
    U = sy.gauge_field(w.dims, w.eps, w.gauge_seed)
    d = DWF(w.dims, w.Ls, w.M5, w.b, w.c, w.mass, U)
    h = Hdcg(w.dims, w.Ls, stream=torch.cuda.current_stream().cuda_stream)
    h.set_dwf(w.M5, w.b, w.c, w.mass)
    h.set_gauge(torch.from_numpy(U).cuda())
    psi = sy.gaussian_fermion(w.dims, w.Ls, w.source_seed)
    x = to_gpu(psi, prec)
    y = torch.empty_like(x)
    h.apply_mdagm(x, y, prec=prec)
    assert rel(from_gpu(y), d.mdagm(psi)) < TOL[prec]


def test_deterministic_and_hermitian():
    torch, d, h = _setup("mobius_8x4x4x6_ls8_apbc")
    u = to_gpu(sy.gaussian_fermion(d.lat.dims, d.Ls, 601), F64)
    v = to_gpu(sy.gaussian_fermion(d.lat.dims, d.Ls, 602), F64)
    hu, hv, hv2 = torch.empty_like(u), torch.empty_like(v), torch.empty_like(v)
    p1 = h.apply_mdagm(v, hv, prec=F64, want_pHp=True)
    p2 = h.apply_mdagm(v, hv2, prec=F64, want_pHp=True)
    assert torch.equal(hv, hv2) and p1 == p2
    h.apply_mdagm(u, hu, prec=F64)
    a = np.vdot(from_gpu(u), from_gpu(hv))
    b = np.conj(np.vdot(from_gpu(v), from_gpu(hu)))
    assert abs(a - b) < 1e-12 * abs(a)


def test_argument_errors():
    torch, d, h = _setup("shamir_4x4x4x4_ls4")
    x = to_gpu(sy.gaussian_fermion(d.lat.dims, d.Ls, 603), F32)
    with pytest.raises(HdcgError):
        h.apply_mpc(x, x, prec=F32)          # aliasing in/out
    with pytest.raises(HdcgError):
        h.apply_mpc(x, torch.empty_like(x), prec=9)
    with pytest.raises(HdcgError):
        Hdcg((4, 4, 4, 3), 4)                 # odd extent
    with pytest.raises(HdcgError):
        Hdcg((4, 4, 4, 4), 12)                # Ls not a power of two
    h2 = Hdcg((4, 4, 4, 4), 4)
    with pytest.raises(HdcgError):
        h2.apply_mpc(x, torch.empty_like(x), prec=F32)   # no gauge field yet


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("prec", [F32, F16, BF16T])
def test_every_hop_variant(case, variant, prec):
    """Each kernel variant the hop autotuner can choose (forced with
    hdcg_set_hop_variant): the scalar register-budget variants, the prefetching
    one, and the packed-FP32 ones with links staged in shared memory (Ls >= 8)
    or expanded per thread (Ls < 8); same bars as above."""
    torch, d, h = _setup(case, seed=1)
    h.set_hop_variant(variant)
    psi = sy.gaussian_fermion(d.lat.dims, d.Ls, 610)
    x = to_gpu(psi, prec)
    y = torch.empty_like(x)
    for dagger, ref in ((False, d.mpc), (True, d.mpc_dag)):
        h.apply_mpc(x, y, dagger=dagger, prec=prec)
        assert rel(from_gpu(y), ref(psi)) < TOL[prec]
    pHp = h.apply_mdagm(x, y, prec=prec, want_pHp=True)
    assert rel(from_gpu(y), d.mdagm(psi)) < TOL[prec]
    assert pHp == pytest.approx(norm2(d.mpc(psi)), rel=TOL[prec])


@pytest.mark.parametrize("variant", [0, 4, 5])
def test_fused_cg_step_every_variant(variant):
    """The CG step fused into the last hop pass (x += alpha p, r -= alpha H p,
    |r|^2) in each variant: a plain FP32 CG solve reaches the oracle's true
    residual and solution (kappa ~ 1e2 on this lattice)."""
    from oracle.solvers import cg
    from paper_1402_2585_gb300 import ALG_CG
    torch, d, h = _setup("mobius_8x4x4x6_ls8_apbc", seed=2)
    h.set_hop_variant(variant)
    b = sy.gaussian_fermion(d.lat.dims, d.Ls, 611)
    xs, _ = cg(d.mdagm, b, 1e-12)
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    st = h.solve(bt, x, 1e-9, Hdcg.default_params(algorithm=ALG_CG, outer_prec=F32, maxiter=20000))
    assert st.status == 0
    xg = x.cpu().numpy()
    assert np.sqrt(norm2(b - d.mdagm(xg)) / norm2(b)) <= 1.05e-9
    assert rel(xg, xs) < 1e-6
