"""Source preparation and reconstruction of the Schur form (Sec. 4) through the
C ABI, against the FP64 oracle: b = Mpc^dag (eta_o - M_oe M_ee^-1 eta_e) and
psi_e = M_ee^-1 (eta_e - M_eo psi_o) element by element (FP64 on both sides:
1e-12), and the whole chain -- prepare, solve H psi_o = b, reconstruct --
solving the full system D psi = eta (the oracle applies D to the result)."""
import numpy as np
import pytest

import synthetic as sy
from oracle.dwf import DWF, norm2
from paper_1402_2585_gb300 import ALG_CG, F64, Hdcg
from tests.gpu_util import rel, torch_or_skip

pytestmark = pytest.mark.gpu

CASES = {
    "shamir_4x4x4x4_ls4": dict(dims=(4, 4, 4, 4), Ls=4, b=1.0, c=0.0, m=0.05, apbc=False),
    "mobius_8x4x4x6_ls8_apbc": dict(dims=(8, 4, 4, 6), Ls=8, b=1.5, c=0.5, m=0.02, apbc=True),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("on_device", [True, False])
def test_prep_solve_reconstruct(case, on_device):
    torch = torch_or_skip()
    p = CASES[case]
    U = sy.gauge_field(p["dims"], 0.4, 700)
    d = DWF(p["dims"], p["Ls"], 1.8, p["b"], p["c"], p["m"], U, antiperiodic_t=p["apbc"])
    h = Hdcg(p["dims"], p["Ls"], antiperiodic_t=p["apbc"], stream=torch.cuda.current_stream().cuda_stream)
    h.set_dwf(1.8, p["b"], p["c"], p["m"])
    h.set_gauge(torch.from_numpy(U).cuda())
    eta_e = sy.gaussian_fermion(p["dims"], p["Ls"], 701)
    eta_o = sy.gaussian_fermion(p["dims"], p["Ls"], 702)

    def buf(a):
        t = torch.from_numpy(np.ascontiguousarray(a))
        return t.cuda() if on_device else t.numpy()

    def host(t):
        return t.cpu().numpy() if hasattr(t, "cpu") else t

    b = buf(np.zeros_like(eta_o))
    h.prep_source(buf(eta_e), buf(eta_o), b)
    assert rel(host(b), d.prep_source(eta_e, eta_o)) < 1e-12
    psi_o = torch.zeros(d.field_shape, dtype=torch.complex128, device="cuda")
    st = h.solve(torch.from_numpy(host(b)).cuda(), psi_o, 1e-11,
                 Hdcg.default_params(algorithm=ALG_CG, outer_prec=F64, maxiter=20000))
    assert st.status == 0
    po = psi_o.cpu().numpy()
    pe = buf(np.zeros_like(eta_e))
    h.reconstruct(buf(eta_e), buf(po), pe)
    assert rel(host(pe), d.reconstruct(eta_e, po)) < 1e-12
    re, ro = d.apply_full(host(pe), po)
    res = np.sqrt((norm2(re - eta_e) + norm2(ro - eta_o)) / (norm2(eta_e) + norm2(eta_o)))
    assert res < 1e-8
    h.close()
