"""Subspace reuse (Sec. 6.4, Table twist) through the C ABI: a subspace built
on the GPU for one operator (theta = 0, m = 0.05) is kept while the links are
twisted (hdcg_set_gauge with the oracle's twisted_gauge phases) or the mass is
changed (hdcg_set_dwf), and hdcg_build_coarse recomputes the little Dirac
operator for the new operator.  The A-DEF2 solve with the reused subspace
meets the oracle's CG solution of the new operator (true residual recomputed
by the oracle; kappa ~ 1e2 on this lattice, so a 1e-9 residual bounds the
solution error well below the 1e-6 bar) in fewer iterations than CG."""
import numpy as np
import pytest

import synthetic as sy
from oracle.dwf import DWF, norm2, twisted_gauge
from oracle.solvers import cg
from paper_1402_2585_gb300 import ALG_ADEF2, F32, Hdcg
from tests.gpu_util import rel, torch_or_skip

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("theta_units,mass", [((0.5, 0.5, 0.0, 0.0), 0.05), ((0.0, 0.0, 0.0, 0.0), 0.02),
                                               ((0.5, 0.0, 0.25, 0.0), 0.02)])
def test_reused_subspace_meets_the_oracle(theta_units, mass):
    torch = torch_or_skip()
    dims, Ls = (8, 8, 8, 8), 4
    U = sy.gauge_field(dims, 0.4, 1950)
    h = Hdcg(dims, Ls, stream=torch.cuda.current_stream().cuda_stream)
    h.set_dwf(1.8, 1.5, 0.5, 0.05)
    h.set_gauge(torch.from_numpy(U).cuda())
    h.build_subspace((4, 4, 4, 4), 8, F32, inv_steps=2, inv_tol=1e-3, seed=1951)
    # the new operator: twisted links and/or another mass; the subspace stays
    theta = np.pi * np.array(theta_units) / np.array(dims)
    Ut = twisted_gauge(U, theta)
    h.set_gauge(torch.from_numpy(Ut).cuda())
    h.set_dwf(1.8, 1.5, 0.5, mass)
    h.build_coarse(F32)
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, mass, Ut)
    b = sy.gaussian_fermion(dims, Ls, 1952)
    hist = []
    xs, _ = cg(d.mdagm, b, 1e-12, history=hist)
    it9 = next(i + 1 for i, r in enumerate(hist) if r <= 1e-9)
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    st = h.solve(bt, x, 1e-9, Hdcg.default_params(algorithm=ALG_ADEF2, outer_prec=F32, sloppy_prec=F32))
    assert st.status == 0
    xg = x.cpu().numpy()
    assert np.sqrt(norm2(b - d.mdagm(xg)) / norm2(b)) <= 1.05e-9
    assert rel(xg, xs) < 1e-6
    assert st.iterations < it9
    h.close()
