"""The coarse solvers' CUDA-graph replay.  Graphs are captured only on a
non-default stream (the legacy default stream cannot be captured), so the
same deflated solves run once on the default stream (direct launches) and
once on a user stream (iteration pairs replayed as graphs): the solutions
must agree bit for bit, since the graph replays the same kernels with the
same deterministic reductions."""
import numpy as np
import pytest

import synthetic as sy
from oracle.coarse import Blocking
from oracle.dwf import DWF, norm2
from oracle.solvers import inverse_iteration_subspace
from paper_1402_2585_gb300 import ALG_ADEF2, F16, F32, Hdcg
from tests.gpu_util import torch_or_skip

pytestmark = pytest.mark.gpu


def _solve(torch, d, phi, B, stream, coarse):
    h = Hdcg(d.lat.dims, d.Ls, stream=stream)
    h.set_dwf(d.M5, d.b, d.c, d.mass)
    h.set_gauge(torch.from_numpy(d.U).cuda())
    h.set_subspace((4, 4, 4, 4), torch.from_numpy(phi).cuda(), prec=F32, already_orthonormal=True)
    h.build_coarse(coarse)
    h.build_coarse_deflation(8, inv_steps=3, tol=1e-6, seed=1500)
    out = []
    for nrhs in (1, 3):
        bt = torch.from_numpy(np.ascontiguousarray(B[:nrhs] if nrhs > 1 else B[0])).cuda()
        x = torch.zeros_like(bt)
        st = h.solve(bt, x, 1e-8, Hdcg.default_params(algorithm=ALG_ADEF2), nrhs=nrhs)
        assert st.status == 0
        torch.cuda.synchronize()
        out.append(x.cpu().numpy())
    h.close()
    return out


@pytest.mark.parametrize("coarse", [F16, F32])
def test_graph_replay_matches_direct_launches(coarse):
    torch = torch_or_skip()
    dims, Ls = (8, 8, 4, 4), 4
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.01, sy.gauge_field(dims, 0.4, 800))
    bl = Blocking(d, (4, 4, 4, 4))
    phi = inverse_iteration_subspace(d.mdagm, sy.gaussian_fermions(dims, Ls, 801, 6), bl, steps=2, tol=1e-3)
    B = sy.gaussian_fermions(dims, Ls, 1501, 3)
    direct = _solve(torch, d, phi, B, torch.cuda.current_stream().cuda_stream, coarse)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        graphed = _solve(torch, d, phi, B, s.cuda_stream, coarse)
    for a, g in zip(direct, graphed):
        assert np.array_equal(a, g)
    x1 = graphed[0]
    assert np.sqrt(norm2(B[0] - d.mdagm(x1)) / norm2(B[0])) <= 1.05e-8
