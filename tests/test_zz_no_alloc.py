"""hdcg_coarse_apply_noalloc: the coarse stencil apply for callers that cannot
allocate device memory on this path.  It must return what hdcg_coarse_apply
returns, on consecutive calls that share its fixed scratch array.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test."""
import pytest

import synthetic as sy
from paper_1402_2585_gb300 import F32, F64, Hdcg
from tests.gpu_util import from_gpu, rel, to_gpu, torch_or_skip

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [(F32, 1e-6), (F64, 1e-12)])
def test_noalloc_coarse_apply_matches_allocating_entry_point(prec, tol):
    torch = torch_or_skip()
    dims, Ls, nvec = (8, 8, 4, 4), 4, 5
    h = Hdcg(dims, Ls, stream=torch.cuda.current_stream().cuda_stream)
    h.set_dwf(1.8, 1.5, 0.5, 0.02)
    h.set_gauge(torch.from_numpy(sy.gauge_field(dims, 0.4, 901)).cuda())
    h.build_subspace((4, 4, 4, 4), nvec, prec, inv_steps=0, seed=902)
    h.build_coarse(prec)
    vc = (dims[0] // 4) * (dims[1] // 4) * (dims[2] // 4) * (dims[3] // 4)
    for call, seed in enumerate((903, 904)):
        x = to_gpu(sy.coarse_gaussian(vc, nvec, seed), F64)
        want = torch.zeros_like(x)
        got = torch.full_like(x, float("nan"))
        h.coarse_apply(x, want)
        h.coarse_apply_noalloc(x, got)
        assert rel(from_gpu(got), from_gpu(want)) < tol, f"call {call}"
    h.close()
