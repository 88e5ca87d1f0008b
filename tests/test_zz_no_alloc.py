"""hdcg_coarse_apply_noalloc: the coarse stencil apply for callers that cannot
allocate device memory on this path (a host code whose device memory all
belongs to its own pool allocator, or one that must not grow its footprint
while other work is resident).  It must return what hdcg_coarse_apply
returns, on consecutive calls that share its fixed scratch array, and what
the FP64 oracle's stencil apply gives for the same stored operator.

The operator stored in FP64, FP32 and FP16 takes every branch of the entry
point: FP64 vectors used in place, FP32 vectors converted into the scratch
array, and the FP16 operator read with 4-wide (Nvec a multiple of 4) and
scalar (Nvec not a multiple of 4) loads.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

import synthetic as sy
from oracle.coarse import Blocking, coarse_apply
from oracle.dwf import DWF
from paper_1402_2585_gb300 import F16, F32, F64, Hdcg
from tests.gpu_util import from_gpu, rel, to_gpu, torch_or_skip

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,nvec,tol", [(F32, 5, 1e-6), (F64, 5, 1e-12), (F16, 8, 1e-6), (F16, 6, 1e-6)])
def test_noalloc_coarse_apply_matches_allocating_entry_point(prec, nvec, tol):
    torch = torch_or_skip()
    dims, Ls = (8, 8, 4, 4), 4
    U = sy.gauge_field(dims, 0.4, 901)
    h = Hdcg(dims, Ls, stream=torch.cuda.current_stream().cuda_stream)
    h.set_dwf(1.8, 1.5, 0.5, 0.02)
    h.set_gauge(torch.from_numpy(U).cuda())
    h.build_subspace((4, 4, 4, 4), nvec, prec, inv_steps=0, seed=902)
    h.build_coarse(prec)
    bl = Blocking(DWF(dims, Ls, 1.8, 1.5, 0.5, 0.02, U), (4, 4, 4, 4))
    A = np.zeros((bl.Vc, 81, nvec, nvec), dtype=np.complex128)
    h.get_coarse(A)   # the operator as stored (FP16/FP32 values widened exactly)
    for call, seed in enumerate((903, 904)):
        xc = sy.coarse_gaussian(bl.Vc, nvec, seed)
        x = to_gpu(xc, F64)
        want = torch.zeros_like(x)
        got = torch.full_like(x, float("nan"))
        h.coarse_apply(x, want)
        h.coarse_apply_noalloc(x, got)
        g = from_gpu(got)
        assert rel(g, from_gpu(want)) < tol, f"call {call}: against hdcg_coarse_apply"
        assert rel(g, coarse_apply(A, xc, bl)) < tol, f"call {call}: against the oracle"
    h.close()
