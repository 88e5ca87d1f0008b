"""Per-step error of the 16-bit preconditioner path against the FP64 oracle on
the full 24^3 x 48 x 16 Moebius lattice (m = 0.002, 4^4 blocks, Nvec 32):
the fine operator H in FP16 (and FP32) storage, restriction and prolongation
with an FP16 subspace, and the little Dirac operator apply with an FP16 A
(Sec. 6.5 and Table sloppy: the preconditioner's 16-bit storage).

Every GPU output is compared element by element with the oracle on the host
(relative L2 and the largest element error relative to the largest element),
and the figures of every step are printed as one JSON line (also written to
the file named by HDCG_STEP_REPORT, if set).  The inputs are FP64; the GPU
sees them rounded to its storage precision, so each figure is the whole
error of that step in that storage.  Bars: 16-bit storage with FP32
arithmetic, unit roundoff 2^-11 = 4.9e-4 per stored value: H (about 200
stored operands per output, errors add in quadrature) 3e-3; restriction and
prolongation 2e-3; coarse apply 5e-3; FP32 H 1e-6.

Host memory: the subspace is 32 complex double fields of 1 GB each.
"""
import json
import os

import numpy as np
import pytest

import synthetic as sy
from oracle.coarse import Blocking, coarse_apply, prolong, restrict
from oracle.dwf import DWF
from paper_1402_2585_gb300 import F16, F32, F64, Hdcg
from tests.gpu_util import from_gpu, to_gpu, torch_or_skip

pytestmark = pytest.mark.gpu

W = sy.WORKLOADS["cfg3_24x24x24x48_ls16_mobius"]


def _err(got, want):
    d = (got - want).ravel()
    return {"rel_l2": float(np.linalg.norm(d) / np.linalg.norm(want.ravel())),
            "max_rel": float(np.abs(d).max() / np.abs(want).max())}


def _complex_normal(rng, shape):
    z = rng.standard_normal(tuple(shape) + (2,))
    z *= np.sqrt(0.5)
    return z.view(np.complex128)[..., 0]


def test_fp16_steps_full_size_24x24x24x48_ls16():
    torch = torch_or_skip()
    U = sy.gauge_field(W.dims, W.eps, W.gauge_seed)
    d = DWF(W.dims, W.Ls, W.M5, W.b, W.c, W.mass, U)
    h = Hdcg(W.dims, W.Ls, stream=torch.cuda.current_stream().cuda_stream)
    h.set_dwf(W.M5, W.b, W.c, W.mass)
    h.set_gauge(torch.from_numpy(U).cuda())
    report = {"workload": W.name, "nvec": W.nvec}

    # fine operator
    psi = sy.gaussian_fermion(W.dims, W.Ls, W.source_seed)
    Hpsi = d.mdagm(psi)
    for prec, name in [(F16, "H_f16"), (F32, "H_f32")]:
        x = to_gpu(psi, prec)
        y = torch.empty_like(x)
        h.apply_mdagm(x, y, prec=prec)
        report[name] = _err(from_gpu(y), Hpsi)
        del x, y
    del Hpsi

    # restriction and prolongation with a 16-bit subspace (Gaussian vectors:
    # both maps are linear in each subspace vector, orthonormality plays no part)
    bl = Blocking(d, W.block)
    rng = np.random.default_rng(3301)
    phi = _complex_normal(rng, (W.nvec,) + d.field_shape)
    h.set_subspace(W.block, phi, prec=F16, already_orthonormal=True)
    c = torch.zeros((bl.Vc, W.nvec, 2), dtype=torch.float64, device="cuda")
    h.restrict(to_gpu(psi, F16), F16, c)
    report["restrict_f16"] = _err(from_gpu(c), restrict(phi, psi, bl))
    cv = _complex_normal(rng, (bl.Vc, W.nvec))
    out = torch.empty(tuple(d.field_shape) + (2,), dtype=torch.float16, device="cuda")
    h.prolong(to_gpu(cv, F64), out, F16)
    report["prolong_f16"] = _err(from_gpu(out), prolong(phi, cv, bl))
    del phi, out

    # little Dirac operator with 16-bit storage
    A = _complex_normal(rng, (bl.Vc, 81, W.nvec, W.nvec))
    h.set_coarse(A, prec=F16)
    y = torch.zeros_like(c)
    h.coarse_apply(to_gpu(cv, F64), y)
    report["coarse_apply_f16"] = _err(from_gpu(y), coarse_apply(A, cv, bl))

    line = json.dumps(report)
    print(line)
    path = os.environ.get("HDCG_STEP_REPORT")
    if path:
        with open(path, "w") as f:
            f.write(line + "\n")
    assert report["H_f16"]["rel_l2"] < 3e-3
    assert report["H_f32"]["rel_l2"] < 1e-6
    assert report["restrict_f16"]["rel_l2"] < 2e-3
    assert report["prolong_f16"]["rel_l2"] < 2e-3
    assert report["coarse_apply_f16"]["rel_l2"] < 5e-3
