"""The reduced-precision codecs of Sec. 6.5 (Table sloppy) through the C ABI.

* hdcg_encode_i8 / hdcg_decode_i8 against the oracle's encode_i8 / decode_i8,
  bit for bit (both FP64): prefactors, bytes and decoded values, on fields
  spanning six orders of magnitude between sites, exact zeros and the
  prefactor's rounding edges (a value just above an FP16 midpoint, subnormal
  halves, the largest value that still rounds to a finite prefactor).
* sloppy_codec in hdcg_solve: the preconditioner's unit-RMS input through
  either codec; the A-DEF2 solve still meets the oracle's solution (true
  residual recomputed by the oracle) within three outer iterations of the
  solve without it (Table sloppy: no change in the iteration count)."""
import numpy as np
import pytest

import synthetic as sy
from oracle.codec import decode_i8, encode_i8
from oracle.dwf import DWF, norm2
from oracle.solvers import cg
from paper_1402_2585_gb300 import ALG_ADEF2, F16, F32, Hdcg
from tests.gpu_util import rel, torch_or_skip

pytestmark = pytest.mark.gpu


def test_i8_codec_bit_exact():
    torch = torch_or_skip()
    dims, Ls = (4, 4, 4, 4), 4
    h = Hdcg(dims, Ls, stream=torch.cuda.current_stream().cuda_stream)
    n4 = 128
    psi = sy.gaussian_fermion(dims, Ls, 1970) * np.geomspace(1e-3, 1e3, n4)[:, None, None, None]
    psi[3] = 0.0
    psi[4, :, :, :] = 0.0
    psi[4, 0, 0, 0] = 1 + 2.0 ** -11 + 2.0 ** -40     # just above an FP16 midpoint
    psi[5, 1, 2, 1] = 3 * 2.0 ** -25                    # subnormal tie
    psi[6, 2, 1, 2] = 65519.0                           # largest value that rounds to 65504
    psi[7, 3, 3, 0] = -0.3
    for nf in (1, 2):
        x = np.stack([psi, 0.5 * psi])[:nf]
        xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        scale = torch.zeros((nf, n4, Ls), dtype=torch.float16, device="cuda")
        q = torch.zeros((nf, n4, Ls, 24), dtype=torch.int8, device="cuda")
        h.encode_i8(xt, scale, q, nf)
        ws, wq = encode_i8(x)
        assert np.array_equal(scale.cpu().numpy().view(np.uint16), ws.view(np.uint16))
        assert np.array_equal(q.cpu().numpy(), wq)
        out = torch.zeros_like(xt)
        h.decode_i8(scale, q, out, nf)
        assert np.array_equal(out.cpu().numpy(), decode_i8(ws, wq))
    h.close()


@pytest.mark.parametrize("codec", [1, 2])
def test_hdcg_with_compressed_preconditioner_input(codec):
    torch = torch_or_skip()
    dims, Ls = (8, 8, 8, 8), 4
    U = sy.gauge_field(dims, 0.4, 1971)
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.02, U)
    h = Hdcg(dims, Ls, stream=torch.cuda.current_stream().cuda_stream)
    h.set_dwf(1.8, 1.5, 0.5, 0.02)
    h.set_gauge(torch.from_numpy(U).cuda())
    h.build_subspace((4, 4, 4, 4), 8, F16, inv_steps=2, inv_tol=1e-3, seed=1972)
    h.build_coarse(F32)
    b = sy.gaussian_fermion(dims, Ls, 1973)
    xs, _ = cg(d.mdagm, b, 1e-12)
    bt = torch.from_numpy(b).cuda()
    its = {}
    for cd in (0, codec):
        x = torch.zeros_like(bt)
        st = h.solve(bt, x, 1e-9, Hdcg.default_params(algorithm=ALG_ADEF2, outer_prec=F32, sloppy_prec=F16,
                                                      sloppy_codec=cd))
        assert st.status == 0
        xg = x.cpu().numpy()
        assert np.sqrt(norm2(b - d.mdagm(xg)) / norm2(b)) <= 1.05e-9
        assert rel(xg, xs) < 1e-6
        its[cd] = st.iterations
    assert its[codec] <= its[0] + 3
    h.close()
