"""Helpers for the GPU tests: canonical fields <-> torch buffers of each ABI precision."""
import numpy as np
import pytest

TORCH_DTYPE = {}


def torch_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def to_gpu(x, prec):
    """complex128 numpy array -> contiguous CUDA tensor of interleaved reals in the ABI precision."""
    import torch
    dt = {0: torch.float64, 1: torch.float32, 2: torch.float16, 3: torch.bfloat16, 4: torch.bfloat16,
          5: torch.float64}[prec]
    r = torch.view_as_real(torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)))
    if prec == 4:
        # truncation of the float32 word: keep its top 16 bits
        f = r.to(torch.float32).contiguous()
        r = (f.view(torch.int32) >> 16).to(torch.int16).view(torch.bfloat16)
    else:
        r = r.to(dt)
    return r.cuda().contiguous()


def from_gpu(t):
    import torch
    return torch.view_as_complex(t.detach().cpu().to(torch.float64).contiguous()).numpy()


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _n2(v):
    return float(np.vdot(v, v).real)


def cg_kappa(apply_H, b, tol):
    """CG on H from zero with the Lanczos tridiagonal of its coefficients
    (diagonal 1/alpha_k + beta_{k-1}/alpha_{k-1}, off-diagonal sqrt(beta_k)/alpha_k):
    returns (x, kappa) with kappa the ratio of the extreme Ritz values, which
    have converged to H's extreme eigenvalues once CG reaches tol ~ 1e-13."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = _n2(r)
    bb = rr
    al, be = [], []
    while np.sqrt(rr / bb) > tol and len(al) < 20000:
        w = apply_H(p)
        a = rr / np.vdot(p, w).real
        x += a * p
        r -= a * w
        rn = _n2(r)
        al.append(a)
        be.append(rn / rr)
        p = r + (rn / rr) * p
        rr = rn
    k = len(al)
    T = np.zeros((k, k))
    for i in range(k):
        T[i, i] = 1.0 / al[i] + (be[i - 1] / al[i - 1] if i else 0.0)
        if i + 1 < k:
            T[i, i + 1] = T[i + 1, i] = np.sqrt(be[i]) / al[i]
    ev = np.linalg.eigvalsh(T)
    return x, ev[-1] / ev[0]


def kappa_tol(kappa, bar=1e-6, cap=1e-8):
    """Relative residual that bounds the solution error by bar / 2:
    |x - x*| / |x*| <= kappa |r| / |b|."""
    return min(cap, 0.5 * bar / kappa)
