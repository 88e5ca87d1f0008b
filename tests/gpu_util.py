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
