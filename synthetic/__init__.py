"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module draws random numbers and builds input arrays (gauge links,
Gaussian fermion fields, point sources, random gauge transforms).  It holds
none of the solver's arithmetic: no Dirac operator, no projector, no Krylov
step.  Both the FP64 oracle and the CUDA library receive the arrays made here,
so the two sides see bit-identical inputs.

Random numbers come from splitmix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: output i of stream ``seed`` is ``mix(seed + (i + 1) * GAMMA)``.
Gaussians use the Box-Muller transform on consecutive pairs of uniforms.

Canonical layouts (the library's ABI layouts):

* lattice site ``lex = x + Lx*(y + Ly*(z + Lz*t))``; parity ``(x+y+z+t) % 2``;
  checkerboard index ``cb = lex >> 1`` (all extents even);
* fermion field on the odd checkerboard: ``[cb][s][spin 4][colour 3]`` complex;
* gauge field: ``[lex][mu = x,y,z,t][row][col]`` complex, ``U_mu(x)`` links
  ``x`` to ``x + mu``.
"""
from __future__ import annotations

import numpy as np

from .configs import WORKLOADS, Workload  # noqa: F401

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+n-1`` of the splitmix64 stream ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed % (1 << 64)) + ctr * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in the open interval (0, 1) from the top 53 bits."""
    z = splitmix64(seed, n, offset)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int) -> np.ndarray:
    """n standard normal doubles; pair i uses uniforms 2i, 2i+1 (Box-Muller)."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m)
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    th = 2.0 * np.pi * u[1::2]
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(th)
    z[1::2] = r * np.sin(th)
    return z[:n]


def complex_normal(seed: int, shape) -> np.ndarray:
    """Complex Gaussian with E|z|^2 = 1, filled in C order of ``shape``."""
    n = int(np.prod(shape))
    z = normal(seed, 2 * n) / np.sqrt(2.0)
    return (z[0::2] + 1j * z[1::2]).reshape(shape)


# ----------------------------------------------------------------------------
# lattice bookkeeping (pure indexing, shared by every consumer of the layouts)
# ----------------------------------------------------------------------------

def volume(dims) -> int:
    return int(np.prod(dims))


def check_dims(dims) -> None:
    if len(dims) != 4 or any(int(d) < 2 or int(d) % 2 for d in dims):
        raise ValueError(f"lattice extents must be four even numbers >= 2, got {dims}")


_GELL_MANN = np.zeros((8, 3, 3), dtype=np.complex128)
_GELL_MANN[0][0, 1] = _GELL_MANN[0][1, 0] = 1
_GELL_MANN[1][0, 1] = -1j
_GELL_MANN[1][1, 0] = 1j
_GELL_MANN[2][0, 0] = 1
_GELL_MANN[2][1, 1] = -1
_GELL_MANN[3][0, 2] = _GELL_MANN[3][2, 0] = 1
_GELL_MANN[4][0, 2] = -1j
_GELL_MANN[4][2, 0] = 1j
_GELL_MANN[5][1, 2] = _GELL_MANN[5][2, 1] = 1
_GELL_MANN[6][1, 2] = -1j
_GELL_MANN[6][2, 1] = 1j
_GELL_MANN[7][0, 0] = _GELL_MANN[7][1, 1] = 1 / np.sqrt(3)
_GELL_MANN[7][2, 2] = -2 / np.sqrt(3)


def _reunitarise(u: np.ndarray) -> np.ndarray:
    """Project (..., 3, 3) onto SU(3): normalise row 0, orthogonalise row 1,
    row 2 = conj(row0 x row1)."""
    r0 = u[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def random_su3(seed: int, count: int, eps: float) -> np.ndarray:
    """``count`` matrices exp(i eps H), H = sum_a w_a lambda_a / 2 with
    w_a ~ N(0,1) (traceless Hermitian), reunitarised.  Shape (count, 3, 3)."""
    w = normal(seed, 8 * count).reshape(count, 8)
    h = np.einsum("na,aij->nij", w, _GELL_MANN) * 0.5
    evals, evecs = np.linalg.eigh(h)
    phase = np.exp(1j * eps * evals)
    u = np.einsum("nij,nj,nkj->nik", evecs, phase, np.conj(evecs))
    return _reunitarise(u)


def gauge_field(dims, eps: float, seed: int) -> np.ndarray:
    """Random SU(3) gauge field, canonical layout (V, 4, 3, 3) complex128."""
    check_dims(dims)
    v = volume(dims)
    return random_su3(seed, 4 * v, eps).reshape(v, 4, 3, 3)


def unit_gauge(dims) -> np.ndarray:
    v = volume(dims)
    u = np.zeros((v, 4, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def gaussian_fermion(dims, Ls: int, seed: int) -> np.ndarray:
    """Gaussian odd-checkerboard 5D field, canonical (V/2, Ls, 4, 3) complex128."""
    check_dims(dims)
    return complex_normal(seed, (volume(dims) // 2, Ls, 4, 3))


def gaussian_fermions(dims, Ls: int, seed: int, count: int) -> np.ndarray:
    """``count`` independent Gaussian odd-checkerboard fields, stream ``seed``."""
    check_dims(dims)
    return complex_normal(seed, (count, volume(dims) // 2, Ls, 4, 3))


def coarse_gaussian(n_sites: int, nvec: int, seed: int) -> np.ndarray:
    """Gaussian coarse vector, canonical (n_sites, nvec) complex128."""
    return complex_normal(seed, (n_sites, nvec))


def point_sources(dims, Ls, count: int = 12) -> np.ndarray:
    """Spin-colour point sources on the odd-checkerboard system, one per
    (spin, colour) pair, at the odd site x = (1, 0, 0, 0): chirality-plus spins
    (0, 1) on the wall s = 0, chirality-minus spins (2, 3) on the wall s = Ls - 1.
    Shape (count, V/2, Ls, 4, 3); count <= 12 takes the first pairs."""
    check_dims(dims)
    v2 = volume(dims) // 2
    out = np.zeros((count, v2, Ls, 4, 3), dtype=np.complex128)
    cb = 1 >> 1                      # lex index 1 (x = 1) is odd; cb = lex >> 1
    for k in range(count):
        spin, colour = (k // 3) % 4, k % 3
        s = 0 if spin < 2 else Ls - 1
        out[k, cb, s, spin, colour] = 1.0
    return out
