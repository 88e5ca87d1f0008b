"""Pins of subspace reuse (Sec. 6.4, Table twist): twisted boundary conditions
as link phases, and an HDCG solve with the subspace of another twist or mass.
No GPU.

What fixes them, independently of the oracle's own code:
* the free-field symbol: with links e^{i theta_mu}, a plane wave of momentum
  p sees the closed-form Mpc(p + theta) (the test_oracle_dwf symbol);
* reuse: the subspace built for theta = 0 and m = 0.05 (the shared
  two-level problem of conftest), with the coarse
  operator recomputed for the new operator, gives A-DEF2 solves that reach
  CG's solution in fewer iterations than CG, as Table twist reports.
"""
import numpy as np
import pytest

import synthetic as sy
from oracle.coarse import Blocking, coarse_dense_bruteforce, dense_to_stencil
from oracle.dwf import DWF, norm2, twisted_gauge
from oracle.solvers import DeflationSpace, adef2, cg
from tests.test_oracle_dwf import _free_mpc_p


def test_twisted_free_field_symbol():
    dims, Ls = (4, 6, 4, 8), 4
    theta = np.array([np.pi * 0.5 / 4, np.pi * 0.2 / 6, 0.0, 0.1])
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.02, twisted_gauge(sy.unit_gauge(dims), theta))
    x = d.lat.coords[d.lat.sites[1]].astype(float)
    rng = np.random.default_rng(1)
    for n in [(0, 0, 0, 0), (1, 2, 3, 4), (3, 5, 1, 7)]:
        p = 2 * np.pi * np.array(n) / np.array(dims)
        e = rng.standard_normal((Ls, 4)) + 1j * rng.standard_normal((Ls, 4))
        psi = np.zeros(d.field_shape, dtype=np.complex128)
        phase = np.exp(1j * x @ p)
        psi[:, :, :, 2] = phase[:, None, None] * e[None]
        Mp = _free_mpc_p(p + theta, d.S)
        want = (Mp.conj().T @ Mp @ e.ravel()).reshape(Ls, 4)
        got = d.mdagm(psi)
        assert np.abs(got[:, :, :, 2] - phase[:, None, None] * want[None]).max() < 1e-12 * np.abs(want).max()


@pytest.fixture(scope="module")
def base(two_level_8x8x4x4):
    d0, bl, phi, A, b, xs, it8 = two_level_8x8x4x4
    return d0.lat.dims, d0.Ls, d0.U, phi


@pytest.mark.parametrize("theta_units,mass", [((0.5, 0.5, 0.0, 0.0), 0.05), ((0.0, 0.0, 0.0, 0.0), 0.02)])
def test_reused_subspace(base, theta_units, mass):
    dims, Ls, U, phi = base
    theta = np.pi * np.array(theta_units) / np.array(dims)
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, mass, twisted_gauge(U, theta))
    bl = Blocking(d, (4, 4, 4, 4))
    A = dense_to_stencil(coarse_dense_bruteforce(d.mdagm, phi, bl), bl)
    b = sy.gaussian_fermion(dims, Ls, 1902)
    res = adef2(d.mdagm, b, DeflationSpace(phi, bl, A, coarse_tol=0.04), 1e-8)
    hist = []
    xs, _ = cg(d.mdagm, b, 1e-12, history=hist)
    it8 = next(i + 1 for i, h in enumerate(hist) if h <= 1e-8)
    assert res.true_residual < 2e-8
    assert np.sqrt(norm2(res.x - xs) / norm2(xs)) < 1e-5
    assert res.iterations < it8
