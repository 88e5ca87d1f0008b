"""Host logic without a GPU: the dense third level's Hermitian eigensolver
(hdcg_dense_heev, the prediagonalisation of the global deflation level,
Sec. 5.2) against numpy's eigh, on seeded matrices with clustered and exactly
degenerate spectra."""
import numpy as np
import pytest

import synthetic as sy


def _lib():
    import __graft_entry__ as g
    g.build()
    from paper_1402_2585_gb300 import dense_heev
    return dense_heev


def _hermitian(n, seed, spectrum=None):
    X = sy.complex_normal(seed, (n, n))
    Q, _ = np.linalg.qr(X)
    w = spectrum if spectrum is not None else np.linspace(1e-6, 50.0, n)
    return (Q * w) @ Q.conj().T, np.sort(w)


@pytest.mark.parametrize("n", [1, 2, 7, 64])
def test_eigenpairs_match_numpy(n):
    heev = _lib()
    H, w0 = _hermitian(n, 1400 + n)
    w, V = heev(H)
    scale = np.abs(w0).max()
    assert np.abs(w - np.linalg.eigvalsh(H)).max() < 1e-12 * scale
    assert np.abs(V.conj().T @ V - np.eye(n)).max() < 1e-12
    assert np.abs(V.conj().T @ H @ V - np.diag(w)).max() < 1e-12 * scale
    assert np.all(np.diff(w) >= 0)


def test_degenerate_and_clustered_spectrum():
    """Light-mass-like spectrum: a cluster near 1e-6, an exact triple, a gap."""
    heev = _lib()
    spec = np.concatenate([[1e-6, 1.1e-6, 1.2e-6], [0.5, 0.5, 0.5], np.linspace(2.0, 60.0, 26)])
    H, w0 = _hermitian(32, 1450, spec)
    w, V = heev(H)
    assert np.abs(w - w0).max() < 1e-12 * 60
    assert np.abs(V.conj().T @ H @ V - np.diag(w)).max() < 1e-12 * 60


def test_uses_the_hermitian_part_and_rejects_bad_sizes():
    heev = _lib()
    H, _ = _hermitian(8, 1460)
    A = H + 1e-3 * (sy.complex_normal(1461, (8, 8)) - sy.complex_normal(1461, (8, 8)).conj().T)  # anti-Hermitian
    w = heev(A, vectors=False)
    assert np.abs(w - np.linalg.eigvalsh(0.5 * (A + A.conj().T))).max() < 1e-11
    from paper_1402_2585_gb300 import lib
    assert lib().hdcg_dense_heev(0, None, None, None) == -1
