"""FP64 oracle: subspace generation by a rational low-pass filter (Sec. 4.2,
"Subspace generation", Eq. ratfilt, Table FineSubspaceParams).

TEST INFRASTRUCTURE (see ``oracle/__init__``): never imported by the library.

* ``multishift_cg``   the systems (H + sigma_i) x_i = b for several shifts from
               one Krylov space: CG on the smallest shift, and every shifted
               residual collinear with the base one, r_i = zeta_i r with
               zeta_i = 1 / R_k(-delta_i), R_k the base residual polynomial
               and delta_i = sigma_i - sigma_0 (multi-shift CG, as in Frommer
               et al. and Jegerlehner; the recurrences below are derived from
               R_k's three-term recurrence).
* ``rational_filter_shifts``  the shifts lambda + i eps of Eq. ratfilt and
               the partial-fraction weights c_i = prod_{j != i} 1/(sigma_j -
               sigma_i), so that sum_i c_i / (x + sigma_i) = prod_i 1/(x +
               sigma_i).
* ``rational_filter``  phi = prod_i (H + sigma_i)^-1 eta as sum_i c_i x_i from
               one multi-shift solve (Eq. ratfilt; the paper fixes phi only up
               to normalisation, and the block Gram-Schmidt removes it).
* ``wall_noise``  4D Gaussian noise on the physical components of the walls,
               P_- psi(s = 0) and P_+ psi(s = Ls - 1): the components that the
               mass term of P_s couples (our reading of where Sec. 4.2 puts
               the noise).
* ``surface_truncate``  SubspaceSurfaceDepth: the s-slices farther than
               ``depth`` from both walls set to zero.
* ``rational_subspace``  wall noise, the filter, block Gram-Schmidt.
* ``promote``  a field of a reduced fifth dimension Ls1 placed into Ls: the
               half of the s-slices nearer each wall keeps its distance to that
               wall, the bulk between is zero (our reading of the promotion to
               the full system's surfaces in Sec. 4.2).
* ``two_pass_subspace``  the two-stage generation (Sec. 4.2, Table optimised,
               first and second pass controls): the subspace of a reduced-Ls
               operator with its own mass (the filter and block Gram-Schmidt:
               the first pass yields a subspace), promotion (an isometry, so the
               promoted vectors stay block-orthonormal), then one shifted inversion
               (H + lam2)^-1 of every promoted vector on the full system by
               A-DEF2 deflated with the promoted vectors (the solver that the
               first pass provides), to a loose residual, and block Gram-Schmidt.
               Reading: the deflation space of the second pass is the block
               Gram-Schmidt of the promoted vectors, its coarse operator that of
               H + lam2 (A + lam2 on the diagonal blocks, exact for orthonormal
               blocks), the smoother M_IRS as in the solver.

Parity: pinned by tests/test_oracle_subspace.py (the partial fractions
against the product at sample points; multi-shift solutions against numpy's
dense solves and, for one shift, against the textbook CG iterate by iterate;
the filter against the eigendecomposition of a dense Hermitian matrix; the
coarse operator of H + lam2 against its brute-force assembly; the
support and chirality of the wall noise; the truncation; the filtered
subspace of a domain wall operator concentrating on its low modes; the
promotion's placement; the two-pass result solving its shifted systems, equal
to the single pass when Ls1 = Ls without refinement, and concentrating on the
low modes).
"""
from __future__ import annotations

import numpy as np

from .coarse import Blocking, block_gram_schmidt, coarse_dense_bruteforce, dense_to_stencil
from .dwf import DWF, gamma_matrices


def _dot(a, b):
    return np.vdot(a, b)


def _n2(a):
    return float(np.vdot(a, a).real)


def multishift_cg(apply_H, b, shifts, tol: float, maxiter: int = 100000):
    """x_i = (H + shifts[i])^-1 b for every shift, from one Krylov space.

    Base system B = H + sigma_0 with sigma_0 = min(shifts).  CG on B:
      alpha_k = (r_k, r_k) / (p_k, B p_k), x += alpha_k p_k,
      r_{k+1} = r_k - alpha_k B p_k, beta_k = (r_{k+1}, r_{k+1}) / (r_k, r_k),
      p_{k+1} = r_{k+1} + beta_k p_k.
    Its residual polynomial obeys R_{k+1}(t) = (1 - alpha_k t + g_k) R_k(t) -
    g_k R_{k-1}(t), g_k = alpha_k beta_{k-1} / alpha_{k-1} (g_0 = 0).  For the
    shift delta the residual of the shifted CG is r^d_k = zeta_k r_k with
    zeta_k = 1 / R_k(-delta); its coefficients are alpha^d_k = alpha_k
    zeta_{k+1} / zeta_k and beta^d_k = beta_k (zeta_{k+1} / zeta_k)^2, and
    p^d_{k+1} = zeta_{k+1} r_{k+1} + beta^d_k p^d_k (p^d_0 = b).
    Stops when the base residual reaches ``tol`` relative to |b| (the
    shifted residuals are smaller by |zeta| <= 1).  Returns (list of x_i in
    the order of ``shifts``, iterations).
    """
    shifts = [float(s) for s in shifts]
    s0 = min(shifts)
    deltas = [s - s0 for s in shifts]
    ns = len(shifts)
    x = [np.zeros_like(b) for _ in range(ns)]
    p = [np.array(b, copy=True) for _ in range(ns)]
    r = np.array(b, copy=True)
    pb = np.array(b, copy=True)
    rr = _n2(r)
    bb = rr
    if bb == 0.0:
        return x, 0
    R_prev = [1.0] * ns          # R_{k-1}(-delta)
    R_cur = [1.0] * ns           # R_k(-delta)
    alpha_prev, beta_prev = 1.0, 0.0
    it = 0
    while it < maxiter:
        w = apply_H(pb) + s0 * pb
        alpha = rr / _dot(pb, w).real
        g = alpha * beta_prev / alpha_prev
        R_next = [(1.0 + alpha * d + g) * R_cur[i] - g * R_prev[i] for i, d in enumerate(deltas)]
        for i in range(ns):
            ratio = R_cur[i] / R_next[i]                # zeta_{k+1} / zeta_k
            x[i] = x[i] + (alpha * ratio) * p[i]
        r = r - alpha * w
        rr_new = _n2(r)
        beta = rr_new / rr
        it += 1
        for i in range(ns):
            ratio = R_cur[i] / R_next[i]
            p[i] = r / R_next[i] + (beta * ratio * ratio) * p[i]
        pb = r + beta * pb
        R_prev, R_cur = R_cur, R_next
        alpha_prev, beta_prev = alpha, beta
        rr = rr_new
        if rr <= tol * tol * bb:
            break
    return x, it


def rational_filter_shifts(lam: float, eps: float, order: int = 4):
    """(shifts, weights) of Eq. ratfilt: sigma_i = lam + i eps, i < order, and
    c_i = prod_{j != i} 1 / (sigma_j - sigma_i)."""
    sig = [lam + i * eps for i in range(order)]
    c = []
    for i in range(order):
        w = 1.0
        for j in range(order):
            if j != i:
                w /= (sig[j] - sig[i])
        c.append(w)
    return sig, c


def rational_filter(apply_H, eta, lam: float, eps: float, tol: float, order: int = 4):
    """prod_{i < order} (H + lam + i eps)^-1 eta by one multi-shift solve."""
    sig, c = rational_filter_shifts(lam, eps, order)
    xs, _ = multishift_cg(apply_H, eta, sig, tol)
    out = np.zeros_like(eta)
    for ci, xi in zip(c, xs):
        out = out + ci * xi
    return out


def wall_noise(n4: int, Ls: int, count: int, seed: int):
    """``count`` fields (count, n4, Ls, 4, 3): 4D Gaussian noise xi(x) (the
    shared generator, ``synthetic.complex_normal``, shape (count, n4, 4, 3))
    placed as P_- xi at s = 0 and P_+ xi at s = Ls - 1."""
    import synthetic as sy
    _, g5 = gamma_matrices()
    Pp = (np.eye(4) + g5) / 2
    Pm = (np.eye(4) - g5) / 2
    xi = sy.complex_normal(seed, (count, n4, 4, 3))
    out = np.zeros((count, n4, Ls, 4, 3), dtype=np.complex128)
    out[:, :, 0] = np.einsum("ab,kxbc->kxac", Pm, xi)
    out[:, :, Ls - 1] = np.einsum("ab,kxbc->kxac", Pp, xi)
    return out


def surface_truncate(phi, depth: int):
    """Zero the s-slices farther than ``depth`` from both walls (s < depth or
    s >= Ls - depth are kept).  ``phi`` (..., n4, Ls, 4, 3)."""
    out = np.array(phi, copy=True)
    Ls = out.shape[-3]
    keep = np.zeros(Ls, dtype=bool)
    keep[:depth] = True
    keep[Ls - depth:] = True
    out[..., ~keep, :, :] = 0
    return out


def rational_subspace(apply_H, blocking: Blocking, nvec: int, seed: int, lam: float, eps: float,
                      tol: float = 1e-6, depth: int = 0):
    """Nvec subspace vectors: wall noise, the rational filter, optionally the
    surface truncation, then block Gram-Schmidt."""
    d = blocking.dwf
    eta = wall_noise(d.lat.V // 2, d.Ls, nvec, seed)
    phi = np.stack([rational_filter(apply_H, e, lam, eps, tol) for e in eta])
    if depth:
        phi = surface_truncate(phi, depth)
    return block_gram_schmidt(phi, blocking)


def promote(phi, Ls: int):
    """(..., n4, Ls1, 4, 3) -> (..., n4, Ls, 4, 3): slices s < ceil(Ls1/2) stay
    at s, slices s >= ceil(Ls1/2) move to s + Ls - Ls1, the bulk is zero."""
    Ls1 = phi.shape[-3]
    if Ls1 > Ls:
        raise ValueError("the first-pass fifth dimension must not exceed Ls")
    h = (Ls1 + 1) // 2
    shape = phi.shape[:-3] + (Ls,) + phi.shape[-2:]
    out = np.zeros(shape, dtype=np.complex128)
    out[..., :h, :, :] = phi[..., :h, :, :]
    out[..., Ls - (Ls1 - h):, :, :] = phi[..., h:, :, :]
    return out


def two_pass_subspace(d: DWF, blocking: Blocking, nvec: int, seed: int, Ls1: int, mass1: float, lam: float,
                      eps: float, tol1: float, lam2: float = 0.0, tol2: float = 1e-3, depth: int = 0,
                      mirs_iter: int = 7, mirs_shift: float = 1.0):
    """The two-stage subspace: the rational filter on the Ls1, mass1 operator
    (same gauge field and 4D lattice), promotion to Ls, and with lam2 > 0 one
    solve of (H + lam2) x = v per promoted vector v by A-DEF2 deflated with
    the promoted vectors (relative residual tol2), then the surface truncation
    (depth > 0) and block Gram-Schmidt."""
    from .solvers import DeflationSpace, adef2
    d1 = DWF(d.lat.dims, Ls1, d.M5, d.b, d.c, mass1, d.U, antiperiodic_t=d.apbc)
    phi1 = rational_subspace(d1.mdagm, Blocking(d1, blocking.block), nvec, seed, lam, eps, tol=tol1)
    v = promote(phi1, d.Ls)
    if lam2 > 0:
        def Hs(x):
            return d.mdagm(x) + lam2 * x
        basis = block_gram_schmidt(v, blocking)
        A = dense_to_stencil(coarse_dense_bruteforce(d.mdagm, basis, blocking), blocking)
        A[:, 40] += lam2 * np.eye(nvec)
        defl = DeflationSpace(basis, blocking, A, coarse_tol=0.0)
        v = np.stack([adef2(Hs, vk, defl, tol2, mirs_iter=mirs_iter, mirs_shift=mirs_shift).x for vk in v])
    if depth:
        v = surface_truncate(v, depth)
    return block_gram_schmidt(v, blocking)
