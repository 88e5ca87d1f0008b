"""FP64 oracle: Krylov solvers of the HDCG method.

TEST INFRASTRUCTURE (see ``oracle/__init__``): never imported by the library.

* ``cg``       textbook (Hestenes-Stiefel) conjugate gradients on an HPD operator.
* ``mirs``     the infra-red shifted smoother M_IRS(H, N, lambda) = (H + lambda)^-1
               truncated to N CG iterations from a zero start (Sec. 4.3).
* ``inverse_iteration_subspace``  Gaussian vectors refined by steps of
               (H + lambda_s)^-1 and block Gram-Schmidt after each step
               (Sec. 1 and Sec. 5.2.1 name inverse iteration; step count,
               shift and tolerance are readings, not values printed by the paper).
* ``DeflationSpace``  Q = P A^-1 R (Sec. 2) with the coarse solve by CG to a
               relative residual (Table optimised: 0.04 inside the solver) or exact.
* ``ldop_deflation_space``  second-level (global, unblocked) deflation vectors
               of the little Dirac operator (Sec. 5.2, "Little Dirac operator
               deflation"): steps of shifted inverse iteration on Gaussian start
               vectors, each followed by a global Gram-Schmidt, then the
               prediagonalisation (Rayleigh-Ritz on their span) that makes the
               third, dense level diagonal.
* ``adef1``    the A-DEF1 method applied to the little Dirac operator with those
               vectors: V_start = 0, M_1 = M P_L + Q, M_2 = M_3 = 1 (Sec. 5.2,
               "Truncated little Dirac operator as preconditioner"), with the
               high-mode preconditioner M = 1 or M = ``qtrunc_chebyshev``.
               Reading: Table algos prints
               M_2 = P_R in the A-DEF1 row; with V_start = x that keeps every
               search direction out of span(Z), so the iteration cannot reach
               the deflated part of the solution (with a complete basis P_R = 0).
               The generalised algorithm's source (Tang et al., cited with
               Fig. pcg_general) has M_2 = 1 for A-DEF1, which is taken here.
* ``adef2``    generalised preconditioned CG of Fig. pcg_general with the
               A-DEF2 row of Table algos: V_start = Q b + P_R x, M_1 = P_R M_IRS + Q,
               M_2 = M_3 = 1.  ``flexible=True`` uses the Polak-Ribiere
               (flexible CG) beta = (r_{k+1}, y_{k+1} - y_k) / (r_k, y_k); the
               paper cites Notay's flexible CG without printing beta (reading).
* ``truncate_stencil``, ``chebyshev_inverse``, ``qtrunc_chebyshev``  the
               high-mode preconditioner of the A-DEF1 coarse solver: the
               Chebyshev approximation to the inverse of the range-truncated
               (0- and 1-hop) little Dirac operator Q_trunc (Sec. 5.2, Table
               frobnorm, Table hierarchy).

Random numbers drawn by the method (the Gaussian start vectors of the
subspace) are inputs to these functions.

Parity: ldop_deflation_space and adef1 are pinned by tests/test_oracle_ldop.py
(Rayleigh-Ritz interlacing and convergence to the exact lowest eigenvalues of
the dense little Dirac operator, prediagonal third level, A-DEF1 with the
complete eigenbasis is a direct solve, A-DEF1 reaches the dense solution in
fewer iterations than CG).
truncate_stencil, chebyshev_inverse and qtrunc_chebyshev are pinned by
tests/test_oracle_chebyshev.py (the scalar residual polynomial against
numpy's Chebyshev T_n, the 1/T_n(sigma) bound on the spectrum of a dense
Hermitian matrix, positivity on (0, hi], the 9 kept offsets and Hermiticity
of Q_trunc, A-DEF1 with M reaching the dense solution in fewer iterations,
and with no vectors reducing to CG, preconditioned or not).
cg, mirs, DeflationSpace and adef2 are pinned by
tests/test_oracle_solvers.py (true residual, free-field exact solution,
A-DEF2 invariants Q r_k = 0 and P_L r_k = r_k with exact Q, QH = 1 - P_R in
the block form of Sec. 2, deflated and undeflated solutions equal).
The iteration counts themselves are parity unpinned (the paper's counts use
gauge configurations that are not available).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .coarse import Blocking, block_gram_schmidt, coarse_apply, prolong, restrict, stencil_to_dense


def _dot(a, b):
    return complex(np.vdot(a.ravel(), b.ravel()))


def _n2(a):
    return float(np.vdot(a.ravel(), a.ravel()).real)


def cg(apply_A, b, tol, maxiter=100000, x0=None, history=None):
    """Solve A x = b (A HPD) until ||b - A x|| <= tol ||b|| (recursive residual).

    Returns (x, iterations).  The caller recomputes the true residual.
    """
    x = np.zeros_like(b) if x0 is None else np.array(x0, copy=True)
    r = b - apply_A(x) if x0 is not None else np.array(b, copy=True)
    p = r.copy()
    rr = _n2(r)
    bb = _n2(b)
    if bb == 0.0:
        return x, 0
    stop = tol * tol * bb
    it = 0
    while rr > stop and it < maxiter:
        w = apply_A(p)
        alpha = rr / _dot(p, w).real
        x = x + alpha * p
        r = r - alpha * w
        rr_new = _n2(r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
        if history is not None:
            history.append(np.sqrt(rr / bb))
    return x, it


def mirs(apply_H, r, n_iter: int = 7, shift: float = 1.0):
    """M_IRS(H, N, lambda) r: exactly ``n_iter`` CG iterations on (H + lambda) from zero."""
    x = np.zeros_like(r)
    res = np.array(r, copy=True)
    p = res.copy()
    rr = _n2(res)
    for _ in range(n_iter):
        if rr == 0.0:
            break
        w = apply_H(p) + shift * p
        alpha = rr / _dot(p, w).real
        x = x + alpha * p
        res = res - alpha * w
        rr_new = _n2(res)
        p = res + (rr_new / rr) * p
        rr = rr_new
    return x


def inverse_iteration_subspace(apply_H, noise, blocking: Blocking, steps: int = 3,
                               shift: float = 0.0, tol: float = 1e-4, maxiter: int = 100000):
    """Subspace by inverse iteration: phi <- block_GS((H + shift)^-1 phi), ``steps`` times.

    ``noise`` (Nvec, V/2, Ls, 4, 3) are the Gaussian start vectors.
    """
    phi = np.array(noise, dtype=np.complex128, copy=True)
    Hs = (lambda v: apply_H(v) + shift * v) if shift else apply_H
    for _ in range(steps):
        for k in range(phi.shape[0]):
            phi[k], _ = cg(Hs, phi[k], tol, maxiter)
        phi = block_gram_schmidt(phi, blocking)
    return phi


def _global_gram_schmidt(Z):
    """Modified Gram-Schmidt, applied twice, over whole (unblocked) coarse vectors."""
    Z = np.array(Z, dtype=np.complex128, copy=True)
    for _ in range(2):
        for i in range(Z.shape[0]):
            for j in range(i):
                Z[i] -= _dot(Z[j], Z[i]) * Z[j]
            Z[i] /= np.sqrt(_n2(Z[i]))
    return Z


def ldop_deflation_space(A, blocking: Blocking, noise, steps: int = 3, shift: float = 0.0,
                         tol: float = 1e-7, maxiter: int = 100000):
    """Global deflation vectors of the little Dirac operator A (Sec. 5.2).

    ``noise`` (nd, Vc, Nvec) are Gaussian start vectors.  Each of ``steps``
    steps replaces every vector by (A + shift)^-1 of it (CG to ``tol``, the
    paper's LittleDopSolverResidualSubspace) and then orthonormalises the set;
    finally the set is prediagonalised: with G = Z^dag A Z = S diag(lam) S^dag,
    Z <- Z S.  Returns (Z, AZ, lam), lam ascending, so Z^dag A Z = diag(lam).
    """
    Aop = lambda v: coarse_apply(A, v, blocking)
    As = (lambda v: Aop(v) + shift * v) if shift else Aop
    Z = np.array(noise, dtype=np.complex128, copy=True)
    for _ in range(steps):
        for i in range(Z.shape[0]):
            Z[i], _ = cg(As, Z[i], tol, maxiter)
        Z = _global_gram_schmidt(Z)
    nd = Z.shape[0]
    AZ = np.array([Aop(z) for z in Z])
    G = Z.reshape(nd, -1).conj() @ AZ.reshape(nd, -1).T
    G = 0.5 * (G + G.conj().T)
    lam, S = np.linalg.eigh(G)
    Zs = np.einsum("ik,i...->k...", S, Z)
    AZs = np.einsum("ik,i...->k...", S, AZ)
    return Zs, AZs, lam


def truncate_stencil(A, max_hops: int = 1):
    """Q_trunc of Sec. 5.2: the stencil restricted to the blocks at most
    ``max_hops`` block hops (taxicab) away; the 0- and 1-hop terms (9 of the
    81) for the paper's choice.  Dropping whole (l, -l) pairs keeps it
    Hermitian."""
    from .coarse import stencil_offsets
    hops = np.abs(stencil_offsets()).sum(axis=1)
    T = np.array(A, copy=True)
    T[:, hops > max_hops] = 0
    return T


def chebyshev_inverse(apply_M, r, order: int, lo: float, hi: float):
    """p(M) r, the Chebyshev approximation to M^-1 of order ``order`` on the
    interval [lo, hi] (Sec. 5.2 and Table hierarchy: order 16 on [0.5, 45],
    applied to Q_trunc).

    Reading: p is the degree order-1 polynomial of Chebyshev acceleration
    (the minimax polynomials the paper cites from Saad in Sec. 1), defined by
    1 - x p(x) = T_order((theta - x)/delta) / T_order(theta/delta) with
    theta = (hi + lo)/2 and delta = (hi - lo)/2.  So |1 - x p(x)| <=
    1/T_order(theta/delta) on [lo, hi], p > 0 on (0, hi] (a positive
    definite preconditioner for any M with spectrum there), and lo acts as
    the infra-red regulator: modes below lo are left partly uncorrected.

    Steps (the three-term recurrence of Chebyshev acceleration from y_0 = 0,
    s_0 = r): sigma = theta/delta, rho_0 = 1/sigma, d_0 = r/theta; then
    y_{k+1} = y_k + d_k, s_{k+1} = s_k - M d_k,
    rho_{k+1} = 1/(2 sigma - rho_k),
    d_{k+1} = rho_{k+1} rho_k d_k + (2 rho_{k+1}/delta) s_{k+1};
    y_order is returned after order-1 products with M.
    """
    if order < 1 or not 0 < lo < hi:
        raise ValueError("need order >= 1 and 0 < lo < hi")
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    sigma = theta / delta
    rho = 1.0 / sigma
    y = np.zeros_like(r)
    s = np.array(r, copy=True)
    d = r / theta
    for k in range(order):
        y = y + d
        if k == order - 1:
            break
        s = s - apply_M(d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * s
        rho = rho_new
    return y


def qtrunc_chebyshev(A, blocking: Blocking, order: int = 16, lo: float = 0.5, hi: float = 45.0,
                     shift: float = 0.0):
    """The A-DEF1 high-mode preconditioner of Sec. 5.2 (Table hierarchy):
    M = p(Q_trunc + shift) with Q_trunc the 0- and 1-hop part of the stencil
    A and p the order-``order`` Chebyshev approximation to 1/x on [lo, hi].
    ``shift`` is an explicit infra-red shift of Q_trunc (reading: the paper
    names one without a value; its tuned parameters give only [lo, hi], so 0
    by default).  Returns the map r -> M r."""
    T = truncate_stencil(A, 1)

    def apply_T(v):
        return coarse_apply(T, v, blocking) + shift * v

    return lambda r: chebyshev_inverse(apply_T, r, order, lo, hi)


def adef1(apply_A, b, Z, AZ, lam, tol: float, maxiter: int = 100000, flexible: bool = True,
          history=None, M=None):
    """A-DEF1 for A x = b with Q = Z diag(lam)^-1 Z^dag (M_2 = 1, see above) and
    the high-mode preconditioner M (default 1; the paper's choice is a
    Chebyshev polynomial of the shifted Q_trunc, ``qtrunc_chebyshev``).
    With no vectors (nd = 0) this is CG preconditioned by M.

    x_0 = 0, r_0 = b; y = M_1 r = M P_L r + Q r = M (r - A Q r) + Q r; p_0 = y_0; then
    w = A p, alpha = (r, y)/(p, w), x += alpha p, r -= alpha w, y' = M_1 r,
    beta = (r, y' - y)/(r_old, y_old) (flexible) or (r, y')/(r_old, y_old),
    p = y' + beta p.  A Q v = (A Z) diag(lam)^-1 Z^dag v uses the stored A Z, so
    every iteration applies A once.  Returns (x, iterations).
    """
    nd = Z.shape[0]
    Zf = Z.reshape(nd, b.size)
    AZf = AZ.reshape(nd, b.size)
    shape = b.shape

    def M1(r):
        d = (Zf.conj() @ r.ravel()) / lam
        if M is None:
            return r + ((Zf - AZf).T @ d).reshape(shape)
        return M(r - (AZf.T @ d).reshape(shape)) + (Zf.T @ d).reshape(shape)

    x = np.zeros_like(b)
    r = np.array(b, copy=True)
    bb = _n2(b)
    if bb == 0.0:
        return x, 0
    y = M1(r)
    p = y.copy()
    ry = _dot(r, y).real
    it = 0
    while it < maxiter:
        w = apply_A(p)
        alpha = ry / _dot(p, w).real
        x = x + alpha * p
        r = r - alpha * w
        it += 1
        rel = np.sqrt(_n2(r) / bb)
        if history is not None:
            history.append(rel)
        if rel <= tol:
            break
        y_new = M1(r)
        ry_new = _dot(r, y_new).real
        beta = (ry_new - _dot(r, y).real) / ry if flexible else ry_new / ry
        p = y_new + beta * p
        y = y_new
        ry = ry_new
    return x, it


@dataclass
class DeflationSpace:
    """Q = sum_{ab} |phi^a> (A^-1)^{ab} <phi^b| (Sec. 2) on an orthonormal block basis."""

    phi: np.ndarray
    blocking: Blocking
    A: np.ndarray                  # canonical stencil [Vc][81][N][N]
    coarse_tol: float = 0.0        # 0 -> exact dense solve
    coarse_maxiter: int = 100000
    coarse_iters: list = field(default_factory=list)
    ldop: tuple = None             # (Z, AZ, lam): coarse solve by A-DEF1 with these vectors
    # blocked second level (oracle.level2): the coarse solve is A-DEF2 on A with
    # this DeflationSpace of coarse vectors and the smoother level2_M (None: M = 1)
    level2: object = None
    level2_M: object = None

    def __post_init__(self):
        self._dense = None

    def dense(self):
        if self._dense is None:
            D = stencil_to_dense(self.A, self.blocking)
            n = D.shape[0] * D.shape[1]
            self._dense = D.reshape(n, n)
        return self._dense

    def coarse_solve(self, c):
        if self.coarse_tol == 0.0:
            return np.linalg.solve(self.dense(), c.ravel()).reshape(c.shape)
        Aop = lambda v: coarse_apply(self.A, v, self.blocking)
        if self.level2 is not None:
            M = self.level2_M if self.level2_M is not None else (lambda v: v)
            res = adef2(Aop, c, self.level2, self.coarse_tol, self.coarse_maxiter, M=M)
            y, it = res.x, res.iterations
        elif self.ldop is not None:
            y, it = adef1(Aop, c, *self.ldop, self.coarse_tol, self.coarse_maxiter)
        else:
            y, it = cg(Aop, c, self.coarse_tol, self.coarse_maxiter)
        self.coarse_iters.append(it)
        return y

    def R(self, v):
        return restrict(self.phi, v, self.blocking)

    def P(self, c):
        return prolong(self.phi, c, self.blocking)

    def Q(self, v):
        return self.P(self.coarse_solve(self.R(v)))


@dataclass
class SolveResult:
    x: np.ndarray
    iterations: int
    true_residual: float
    history: list
    invariants: list = field(default_factory=list)


def adef2(apply_H, b, defl: DeflationSpace, tol: float, maxiter: int = 10000,
          mirs_iter: int = 7, mirs_shift: float = 1.0, flexible: bool = True,
          x_guess=None, track_invariants: bool = False, apply_H_sloppy=None, M=None):
    """A-DEF2 preconditioned CG (Fig. pcg_general, Table algos row A-DEF2).

    x_0 = Q b + P_R x (x = x_guess or 0), r_0 = b - H x_0,
    y = M_1 r = z + Q (r - H z) with z = M_IRS r  (since P_R = 1 - Q H),
    p_0 = y_0; per iteration w = H p, alpha = (r, y)/(p, w), x += alpha p,
    r -= alpha w, y' = M_1 r, beta (flexible or standard), p = y' + beta p.
    Stops when the recursive residual reaches ``tol``; returns the true residual.
    ``apply_H_sloppy`` (default: ``apply_H``) is the operator inside M_1.
    ``M`` replaces M_IRS by another smoother z = M r (the level-1 solve of the
    three-level method uses M = 1 or the Chebyshev of Q_trunc).
    """
    Hs = apply_H if apply_H_sloppy is None else apply_H_sloppy
    Q = defl.Q
    if x_guess is None:
        x = Q(b)
    else:
        x = Q(b) + x_guess - Q(apply_H(x_guess))
    r = b - apply_H(x)
    bb = _n2(b)

    def M1(res):
        z = mirs(Hs, res, mirs_iter, mirs_shift) if M is None else M(res)
        return z + Q(res - Hs(z))

    y = M1(r)
    p = y.copy()
    ry = _dot(r, y).real
    hist = [np.sqrt(_n2(r) / bb)]
    inv = []
    it = 0
    while hist[-1] > tol and it < maxiter:
        w = apply_H(p)
        alpha = ry / _dot(p, w).real
        x = x + alpha * p
        r = r - alpha * w
        it += 1
        hist.append(np.sqrt(_n2(r) / bb))
        if track_invariants:
            qr = Q(r)
            inv.append((np.sqrt(_n2(qr) / _n2(r)), np.sqrt(_n2(apply_H(qr)) / _n2(r))))
        if hist[-1] <= tol:
            break
        y_new = M1(r)
        ry_new = _dot(r, y_new).real
        if flexible:
            beta = (ry_new - _dot(r, y).real) / ry
        else:
            beta = ry_new / ry
        p = y_new + beta * p
        y = y_new
        ry = ry_new
    true_res = np.sqrt(_n2(b - apply_H(x)) / bb)
    return SolveResult(x, it, true_res, hist, inv)
