"""FP64 oracle: the generalised preconditioned CG and its family of
preconditioners (Sec. 4.5, Fig. pcg_general, Tables precs and algos).

TEST INFRASTRUCTURE (see ``oracle/__init__``): never imported by the library.

* ``generalised_pcg``  Fig. pcg_general: x_0 = V_start, r_0 = b - H x_0,
               y_0 = M_1 r_0, p_0 = M_2 y_0; per iteration w = M_3 H p,
               alpha = (r, y)/(p, w), x += alpha p, r -= alpha w, y = M_1 r,
               beta = (r_new, y_new)/(r, y) (or the flexible form), p = M_2 y +
               beta p; x = V_end.
* ``METHODS``  Table algos: PREC, AD, DEF1, DEF2, A-DEF1, A-DEF2, BNN, the
               Hermitian V(1,1) multigrid cycle and MssDef, built from
               Q = P A^-1 R and a smoother M, with P_L = 1 - H Q and
               P_R = 1 - Q H.
               Readings: (i) DEF1 (M_3 = P_L) iterates on the deflated system
               P_L H x = P_L b, so its start residual is P_L (b - H x_0); with
               the unprojected residual of the figure the recursion could not
               reach zero.  (ii) A-DEF1 takes M_2 = 1 (the table prints P_R;
               see ``solvers.adef1``).  (iii) BNN may start from x or from the
               DEF2 start Q b + P_R x (the equivalence of Sec. 4.5 holds for
               suitably chosen start vectors).
               (iv) MssDef, the little Dirac operator as the only
               preconditioner with no smoother, is A-DEF2 with M = 1:
               V_start = Q b + P_R x and M_1 = P_R + Q.
* ``ChebyshevSmoother``  the Chebyshev option of Table preconditioner: the
               order-n Chebyshev approximation to H^-1 on [lo, hi]
               (``solvers.chebyshev_inverse`` with H in place of Q_trunc), a
               fixed polynomial in H, so linear and Hermitian.
* ``MirsPoly``  M_IRSpoly (Table preconditioner): the CG polynomial of a fixed
               number of iterations on H + lambda, frozen from one CG pass on a
               reference vector (its alpha_k and beta_k) and replayed on any
               vector, so it is a fixed linear, Hermitian operator.

Parity: pinned by tests/test_oracle_pcg_family.py (PREC with M = 1 is the
textbook CG, residual by residual; each M_1 equals its form as smoothing and
coarse-correction steps, V(1,1) the symmetric two-grid cycle; every method reaches the CG solution; MssDef iterates as DEF2 with M = 1 (the same equivalence);
A-DEF2 with the Chebyshev smoother reaches it too, and that smoother is the
polynomial of its eigenvalues (checked on a dense Hermitian matrix) and
Hermitian; with exact Q and a linear smoother DEF2, A-DEF2 and BNN from the
DEF2 start produce the same iterates, and DEF1's V_end the same solution, as
the equivalence of Sec. 4.5 states; the V(1,1) and BNN preconditioners are
Hermitian; M_IRSpoly reproduces M_IRS on its reference vector and is linear
and Hermitian).
"""
from __future__ import annotations

import numpy as np

from .solvers import DeflationSpace, chebyshev_inverse


def _dot(a, b):
    return np.vdot(a, b)


def _n2(a):
    return float(np.vdot(a, a).real)


class MirsPoly:
    """M_IRSpoly(H, N, lambda): N CG iterations on H + lambda from zero for the
    reference vector, their alpha_k and beta_k recorded; ``__call__`` replays
    the same recurrences (a fixed polynomial in H of degree N - 1)."""

    def __init__(self, apply_H, r_ref, n_iter: int = 7, shift: float = 1.0):
        self.apply_H, self.shift = apply_H, shift
        self.alpha, self.beta = [], []
        res = np.array(r_ref, copy=True)
        p = res.copy()
        rr = _n2(res)
        for k in range(n_iter):
            w = apply_H(p) + shift * p
            a = rr / _dot(p, w).real
            res = res - a * w
            rr_new = _n2(res)
            self.alpha.append(a)
            self.beta.append(rr_new / rr)
            p = res + self.beta[-1] * p
            rr = rr_new

    def __call__(self, v):
        x = np.zeros_like(v)
        r = np.array(v, copy=True)
        p = r.copy()
        for a, bt in zip(self.alpha, self.beta):
            x = x + a * p
            r = r - a * (self.apply_H(p) + self.shift * p)
            p = r + bt * p
        return x


class ChebyshevSmoother:
    """p(H): order ``order`` (PreconditionerKrylovIterMax) on [lo, hi]
    (PreconditionerKrylovLo, PreconditionerKrylovHi)."""

    def __init__(self, apply_H, order: int, lo: float, hi: float):
        self.apply_H, self.order, self.lo, self.hi = apply_H, order, lo, hi

    def __call__(self, v):
        return chebyshev_inverse(self.apply_H, v, self.order, self.lo, self.hi)


def _ops(apply_H, defl: DeflationSpace, M):
    Q = defl.Q

    def PL(v):          # P_L = 1 - H Q
        return v - apply_H(Q(v))

    def PR(v):          # P_R = 1 - Q H
        return v - Q(apply_H(v))

    return Q, PL, PR


def method(name: str, apply_H, defl: DeflationSpace, M):
    """(V_start, M_1, M_2, M_3, V_end, project_r0) of Table algos for ``name``."""
    Q, PL, PR = _ops(apply_H, defl, M)
    ident = lambda v: v

    def start_x(b, x):
        return x

    def start_def2(b, x):
        return Q(b) + PR(x)

    def end_x(b, x):
        return x

    def end_def1(b, x):
        return Q(b) + PR(x)

    if name == "PREC":
        return start_x, M, ident, ident, end_x, False
    if name == "AD":
        return start_x, lambda r: M(r) + Q(r), ident, ident, end_x, False
    if name == "DEF1":
        return start_x, M, ident, PL, end_def1, True
    if name == "DEF2":
        return start_def2, M, PR, ident, end_x, False
    if name == "A-DEF1":
        return start_x, lambda r: M(PL(r)) + Q(r), ident, ident, end_x, False
    if name == "A-DEF2":
        return start_def2, lambda r: PR(M(r)) + Q(r), ident, ident, end_x, False
    if name == "BNN":
        return start_x, lambda r: PR(M(PL(r))) + Q(r), ident, ident, end_x, False
    if name == "BNN-DEF2-start":
        return start_def2, lambda r: PR(M(PL(r))) + Q(r), ident, ident, end_x, False
    if name == "MssDef":
        return start_def2, lambda r: PR(r) + Q(r), ident, ident, end_x, False
    if name == "V11":
        def m1(r):
            mr = M(r)
            return M(PL(r)) + PR(mr) + Q(r) - M(PL(apply_H(mr)))
        return start_x, m1, ident, ident, end_x, False
    raise ValueError(f"unknown method {name}")


METHODS = ("PREC", "AD", "DEF1", "DEF2", "A-DEF1", "A-DEF2", "BNN", "BNN-DEF2-start", "V11", "MssDef")


def generalised_pcg(name: str, apply_H, b, defl: DeflationSpace, M, tol: float, maxiter: int = 10000,
                    x_guess=None, flexible: bool = False, history=None):
    """Fig. pcg_general with the row ``name`` of Table algos.  Stops when the
    recursive residual reaches ``tol`` relative to |b|; ``history`` (a list)
    receives the iterates x_k (after V_end) if given.  Returns (x, iterations)."""
    Vs, M1, M2, M3, Ve, proj = method(name, apply_H, defl, M)
    _, PL, _ = _ops(apply_H, defl, M)
    x = Vs(b, np.zeros_like(b) if x_guess is None else x_guess)
    r = b - apply_H(x)
    if proj:
        r = PL(r)
    bb = _n2(b)
    y = M1(r)
    p = M2(y)
    ry = _dot(r, y).real
    it = 0
    while it < maxiter and np.sqrt(_n2(r) / bb) > tol:
        w = M3(apply_H(p))
        alpha = ry / _dot(p, w).real
        x = x + alpha * p
        r = r - alpha * w
        it += 1
        if history is not None:
            history.append(Ve(b, x))
        if np.sqrt(_n2(r) / bb) <= tol:
            break
        y_new = M1(r)
        ry_new = _dot(r, y_new).real
        beta = (ry_new - _dot(r, y).real) / ry if flexible else ry_new / ry
        p = M2(y_new) + beta * p
        y, ry = y_new, ry_new
    return Ve(b, x), it
