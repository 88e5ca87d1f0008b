"""FP64 oracle: the red-black preconditioned Shamir / Moebius domain-wall operator.

TEST INFRASTRUCTURE (see ``oracle/__init__``): never imported by the library.

The paper fixes the operator only through its Schur form (Sec. 4, the
equation defining the Hermitian red-black operator):

    H = (M_oo - M_oe M_ee^-1 M_eo)^dag (M_oo - M_oe M_ee^-1 M_eo) = Mpc^dag Mpc

and states that M_ee^-1 is non-local in the fifth dimension for Moebius
fermions (Sec. 5.1).  The form of the 5D operator itself is not written in
the paper; this module uses the standard Moebius (Cayley) form, read as

    D psi_s = D_W (K psi)_s + ((1 - P_s) psi)_s,   K = b + c P_s,
    (P_s psi)_s = P_- psi_{s+1} + P_+ psi_{s-1},
    psi_{Ls} -> -m psi_0,  psi_{-1} -> -m psi_{Ls-1},
    D_W = (4 - M5) - Dh / 2,
    Dh psi(x) = sum_mu (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu),

Shamir being b = 1, c = 0.  With 4D red-black parity (origin even, the
solved system on odd sites):

    M_ee = M_oo = (4 - M5) K + 1 - P_s,     M_eo = -Dh_eo K / 2,  M_oe = -Dh_oe K / 2.

Gamma matrices are the chiral basis (gamma_5 = diag(1, 1, -1, -1)).

Parity: pinned by tests/test_oracle_dwf.py (dense Schur complement of the
textbook 5D operator, free-field closed form, adjoint identity, Hermiticity
and positivity, gauge covariance, stencil support, closed-form M_ee^-1).
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------
# gamma matrices
# ----------------------------------------------------------------------------

def gamma_matrices():
    """Chiral-basis Euclidean gammas: returns (g, g5) with g[mu], mu = x,y,z,t.

    g_k = [[0, -i sigma_k], [i sigma_k, 0]] (k = 1..3), g_4 = [[0, 1], [1, 0]],
    g5 = g1 g2 g3 g4 = diag(1, 1, -1, -1).
    """
    sig = [np.array([[0, 1], [1, 0]], dtype=np.complex128),
           np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
           np.array([[1, 0], [0, -1]], dtype=np.complex128)]
    g = np.zeros((4, 4, 4), dtype=np.complex128)
    for k in range(3):
        g[k, 0:2, 2:4] = -1j * sig[k]
        g[k, 2:4, 0:2] = 1j * sig[k]
    g[3, 0:2, 2:4] = np.eye(2)
    g[3, 2:4, 0:2] = np.eye(2)
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


# ----------------------------------------------------------------------------
# lattice indexing
# ----------------------------------------------------------------------------

class Lattice:
    """4D periodic lattice with even-odd (red-black) checkerboarding.

    ``lex = x + Lx*(y + Ly*(z + Lz*t))``; parity ``(x+y+z+t) % 2``;
    checkerboard index ``cb = lex >> 1`` (requires even extents).
    ``sites[p]`` lists the lex indices of parity ``p`` in checkerboard order.
    """

    def __init__(self, dims):
        self.dims = tuple(int(d) for d in dims)
        if len(self.dims) != 4 or any(d < 2 or d % 2 for d in self.dims):
            raise ValueError("extents must be four even numbers")
        self.V = int(np.prod(self.dims))
        lex = np.arange(self.V)
        Lx, Ly, Lz, _ = self.dims
        self.coords = np.stack([lex % Lx, (lex // Lx) % Ly,
                                (lex // (Lx * Ly)) % Lz, lex // (Lx * Ly * Lz)], axis=1)
        self.parity = self.coords.sum(axis=1) % 2
        self.sites = [lex[self.parity == 0], lex[self.parity == 1]]
        for p in (0, 1):
            assert np.array_equal(self.sites[p] >> 1, np.arange(self.V // 2))

    def lex_of(self, coords):
        c = np.asarray(coords) % np.array(self.dims)
        Lx, Ly, Lz, _ = self.dims
        return c[..., 0] + Lx * (c[..., 1] + Ly * (c[..., 2] + Lz * c[..., 3]))

    def neighbour(self, lex, mu: int, step: int):
        """lex index of x + step * mu_hat (periodic)."""
        c = self.coords[lex].copy()
        c[..., mu] += step
        return self.lex_of(c)


# ----------------------------------------------------------------------------
# Wilson hop on the checkerboard
# ----------------------------------------------------------------------------

def hop(lat: Lattice, U, psi_in, out_parity: int, dagger: bool = False,
        antiperiodic_t: bool = False):
    """Dh restricted to output sites of ``out_parity`` (input: the other parity).

    Dh psi(x) = sum_mu (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu).
    ``dagger=True`` gives Dh^dag, which is Dh with g_mu -> -g_mu.
    Antiperiodic time: a hop across the t boundary picks up a factor -1.
    Fields are checkerboard arrays of shape (V/2, Ls, 4, 3).
    """
    g, _ = gamma_matrices()
    sgn = -1.0 if dagger else 1.0
    one = np.eye(4)
    out_lex = lat.sites[out_parity]
    Lt = lat.dims[3]
    out = np.zeros(psi_in.shape, dtype=np.complex128)
    for mu in range(4):
        fwd = lat.neighbour(out_lex, mu, +1)
        bwd = lat.neighbour(out_lex, mu, -1)
        Uf = U[out_lex, mu]
        Ub = np.conj(np.transpose(U[bwd, mu], (0, 2, 1)))
        if antiperiodic_t and mu == 3:
            t = lat.coords[out_lex, 3]
            Uf = Uf * np.where(t == Lt - 1, -1.0, 1.0)[:, None, None]
            Ub = Ub * np.where(t == 0, -1.0, 1.0)[:, None, None]
        out += spin_mul(one - sgn * g[mu], colour_mul(Uf, psi_in[fwd >> 1]))
        out += spin_mul(one + sgn * g[mu], colour_mul(Ub, psi_in[bwd >> 1]))
    return out


def colour_mul(U, psi):
    """(U psi)[n, s, i, a] = sum_b U[n, a, b] psi[n, s, i, b]."""
    return np.matmul(psi, np.transpose(U, (0, 2, 1))[:, None])


def spin_mul(G, psi):
    """(G psi)[n, s, i, a] = sum_j G[i, j] psi[n, s, j, a]."""
    return np.matmul(G, psi)


def twisted_gauge(U, theta):
    """Links for twisted boundary conditions (Sec. 6.4, "Subspace reuse", Table
    twist): psi(x + L_mu) = e^{i L_mu theta_mu} psi(x) is, after the U(1) gauge
    transformation psi -> e^{-i theta.x} psi, the same operator as uniform link
    phases U_mu(x) -> e^{i theta_mu} U_mu(x); the paper's twist (pi/L)(a, b, c)
    is theta_mu = pi a_mu / L_mu."""
    return np.asarray(U, dtype=np.complex128) * np.exp(1j * np.asarray(theta, dtype=float))[None, :, None, None]


# ----------------------------------------------------------------------------
# fifth-dimension operators (site independent, real, 4Ls x 4Ls over (s, spin))
# ----------------------------------------------------------------------------

def s_operators(Ls: int, M5: float, b: float, c: float, m: float):
    """Dense (4Ls x 4Ls) matrices over the index (s, spin):

    ``Ps`` (P_s), ``K`` = b + c P_s, ``Mee`` = (4 - M5) K + 1 - P_s and
    ``Meeinv`` = Mee^-1 by dense LU (numpy.linalg.inv).
    """
    if Ls < 2:
        raise ValueError("Ls >= 2")
    _, g5 = gamma_matrices()
    Pp = ((np.eye(4) + g5) / 2).real
    Pm = ((np.eye(4) - g5) / 2).real
    Ps = np.zeros((Ls, 4, Ls, 4))
    for s in range(Ls):
        if s + 1 < Ls:
            Ps[s, :, s + 1, :] += Pm
        else:
            Ps[s, :, 0, :] += -m * Pm
        if s - 1 >= 0:
            Ps[s, :, s - 1, :] += Pp
        else:
            Ps[s, :, Ls - 1, :] += -m * Pp
    Ps = Ps.reshape(4 * Ls, 4 * Ls)
    one = np.eye(4 * Ls)
    K = b * one + c * Ps
    Mee = (4.0 - M5) * K + one - Ps
    return {"Ps": Ps, "K": K, "Mee": Mee, "Meeinv": np.linalg.inv(Mee)}


def apply_s(M, psi):
    """out[n, s, i, a] = sum_{s', j} M[(s, i), (s', j)] psi[n, s', j, a]."""
    n, Ls = psi.shape[0], psi.shape[1]
    r = psi.reshape(n, 4 * Ls, 3)
    return np.matmul(M, r).reshape(psi.shape)


# ----------------------------------------------------------------------------
# the Schur-complement operator and H
# ----------------------------------------------------------------------------

class DWF:
    """Red-black preconditioned Moebius/Shamir operator on the odd checkerboard."""

    def __init__(self, dims, Ls, M5, b, c, mass, U, antiperiodic_t=False):
        self.lat = Lattice(dims)
        self.Ls = int(Ls)
        self.M5, self.b, self.c, self.mass = float(M5), float(b), float(c), float(mass)
        self.U = np.asarray(U, dtype=np.complex128)
        if self.U.shape != (self.lat.V, 4, 3, 3):
            raise ValueError("gauge field must have shape (V, 4, 3, 3)")
        self.apbc = bool(antiperiodic_t)
        self.S = s_operators(self.Ls, self.M5, self.b, self.c, self.mass)

    @property
    def field_shape(self):
        return (self.lat.V // 2, self.Ls, 4, 3)

    def _hop(self, psi, out_parity, dagger=False):
        return hop(self.lat, self.U, psi, out_parity, dagger, self.apbc)

    def mpc(self, psi):
        """Mpc psi = M_oo psi - (1/4) Dh_oe K Mee^-1 Dh_eo K psi."""
        S = self.S
        t = apply_s(S["K"], psi)
        t = self._hop(t, 0)
        t = apply_s(S["Meeinv"], t)
        t = apply_s(S["K"], t)
        t = self._hop(t, 1)
        return apply_s(S["Mee"], psi) - 0.25 * t

    def mpc_dag(self, chi):
        """Mpc^dag chi = M_oo^dag chi - (1/4) K^dag (Dh_eo)^dag Mee^-dag K^dag (Dh_oe)^dag chi.

        (Dh_oe)^dag is (Dh^dag) from odd to even sites; all s-operators are real.
        """
        S = self.S
        t = self._hop(chi, 0, dagger=True)
        t = apply_s(S["K"].T, t)
        t = apply_s(S["Meeinv"].T, t)
        t = self._hop(t, 1, dagger=True)
        t = apply_s(S["K"].T, t)
        return apply_s(S["Mee"].T, chi) - 0.25 * t

    def mdagm(self, psi):
        """H psi = Mpc^dag Mpc psi."""
        return self.mpc_dag(self.mpc(psi))

    # -- the full (unpreconditioned) system and its Schur-form reduction (Sec. 4) --
    # D = [[M_ee, M_eo], [M_oe, M_oo]] on (even, odd) sites with
    # M_ee = M_oo = (4 - M5) K + 1 - P_s and M_eo, M_oe = -1/2 Dh K.

    def apply_full(self, psi_e, psi_o):
        """(eta_e, eta_o) = D (psi_e, psi_o)."""
        S = self.S
        eta_e = apply_s(S["Mee"], psi_e) - 0.5 * self._hop(apply_s(S["K"], psi_o), 0)
        eta_o = apply_s(S["Mee"], psi_o) - 0.5 * self._hop(apply_s(S["K"], psi_e), 1)
        return eta_e, eta_o

    def prep_source(self, eta_e, eta_o):
        """b = Mpc^dag (eta_o - M_oe M_ee^-1 eta_e): the right-hand side of the
        odd-site normal equation H psi_o = b whose solution is the odd half of
        D psi = eta."""
        S = self.S
        eta_p = eta_o + 0.5 * self._hop(apply_s(S["K"], apply_s(S["Meeinv"], eta_e)), 1)
        return self.mpc_dag(eta_p)

    def reconstruct(self, eta_e, psi_o):
        """psi_e = M_ee^-1 (eta_e - M_eo psi_o), the even half of the solution."""
        S = self.S
        return apply_s(S["Meeinv"], eta_e + 0.5 * self._hop(apply_s(S["K"], psi_o), 0))

    def mdagm_shift(self, psi, shift):
        return self.mdagm(psi) + shift * psi


def inner(a, b) -> complex:
    """<a, b> = sum conj(a) b over all components."""
    return complex(np.vdot(a.ravel(), b.ravel()))


def norm2(a) -> float:
    return float(np.vdot(a.ravel(), a.ravel()).real)
