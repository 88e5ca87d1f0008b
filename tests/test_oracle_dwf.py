"""Pins of the FP64 oracle's fine operator against facts fixed by the paper and
by the mathematics (no GPU).  Each test would fail on a plausible mistake in
oracle/dwf.py: a wrong projector pairing, sign, link direction, dagger,
checkerboard index, misplaced K or a dropped wall term."""
import itertools

import numpy as np
import pytest

import synthetic as sy
from oracle.dwf import DWF, Lattice, gamma_matrices, inner, norm2, s_operators

# ----------------------------------------------------------------------------
# gamma matrices and indexing
# ----------------------------------------------------------------------------


def test_gamma_clifford_algebra():
    g, g5 = gamma_matrices()
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            ac = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(ac, 2 * np.eye(4) * (mu == nu))
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))


@pytest.mark.parametrize("dims", [(4, 6, 2, 4), (2, 2, 2, 2), (6, 4, 4, 2)])
def test_checkerboard_and_neighbours_bruteforce(dims):
    lat = Lattice(dims)
    Lx, Ly, Lz, Lt = dims
    seen = {0: set(), 1: set()}
    for t, z, y, x in itertools.product(range(Lt), range(Lz), range(Ly), range(Lx)):
        lex = x + Lx * (y + Ly * (z + Lz * t))
        p = (x + y + z + t) % 2
        assert lat.parity[lex] == p
        cb = lex >> 1
        assert cb not in seen[p]
        seen[p].add(cb)
        assert lat.sites[p][cb] == lex
        c = [x, y, z, t]
        for mu in range(4):
            for step in (+1, -1):
                d = list(c)
                d[mu] = (d[mu] + step) % dims[mu]
                nlex = d[0] + Lx * (d[1] + Ly * (d[2] + Lz * d[3]))
                assert lat.neighbour(np.array([lex]), mu, step)[0] == nlex
                assert lat.parity[nlex] == 1 - p
    assert seen[0] == seen[1] == set(range(lat.V // 2))


# ----------------------------------------------------------------------------
# fifth dimension: closed-form M_ee^-1
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("Ls,M5,b,c,m", [(8, 1.8, 1.0, 0.0, 0.01), (16, 1.8, 1.5, 0.5, 0.002),
                                          (5, 1.2, 2.0, 1.0, 0.3), (4, 1.8, 1.5, 0.5, 0.0)])
def test_meeinv_closed_form_geometric_series(Ls, M5, b, c, m):
    """Per chirality M_ee = alpha (1 - T), T = -(beta/alpha) S, S^Ls = -m, so
    M_ee^-1 = (1/alpha) sum_{k<Ls} T^k / (1 + m (-beta/alpha)^Ls)."""
    S = s_operators(Ls, M5, b, c, m)
    alpha = b * (4 - M5) + 1
    beta = c * (4 - M5) - 1
    r = -beta / alpha
    norm = 1.0 / (alpha * (1 + m * r ** Ls))
    inv = S["Meeinv"].reshape(Ls, 4, Ls, 4)
    for spin in range(4):
        up = spin >= 2          # chirality minus (gamma5 = -1): S shifts s -> s+1
        for s in range(Ls):
            for k in range(Ls):
                sp = s + k if up else s - k
                f = 1.0
                if sp >= Ls:
                    sp -= Ls
                    f = -m
                if sp < 0:
                    sp += Ls
                    f = -m
                assert inv[s, spin, sp, spin] == pytest.approx(norm * r ** k * f, abs=1e-13)
        # no mixing between spins
        for spin2 in range(4):
            if spin2 != spin:
                assert np.abs(inv[:, spin, :, spin2]).max() == 0.0


# ----------------------------------------------------------------------------
# Schur complement of the textbook (unpreconditioned) 5D operator
# ----------------------------------------------------------------------------

def _textbook_5d_dense(dims, Ls, M5, b, c, m, U, apbc):
    """Dense unpreconditioned Moebius operator, written out with loops:
    D psi_s = (b D_W + 1) psi_s + (c D_W - 1)(P_- psi_{s+1} + P_+ psi_{s-1}),
    P_- psi_{Ls} = -m P_- psi_0, P_+ psi_{-1} = -m P_+ psi_{Ls-1},
    D_W psi(x) = (4 - M5) psi(x) - 1/2 sum_mu [(1 - g_mu) U_mu(x) psi(x + mu)
                                              + (1 + g_mu) U_mu(x - mu)^dag psi(x - mu)].
    Index order: (parity-major checkerboard site, s, spin, colour)."""
    g, g5 = gamma_matrices()
    Lx, Ly, Lz, Lt = dims
    V = Lx * Ly * Lz * Lt
    coords = [(x, y, z, t) for t in range(Lt) for z in range(Lz) for y in range(Ly) for x in range(Lx)]

    def lex(c4):
        x, y, z, t = [c4[i] % dims[i] for i in range(4)]
        return x + Lx * (y + Ly * (z + Lz * t))

    def row(lx):   # position of the 4D site in (even sites, then odd sites) order
        x, y, z, t = coords[lx]
        return ((x + y + z + t) % 2) * (V // 2) + (lx >> 1)

    DW = np.zeros((V, 12, V, 12), dtype=np.complex128)
    for lx in range(V):
        DW[row(lx), :, row(lx), :] += (4 - M5) * np.eye(12)
        for mu in range(4):
            c4 = list(coords[lx])
            c4[mu] += 1
            ly = lex(c4)
            u = U[lx, mu].copy()
            if apbc and mu == 3 and coords[lx][3] == Lt - 1:
                u = -u
            # forward: x -> x + mu with (1 - g) U_mu(x)
            DW[row(lx), :, row(ly), :] += -0.5 * np.kron(np.eye(4) - g[mu], u)
            # backward: from y = x + mu to x with (1 + g) U_mu(x)^dag
            DW[row(ly), :, row(lx), :] += -0.5 * np.kron(np.eye(4) + g[mu], u.conj().T)
    DW = DW.reshape(V * 12, V * 12)
    Pp = np.kron(np.eye(V), np.kron((np.eye(4) + g5) / 2, np.eye(3)))
    Pm = np.kron(np.eye(V), np.kron((np.eye(4) - g5) / 2, np.eye(3)))
    one = np.eye(V * 12)
    N = V * 12
    D = np.zeros((V, Ls, 12, V, Ls, 12), dtype=np.complex128)

    def put(s, sp, blk):
        D[:, s, :, :, sp, :] += blk.reshape(V, 12, V, 12)

    for s in range(Ls):
        put(s, s, b * DW + one)
        hop5 = c * DW - one
        if s + 1 < Ls:
            put(s, s + 1, hop5 @ Pm)
        else:
            put(s, 0, -m * hop5 @ Pm)
        if s - 1 >= 0:
            put(s, s - 1, hop5 @ Pp)
        else:
            put(s, Ls - 1, -m * hop5 @ Pp)
    half = V // 2 * Ls * 12
    D = D.reshape(2 * half, 2 * half)
    assert D.shape[0] == N * Ls
    return D, half


@pytest.mark.parametrize("params", [
    dict(dims=(4, 2, 2, 2), Ls=4, M5=1.8, b=1.0, c=0.0, m=0.01, apbc=False),
    dict(dims=(2, 2, 4, 2), Ls=4, M5=1.8, b=1.5, c=0.5, m=0.02, apbc=True),
    dict(dims=(2, 4, 2, 2), Ls=3, M5=1.4, b=2.0, c=1.0, m=0.1, apbc=False),
])
def test_mpc_equals_dense_schur_complement(params):
    p = params
    U = sy.gauge_field(p["dims"], 0.7, 11)
    d = DWF(p["dims"], p["Ls"], p["M5"], p["b"], p["c"], p["m"], U, antiperiodic_t=p["apbc"])
    D, half = _textbook_5d_dense(p["dims"], p["Ls"], p["M5"], p["b"], p["c"], p["m"], U, p["apbc"])
    Dee, Deo = D[:half, :half], D[:half, half:]
    Doe, Doo = D[half:, :half], D[half:, half:]
    S = Doo - Doe @ np.linalg.solve(Dee, Deo)
    Mpc = np.zeros_like(S)
    Mdag = np.zeros_like(S)
    shape = d.field_shape
    for j in range(half):
        e = np.zeros(half, dtype=np.complex128)
        e[j] = 1.0
        Mpc[:, j] = d.mpc(e.reshape(shape)).ravel()
        Mdag[:, j] = d.mpc_dag(e.reshape(shape)).ravel()
    assert np.abs(Mpc - S).max() < 1e-12 * np.abs(S).max()
    assert np.abs(Mdag - S.conj().T).max() < 1e-12 * np.abs(S).max()
    Hd = Mdag @ Mpc
    ev = np.linalg.eigvalsh((Hd + Hd.conj().T) / 2)
    assert ev.min() > 0
    for j in range(0, half, 97):
        e = np.zeros(half, dtype=np.complex128)
        e[j] = 1.0
        assert np.allclose(d.mdagm(e.reshape(shape)).ravel(), (S.conj().T @ S)[:, j], atol=1e-12)


# ----------------------------------------------------------------------------
# adjoint, Hermiticity, positivity
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("bc", [(1.0, 0.0), (1.5, 0.5)])
def test_adjoint_hermitian_positive(bc):
    dims, Ls = (4, 4, 4, 4), 6
    U = sy.gauge_field(dims, 0.4, 5)
    d = DWF(dims, Ls, 1.8, bc[0], bc[1], 0.01, U, antiperiodic_t=True)
    u = sy.gaussian_fermion(dims, Ls, 6)
    v = sy.gaussian_fermion(dims, Ls, 7)
    a = inner(u, d.mpc(v))
    bq = inner(d.mpc_dag(u), v)
    assert abs(a - bq) < 1e-13 * abs(a)
    Hv, Hu = d.mdagm(v), d.mdagm(u)
    assert abs(inner(u, Hv) - np.conj(inner(v, Hu))) < 1e-13 * abs(inner(u, Hv))
    assert inner(v, Hv).real == pytest.approx(norm2(d.mpc(v)), rel=1e-13)
    assert abs(inner(v, Hv).imag) < 1e-12 * inner(v, Hv).real
    assert inner(v, Hv).real > 0


# ----------------------------------------------------------------------------
# free field: closed-form momentum-space operator
# ----------------------------------------------------------------------------

def _free_mpc_p(p, S):
    """Mpc(p) = M_ee - 1/4 Dh(p) K M_ee^-1 Dh(p) K with Dh(p) = 2 sum cos p - 2 i sum g sin p."""
    g, _ = gamma_matrices()
    Ls = S["K"].shape[0] // 4
    dh4 = 2 * sum(np.cos(p[m]) for m in range(4)) * np.eye(4) \
        - 2j * sum(g[m] * np.sin(p[m]) for m in range(4))
    dh = np.kron(np.eye(Ls), dh4)
    return S["Mee"] - 0.25 * dh @ S["K"] @ S["Meeinv"] @ dh @ S["K"]


@pytest.mark.parametrize("bc", [(1.0, 0.0), (1.5, 0.5)])
def test_free_field_plane_waves(bc):
    dims, Ls = (4, 6, 4, 8), 4
    d = DWF(dims, Ls, 1.8, bc[0], bc[1], 0.02, sy.unit_gauge(dims))
    odd = d.lat.sites[1]
    x = d.lat.coords[odd].astype(float)
    rng = np.random.default_rng(0)
    for n in [(0, 0, 0, 0), (1, 0, 0, 0), (1, 2, 3, 4), (3, 5, 1, 7), (2, 3, 2, 4)]:
        p = 2 * np.pi * np.array(n) / np.array(dims)
        e = rng.standard_normal((Ls, 4)) + 1j * rng.standard_normal((Ls, 4))
        colour = 1
        psi = np.zeros(d.field_shape, dtype=np.complex128)
        phase = np.exp(1j * x @ p)
        psi[:, :, :, colour] = phase[:, None, None] * e[None]
        Mp = _free_mpc_p(p, d.S)
        want = (Mp.conj().T @ Mp @ e.ravel()).reshape(Ls, 4)
        got = d.mdagm(psi)
        assert np.abs(got[:, :, :, colour] - phase[:, None, None] * want[None]).max() < 1e-12 * np.abs(want).max()
        assert np.abs(got[:, :, :, [0, 2]]).max() == 0.0


def test_free_field_full_spectrum():
    """Dense H on a tiny free lattice: its spectrum is the union over the V/2
    odd-site momentum classes of eig(Mpc(p)^dag Mpc(p)), each three times (colour)."""
    dims, Ls = (4, 2, 2, 2), 4
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.05, sy.unit_gauge(dims))
    n = int(np.prod(d.field_shape))
    Hd = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1
        Hd[:, j] = d.mdagm(e.reshape(d.field_shape)).ravel()
    ev = np.sort(np.linalg.eigvalsh((Hd + Hd.conj().T) / 2))
    want = []
    # p and p + (pi, pi, pi, pi) coincide on odd sites; take n_t = 0 representatives
    for nx, ny, nz in itertools.product(range(4), range(2), range(2)):
        p = 2 * np.pi * np.array([nx, ny, nz, 0]) / np.array(dims)
        Mp = _free_mpc_p(p, d.S)
        want += list(np.linalg.eigvalsh(Mp.conj().T @ Mp)) * 3
    want = np.sort(np.array(want))
    assert len(want) == n
    assert np.abs(ev - want).max() < 1e-11 * want.max()


# ----------------------------------------------------------------------------
# gauge covariance
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("apbc", [False, True])
def test_gauge_covariance(apbc):
    dims, Ls = (4, 4, 2, 4), 4
    U = sy.gauge_field(dims, 0.5, 21)
    lat = Lattice(dims)
    g = sy.random_su3(22, lat.V, 1.0)
    Up = np.empty_like(U)
    for mu in range(4):
        nb = lat.neighbour(np.arange(lat.V), mu, +1)
        Up[:, mu] = g @ U[:, mu] @ np.conj(np.transpose(g[nb], (0, 2, 1)))
    d0 = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.01, U, antiperiodic_t=apbc)
    d1 = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.01, Up, antiperiodic_t=apbc)
    psi = sy.gaussian_fermion(dims, Ls, 23)
    go = g[lat.sites[1]]
    rot = lambda f: np.einsum("nab,nsib->nsia", go, f)
    lhs = d1.mdagm(rot(psi))
    rhs = rot(d0.mdagm(psi))
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()


# ----------------------------------------------------------------------------
# stencil support: the paper's 320 neighbours (taxicab <= 4).  On the odd
# sublattice only even taxicab offsets couple (225 with self), and the eight
# straight offsets +-4 mu vanish exactly: the straight two-hop factor of Mpc is
# (s-matrix, identity in spin)(1 - g_mu) K and that of Mpc^dag is
# K^dag (1 + g_mu)(s-matrix), so their product carries (1 + g_mu)(1 - g_mu) = 0.
# ----------------------------------------------------------------------------

def test_h_stencil_support(golden):
    offs = list(itertools.product(range(-4, 5), repeat=4))
    within = [o for o in offs if 0 < sum(abs(v) for v in o) <= 4]
    assert len(within) == golden["fine_stencil_neighbours"]["value"]
    even = {o for o in offs if sum(abs(v) for v in o) in (0, 2, 4)}
    assert len(even) == 225
    straight4 = {o for o in even if sorted(abs(v) for v in o) == [0, 0, 0, 4]}
    assert len(straight4) == 8
    even = even - straight4

    dims, Ls = (10, 10, 10, 10), 2
    d = DWF(dims, Ls, 1.8, 1.5, 0.5, 0.01, sy.gauge_field(dims, 0.6, 31))
    lat = d.lat
    x0 = lat.sites[1][1234]
    psi = np.zeros(d.field_shape, dtype=np.complex128)
    psi[x0 >> 1, 1, 2, 0] = 1.0
    h = d.mdagm(psi)
    nz = np.nonzero(np.abs(h).reshape(h.shape[0], -1).max(axis=1) > 1e-14)[0]
    c0 = lat.coords[x0]
    got = set()
    for cb in nz:
        dc = (lat.coords[lat.sites[1][cb]] - c0 + 5) % 10 - 5
        got.add(tuple(int(v) for v in dc))
    assert got == even


@pytest.mark.parametrize("params", [
    dict(dims=(4, 2, 2, 2), Ls=4, M5=1.8, b=1.0, c=0.0, m=0.01, apbc=False),
    dict(dims=(2, 2, 4, 2), Ls=4, M5=1.8, b=1.5, c=0.5, m=0.02, apbc=True),
])
def test_full_system_source_preparation_and_reconstruction(params):
    """The full operator's even/odd blocks against the textbook dense 5D matrix,
    and the Schur-form reduction: with b = prep_source(eta) the solution of
    H psi_o = b and psi_e = reconstruct(eta_e, psi_o) solve D psi = eta
    (numpy's dense solve of the textbook matrix)."""
    p = params
    U = sy.gauge_field(p["dims"], 0.6, 21)
    d = DWF(p["dims"], p["Ls"], p["M5"], p["b"], p["c"], p["m"], U, antiperiodic_t=p["apbc"])
    D, half = _textbook_5d_dense(p["dims"], p["Ls"], p["M5"], p["b"], p["c"], p["m"], U, p["apbc"])
    shape = d.field_shape
    psi_e = sy.gaussian_fermion(p["dims"], p["Ls"], 22)
    psi_o = sy.gaussian_fermion(p["dims"], p["Ls"], 23)
    eta_e, eta_o = d.apply_full(psi_e, psi_o)
    want = D @ np.concatenate([psi_e.ravel(), psi_o.ravel()])
    assert np.abs(np.concatenate([eta_e.ravel(), eta_o.ravel()]) - want).max() < 1e-12 * np.abs(want).max()
    eta = sy.complex_normal(24, (2 * half,))
    xs = np.linalg.solve(D, eta)
    ee, eo = eta[:half].reshape(shape), eta[half:].reshape(shape)
    b = d.prep_source(ee, eo)
    Hd = np.stack([d.mdagm(v.reshape(shape)).ravel() for v in np.eye(half)], axis=1)
    po = np.linalg.solve(Hd, b.ravel()).reshape(shape)
    pe = d.reconstruct(ee, po)
    got = np.concatenate([pe.ravel(), po.ravel()])
    assert np.abs(got - xs).max() < 1e-9 * np.abs(xs).max()
