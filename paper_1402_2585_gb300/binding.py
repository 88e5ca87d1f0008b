"""ctypes binding of libhdcg with the C ABI's names (argument marshalling only).

Buffers may be torch tensors on the GPU (passed as device pointers) or numpy
arrays / torch CPU tensors (host pointers, for the calls that accept host
memory).  Complex data is passed as interleaved real/imaginary parts; the
binding never computes anything itself.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

F64, F32, F16, BF16, BF16T, DF64 = 0, 1, 2, 3, 4, 5
PREC_NAMES = {"f64": F64, "f32": F32, "f16": F16, "bf16": BF16, "bf16t": BF16T}
ALG_CG, ALG_ADEF2 = 0, 1
ALG_PREC, ALG_AD, ALG_DEF1, ALG_DEF2, ALG_ADEF1, ALG_BNN, ALG_BNN_DEF2START, ALG_V11, ALG_MSSDEF, ALG_ADEF2_FAMILY = \
    range(2, 12)
FAMILY = {"PREC": ALG_PREC, "AD": ALG_AD, "DEF1": ALG_DEF1, "DEF2": ALG_DEF2, "A-DEF1": ALG_ADEF1,
          "A-DEF2": ALG_ADEF2_FAMILY, "BNN": ALG_BNN, "BNN-DEF2-start": ALG_BNN_DEF2START, "V11": ALG_V11,
          "MssDef": ALG_MSSDEF}
ALG_NAMES = {"CG": ALG_CG, "A-DEF2": ALG_ADEF2, "A-DEF2 (generalised PCG)": ALG_ADEF2_FAMILY,
             **{k: v for k, v in FAMILY.items() if k != "A-DEF2"}}
SMOOTHER_MIRS, SMOOTHER_MIRSPOLY, SMOOTHER_CHEBYSHEV, SMOOTHER_NONE = 0, 1, 2, 3
SUBSPACE_INVITER, SUBSPACE_RATIONAL, SUBSPACE_CONTINUE = 0, 1, 2
_ERRORS = {1: "not converged", -1: "invalid argument", -2: "out of device memory", -3: "CUDA error",
           -4: "non-finite value", -5: "Krylov breakdown", -6: "device wait timed out", -7: "missing prerequisite"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def library_path() -> str:
    return os.path.join(_HERE, "libhdcg.so")


class HdcgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hdcg error {code} ({_ERRORS.get(code, '?')}): {msg}")
        self.code = code


class SubspaceParams(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int * 4), ("nvec", ctypes.c_int), ("prec", ctypes.c_int),
                ("inv_steps", ctypes.c_int), ("inv_shift", ctypes.c_double), ("inv_tol", ctypes.c_double),
                ("inv_maxiter", ctypes.c_int), ("seed", ctypes.c_uint64), ("level", ctypes.c_int),
                ("method", ctypes.c_int), ("filter_lambda", ctypes.c_double), ("filter_eps", ctypes.c_double),
                ("filter_order", ctypes.c_int), ("surface_depth", ctypes.c_int)]


class SolveParams(ctypes.Structure):
    _fields_ = [("algorithm", ctypes.c_int), ("outer_prec", ctypes.c_int), ("sloppy_prec", ctypes.c_int),
                ("mirs_iter", ctypes.c_int), ("mirs_shift", ctypes.c_double), ("coarse_tol", ctypes.c_double),
                ("coarse_maxiter", ctypes.c_int), ("flexible", ctypes.c_int), ("maxiter", ctypes.c_int),
                ("reliable_delta", ctypes.c_double), ("batch", ctypes.c_int), ("sloppy_codec", ctypes.c_int),
                ("smoother", ctypes.c_int), ("cheb_order", ctypes.c_int), ("cheb_lo", ctypes.c_double),
                ("cheb_hi", ctypes.c_double)]


class LdopParams(ctypes.Structure):
    _fields_ = [("nvec", ctypes.c_int), ("inv_steps", ctypes.c_int), ("shift", ctypes.c_double),
                ("tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("seed", ctypes.c_uint64)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("coarse_iterations", ctypes.c_int),
                ("coarse_iterations_max", ctypes.c_int), ("n_mdagm_outer", ctypes.c_int),
                ("n_mdagm_sloppy", ctypes.c_int), ("n_mdagm_f64", ctypes.c_int),
                ("reliable_updates", ctypes.c_int), ("status", ctypes.c_int),
                ("true_residual", ctypes.c_double), ("seconds", ctypes.c_double), ("batch_rhs", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SIGS = {
    "hdcg_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(_I), _I, _I, _P]),
    "hdcg_set_dwf": (_I, [_P, _D, _D, _D, _D]),
    "hdcg_set_gauge": (_I, [_P, _P, _I]),
    "hdcg_apply_mpc": (_I, [_P, _P, _P, _I, _I]),
    "hdcg_apply_mdagm": (_I, [_P, _P, _P, _I, ctypes.POINTER(_D)]),
    "hdcg_prep_source": (_I, [_P, _P, _P, _P, _I]),
    "hdcg_reconstruct": (_I, [_P, _P, _P, _P, _I]),
    "hdcg_build_subspace": (_I, [_P, ctypes.POINTER(SubspaceParams)]),
    "hdcg_set_subspace": (_I, [_P, _I, ctypes.POINTER(_I), _I, _I, _P, _I, _I]),
    "hdcg_promote_subspace": (_I, [_P, _P, _I]),
    "hdcg_time_coarse_apply": (_I, [_P, _I, _I, ctypes.POINTER(ctypes.c_double)]),
    "hdcg_set_coarse_tc_shape": (_I, [_P, _I]),
    "hdcg_get_subspace": (_I, [_P, _I, _P]),
    "hdcg_build_coarse": (_I, [_P, _I, _I]),
    "hdcg_get_coarse": (_I, [_P, _I, _P]),
    "hdcg_restrict_coarse": (_I, [_P, _P, _P, _I]),
    "hdcg_prolong_coarse": (_I, [_P, _P, _P, _I]),
    "hdcg_set_coarse": (_I, [_P, _P, _I, _I]),
    "hdcg_restrict": (_I, [_P, _P, _I, _P]),
    "hdcg_prolong": (_I, [_P, _P, _P, _I]),
    "hdcg_coarse_apply": (_I, [_P, _P, _P]),
    "hdcg_coarse_apply_noalloc": (_I, [_P, _P, _P]),
    "hdcg_coarse_apply_multi": (_I, [_P, _P, _P, _I]),
    "hdcg_coarse_solve": (_I, [_P, _P, _P, _I, _D, _I, ctypes.POINTER(_I)]),
    "hdcg_build_coarse_deflation": (_I, [_P, ctypes.POINTER(LdopParams)]),
    "hdcg_set_coarse_preconditioner": (_I, [_P, _I, _D, _D, _D, ctypes.POINTER(_D)]),
    "hdcg_coarse_precondition": (_I, [_P, _P, _P, _I]),
    "hdcg_get_coarse_deflation": (_I, [_P, ctypes.POINTER(_D), _P]),
    "hdcg_dense_heev": (_I, [_I, _P, _P, _P]),
    "hdcg_default_params": (None, [ctypes.POINTER(SolveParams)]),
    "hdcg_solve": (_I, [_P, _P, _P, _I, _D, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveStats), _I]),
    "hdcg_set_profiling": (_I, [_P, _I]),
    "hdcg_get_hop_profile": (_I, [_P, _I, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_D),
                                  ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "hdcg_get_phase_profile": (_I, [_P, ctypes.POINTER(_D)]),
    "hdcg_launch_count": (ctypes.c_longlong, [_P]),
    "hdcg_set_hop_variant": (_I, [_P, _I]),
    "hdcg_encode_i8": (_I, [_P, _P, _P, _P, _I]),
    "hdcg_decode_i8": (_I, [_P, _P, _P, _P, _I]),
    "hdcg_last_error": (ctypes.c_char_p, [_P]),
    "hdcg_destroy": (None, [_P]),
    "hdcg_version": (_I, []),
}


def lib():
    """Load libhdcg.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                               "(paper_1402_2585_gb300/build.py); there is no CPU fallback")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _ptr(x):
    """Raw pointer of a torch tensor or numpy array (contiguous)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError(f"unsupported buffer type {type(x)}")


def _on_device(x) -> int:
    return int(bool(getattr(x, "is_cuda", False)))


def dense_heev(H, vectors=True):
    """hdcg_dense_heev: eigenvalues (and eigenvectors) of a Hermitian complex matrix, on the host."""
    H = np.ascontiguousarray(H, dtype=np.complex128)
    n = H.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n), dtype=np.complex128) if vectors else None
    rc = lib().hdcg_dense_heev(n, ctypes.c_void_p(H.ctypes.data), ctypes.c_void_p(w.ctypes.data),
                               None if V is None else ctypes.c_void_p(V.ctypes.data))
    if rc != 0:
        raise HdcgError(rc, "hdcg_dense_heev failed")
    return (w, V) if vectors else w


class Hdcg:
    """One handle of the C library; methods mirror the hdcg_* calls."""

    def __init__(self, dims, Ls, antiperiodic_t=False, stream=None):
        self._L = lib()
        h = ctypes.c_void_p()
        d = (ctypes.c_int * 4)(*[int(v) for v in dims])
        st = ctypes.c_void_p(int(stream)) if stream is not None else None
        rc = self._L.hdcg_create(ctypes.byref(h), d, int(Ls), int(bool(antiperiodic_t)), st)
        if rc != 0:
            raise HdcgError(rc, "hdcg_create failed")
        self.h = h
        self.dims = tuple(int(v) for v in dims)
        self.Ls = int(Ls)

    # -- helpers ------------------------------------------------------------
    def _check(self, rc, allow_not_converged=False):
        if rc == 0 or (allow_not_converged and rc == 1):
            return rc
        raise HdcgError(rc, self._L.hdcg_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self._L.hdcg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- operator -----------------------------------------------------------
    def set_dwf(self, M5, b, c, mass):
        return self._check(self._L.hdcg_set_dwf(self.h, M5, b, c, mass))

    def set_gauge(self, U):
        return self._check(self._L.hdcg_set_gauge(self.h, _ptr(U), _on_device(U)))

    def apply_mpc(self, inp, out, dagger=False, prec=F32):
        return self._check(self._L.hdcg_apply_mpc(self.h, _ptr(inp), _ptr(out), int(bool(dagger)), prec))

    def apply_mdagm(self, inp, out, prec=F32, want_pHp=False):
        v = ctypes.c_double(0.0)
        self._check(self._L.hdcg_apply_mdagm(self.h, _ptr(inp), _ptr(out), prec,
                                             ctypes.byref(v) if want_pHp else None))
        return v.value if want_pHp else None

    def prep_source(self, eta_e, eta_o, b):
        return self._check(self._L.hdcg_prep_source(self.h, _ptr(eta_e), _ptr(eta_o), _ptr(b), _on_device(b)))

    def reconstruct(self, eta_e, psi_o, psi_e):
        return self._check(self._L.hdcg_reconstruct(self.h, _ptr(eta_e), _ptr(psi_o), _ptr(psi_e),
                                                     _on_device(psi_e)))

    # -- subspace and coarse operator -----------------------------------------
    def build_subspace(self, block, nvec, prec=F32, inv_steps=3, inv_shift=0.0, inv_tol=1e-4,
                       inv_maxiter=20000, seed=0, level=1, method=SUBSPACE_INVITER, filter_lambda=0.0,
                       filter_eps=0.0, filter_order=4, surface_depth=0):
        p = SubspaceParams((ctypes.c_int * 4)(*block), nvec, prec, inv_steps, inv_shift, inv_tol,
                           inv_maxiter, seed, int(level), int(method), float(filter_lambda), float(filter_eps),
                           int(filter_order), int(surface_depth))
        return self._check(self._L.hdcg_build_subspace(self.h, ctypes.byref(p)))

    def promote_subspace(self, src, prec=F32):
        """This handle's subspace := src's (fifth extent Ls1 <= Ls) promoted to Ls."""
        return self._check(self._L.hdcg_promote_subspace(self.h, src.h, int(prec)))

    def set_subspace(self, block, phi, prec=F32, already_orthonormal=False, level=1):
        nvec = int(phi.shape[0])
        return self._check(self._L.hdcg_set_subspace(self.h, int(level), (ctypes.c_int * 4)(*block), nvec, prec,
                                                     _ptr(phi), _on_device(phi), int(bool(already_orthonormal))))

    def get_subspace(self, out, level=1):
        return self._check(self._L.hdcg_get_subspace(self.h, int(level), _ptr(out)))

    def build_coarse(self, prec=F32, level=1):
        return self._check(self._L.hdcg_build_coarse(self.h, int(level), prec))

    def set_coarse(self, A, prec=F32):
        return self._check(self._L.hdcg_set_coarse(self.h, _ptr(A), int(prec), _on_device(A)))

    def get_coarse(self, out, level=1):
        return self._check(self._L.hdcg_get_coarse(self.h, int(level), _ptr(out)))

    def restrict_coarse(self, x, c2, nrhs=1):
        return self._check(self._L.hdcg_restrict_coarse(self.h, _ptr(x), _ptr(c2), int(nrhs)))

    def prolong_coarse(self, c2, x, nrhs=1):
        return self._check(self._L.hdcg_prolong_coarse(self.h, _ptr(c2), _ptr(x), int(nrhs)))

    def restrict(self, v, prec, c_out):
        return self._check(self._L.hdcg_restrict(self.h, _ptr(v), prec, _ptr(c_out)))

    def prolong(self, c_in, v_out, prec):
        return self._check(self._L.hdcg_prolong(self.h, _ptr(c_in), _ptr(v_out), prec))

    def coarse_apply(self, x, y):
        return self._check(self._L.hdcg_coarse_apply(self.h, _ptr(x), _ptr(y)))

    def set_coarse_tc_shape(self, ctas_per_sm):
        """0: autotune the tensor-core stencil's persistent shape; 1 or 2: force it."""
        return self._check(self._L.hdcg_set_coarse_tc_shape(self.h, int(ctas_per_sm)))

    def time_coarse_apply(self, nrhs, reps=20):
        """Mean device microseconds of one tensor-core stencil apply to nrhs vectors."""
        us = ctypes.c_double(0.0)
        self._check(self._L.hdcg_time_coarse_apply(self.h, int(nrhs), int(reps), ctypes.byref(us)))
        return us.value

    def coarse_apply_multi(self, x, y, nrhs):
        return self._check(self._L.hdcg_coarse_apply_multi(self.h, _ptr(x), _ptr(y), int(nrhs)))

    def coarse_solve(self, b, x, nrhs, tol, maxiter=100000):
        it = ctypes.c_int(0)
        self._check(self._L.hdcg_coarse_solve(self.h, _ptr(b), _ptr(x), int(nrhs), float(tol), int(maxiter),
                                               ctypes.byref(it)))
        return it.value

    def set_coarse_preconditioner(self, order, lo=0.0, hi=0.0, shift=0.0):
        """Chebyshev preconditioner of Q_trunc; returns the interval (lo, hi) used."""
        iv = (ctypes.c_double * 2)()
        self._check(self._L.hdcg_set_coarse_preconditioner(self.h, int(order), float(lo), float(hi), float(shift), iv))
        return iv[0], iv[1]

    def coarse_precondition(self, x, y, nrhs=1):
        return self._check(self._L.hdcg_coarse_precondition(self.h, _ptr(x), _ptr(y), int(nrhs)))

    def build_coarse_deflation(self, nvec, inv_steps=3, shift=0.0, tol=1e-7, maxiter=100000, seed=0):
        p = LdopParams(int(nvec), int(inv_steps), float(shift), float(tol), int(maxiter), int(seed))
        return self._check(self._L.hdcg_build_coarse_deflation(self.h, ctypes.byref(p)))

    def get_coarse_deflation(self, nvec, vectors=False, shape=None):
        """Ritz values (nvec,) and, with vectors=True, Z as complex128 of `shape`."""
        lam = np.zeros(nvec)
        Z = np.zeros(shape, dtype=np.complex128) if vectors else None
        self._check(self._L.hdcg_get_coarse_deflation(
            self.h, lam.ctypes.data_as(ctypes.POINTER(_D)), None if Z is None else ctypes.c_void_p(Z.ctypes.data)))
        return (lam, Z) if vectors else lam

    def coarse_apply_noalloc(self, x, y):
        return self._check(self._L.hdcg_coarse_apply_noalloc(self.h, _ptr(x), _ptr(y)))

    # -- solve ----------------------------------------------------------------
    @staticmethod
    def default_params(**kw) -> SolveParams:
        p = SolveParams()
        lib().hdcg_default_params(ctypes.byref(p))
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    def solve(self, b, x, tol, params: SolveParams | None = None, nrhs=1):
        st = SolveStats()
        p = params if params is not None else self.default_params()
        rc = self._L.hdcg_solve(self.h, _ptr(b), _ptr(x), nrhs, tol, ctypes.byref(p), ctypes.byref(st),
                                _on_device(b))
        self._check(rc, allow_not_converged=True)
        return st

    # -- instrumentation ------------------------------------------------------
    def set_profiling(self, on):
        return self._check(self._L.hdcg_set_profiling(self.h, int(bool(on))))

    def get_hop_profile(self, prec, operator_bytes=False):
        n = ctypes.c_longlong()
        ms = ctypes.c_double()
        by = ctypes.c_double()
        ob = ctypes.c_double()
        self._check(self._L.hdcg_get_hop_profile(self.h, prec, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by),
                                                 ctypes.byref(ob)))
        return (n.value, ms.value, by.value, ob.value) if operator_bytes else (n.value, ms.value, by.value)

    PHASES = ("h_outer", "h_sloppy", "h_f64", "coarse_cg", "restrict_prolong", "total")

    def get_phase_profile(self):
        ms = (ctypes.c_double * 6)()
        self._check(self._L.hdcg_get_phase_profile(self.h, ms))
        return dict(zip(self.PHASES, list(ms)))

    def encode_i8(self, x, scale, q, nfields=1):
        return self._check(self._L.hdcg_encode_i8(self.h, _ptr(x), _ptr(scale), _ptr(q), int(nfields)))

    def decode_i8(self, scale, q, x, nfields=1):
        return self._check(self._L.hdcg_decode_i8(self.h, _ptr(scale), _ptr(q), _ptr(x), int(nfields)))

    def set_hop_variant(self, variant):
        return self._check(self._L.hdcg_set_hop_variant(self.h, int(variant)))

    def launch_count(self):
        return int(self._L.hdcg_launch_count(self.h))
