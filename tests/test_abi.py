"""The C-ABI library loads and exports every function include/hdcg.h declares (no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hdcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hdcg_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["hdcg_create", "hdcg_set_dwf", "hdcg_set_gauge", "hdcg_apply_mpc", "hdcg_apply_mdagm",
              "hdcg_build_subspace", "hdcg_set_subspace", "hdcg_build_coarse", "hdcg_get_coarse",
              "hdcg_restrict", "hdcg_prolong", "hdcg_coarse_apply", "hdcg_solve", "hdcg_last_error",
              "hdcg_destroy", "hdcg_prep_source", "hdcg_reconstruct", "hdcg_restrict_coarse",
              "hdcg_prolong_coarse", "hdcg_promote_subspace", "hdcg_coarse_precondition",
              "hdcg_set_coarse_preconditioner", "hdcg_encode_i8", "hdcg_decode_i8"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g
    g.build()
    from paper_1402_2585_gb300 import library_path
    L = ctypes.CDLL(library_path())
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    assert L.hdcg_version() == 1


def test_create_rejects_bad_sizes_without_gpu_work():
    """Argument checks happen before any device call."""
    from paper_1402_2585_gb300 import lib
    L = lib()
    h = ctypes.c_void_p()
    for dims, Ls in [((4, 4, 4, 3), 4), ((4, 4, 4, 4), 12), ((4, 4, 4, 4), 1), ((0, 4, 4, 4), 4),
                     ((4, 4, 4, 4), 64)]:
        d = (ctypes.c_int * 4)(*dims)
        assert L.hdcg_create(ctypes.byref(h), d, Ls, 0, None) == -1
