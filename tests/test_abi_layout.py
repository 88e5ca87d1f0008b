"""The ctypes binding's view of the C ABI agrees with include/hdcg.h: the size
of every parameter and statistics struct and the offset of each of its
fields, as a C program compiled against the header with the host compiler
prints them, and the precision, algorithm and status codes.  No GPU.
"""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_1402_2585_gb300 import binding as bd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hdcg.h")
WORK = os.path.join(ROOT, "paper_1402_2585_gb300", "_build")
STRUCTS = {"hdcg_subspace_params": bd.SubspaceParams, "hdcg_ldop_params": bd.LdopParams,
           "hdcg_params": bd.SolveParams, "hdcg_stats": bd.SolveStats}


def _header_macros(prefix):
    src = open(HEADER).read()
    return sorted(set(re.findall(r"#define\s+(" + prefix + r"\w*)\s", src)))


def _binding_codes():
    codes = {"HDCG_" + n: getattr(bd, n) for n in ("F64", "F32", "F16", "BF16", "BF16T", "DF64")}
    for n in dir(bd):
        if re.fullmatch(r"(ALG|SMOOTHER|SUBSPACE)_[A-Z0-9_]+", n) and n != "ALG_NAMES":
            codes["HDCG_" + n] = getattr(bd, n)
    return codes


@pytest.fixture(scope="module")
def c_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    macros = sorted(set(_binding_codes()) | set(_header_macros("HDCG_ALG_")) | set(_header_macros("HDCG_ERR_"))
                    | {"HDCG_OK", "HDCG_NOT_CONVERGED"})
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "hdcg.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'  printf("{cname} . %zu\\n", sizeof({cname}));')
        for name, _ in cls._fields_:
            lines.append(f'  printf("{cname} {name} %zu\\n", offsetof({cname}, {name}));')
    for m in macros:
        lines.append(f'#ifdef {m}\n  printf("macro {m} %d\\n", (int)({m}));\n#endif')
    lines.append("  return 0;\n}")
    os.makedirs(WORK, exist_ok=True)
    src = os.path.join(WORK, "abi_layout.c")
    exe = os.path.join(WORK, "abi_layout")
    with open(src, "w") as f:
        f.write("\n".join(lines) + "\n")
    r = subprocess.run([cc, "-std=c99", "-I", os.path.dirname(HEADER), src, "-o", exe], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    layout, values = {}, {}
    for line in out.splitlines():
        a, b, v = line.split()
        if a == "macro":
            values[b] = int(v)
        else:
            layout[(a, b)] = int(v)
    return layout, values


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_struct_layout(c_layout, cname):
    layout, _ = c_layout
    cls = STRUCTS[cname]
    assert ctypes.sizeof(cls) == layout[(cname, ".")], cname
    for name, _ in cls._fields_:
        assert getattr(cls, name).offset == layout[(cname, name)], (cname, name)


def test_codes(c_layout):
    _, values = c_layout
    for macro, v in _binding_codes().items():
        assert values.get(macro) == v, macro
    # every algorithm the header defines has a binding constant and a name
    algs = _header_macros("HDCG_ALG_")
    assert set(algs) == {m for m in _binding_codes() if m.startswith("HDCG_ALG_")}
    names = getattr(bd, "ALG_NAMES", {"CG": bd.ALG_CG, "A-DEF2": bd.ALG_ADEF2})
    assert sorted(names.values()) == sorted(values[m] for m in algs)
    # the status codes the binding names are the header's
    status = {values[m] for m in _header_macros("HDCG_ERR_")} | {values["HDCG_NOT_CONVERGED"]}
    assert set(bd._ERRORS) == status
    assert values["HDCG_OK"] == 0
