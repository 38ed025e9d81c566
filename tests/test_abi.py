"""The C-ABI library builds, loads without a GPU, and exports every function
include/ftcj.h declares.  No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "ftcj.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(ftcj_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2509_16460_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["ftcj_plan_create", "ftcj_jbuild", "ftcj_jbuild_host", "ftcj_rho", "ftcj_potential",
              "ftcj_jback", "ftcj_fold_density", "ftcj_unfold_j", "ftcj_plan_destroy", "ftcj_strerror",
              "ftcj_last_error"]:
        assert n in names


def test_every_declared_symbol_is_exported(built_lib):
    missing = [n for n in declared_functions() if not hasattr(built_lib, n)]
    assert not missing, missing


def test_binding_lists_every_symbol():
    from paper_2509_16460_gb300 import ftcj
    assert sorted(ftcj.EXPORTED) == declared_functions()


def test_strerror_without_gpu(built_lib):
    from paper_2509_16460_gb300 import ftcj
    L = ftcj.lib()
    assert L.ftcj_strerror(0).decode() == "ok"
    assert L.ftcj_strerror(-5).decode() == "unsupported input"


def test_struct_sizes_match_header():
    """ctypes mirrors of the ABI structs have the C layout (checked by a tiny
    host-only C program compiled against include/ftcj.h)."""
    import subprocess
    import tempfile
    from paper_2509_16460_gb300 import ftcj
    code = r"""
#include <stdio.h>
#include <stddef.h>
#include "ftcj.h"
int main(void){
 printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(ftcj_cell), sizeof(ftcj_shell), sizeof(ftcj_basis),
        sizeof(ftcj_params), sizeof(ftcj_info), offsetof(ftcj_info, pairs_by_class), offsetof(ftcj_info, gcut));
 return 0;}
"""
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "s.c")
        exe = os.path.join(d, "s")
        with open(src, "w") as f:
            f.write(code)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    sizes = [int(x) for x in out]
    assert sizes[0] == ctypes.sizeof(ftcj.Cell)
    assert sizes[1] == ctypes.sizeof(ftcj.ShellDesc)
    assert sizes[2] == ctypes.sizeof(ftcj.BasisDesc)
    assert sizes[3] == ctypes.sizeof(ftcj.Params)
    assert sizes[4] == ctypes.sizeof(ftcj.Info)
    assert sizes[5] == ftcj.Info.pairs_by_class.offset
    assert sizes[6] == ftcj.Info.gcut.offset


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2509_16460_gb300 import ftcj
    monkeypatch.setattr(ftcj, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(ftcj, "_lib", None)
    with pytest.raises(ftcj.FtcjError):
        ftcj.lib()
