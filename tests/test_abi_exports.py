"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads,
and exports every entry point declared in include/*.h.  Only host-side
functions are called (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(gsyeig_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1111_6374_gb300 import load

    return load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("gsyeig_create", "gsyeig_solve", "gsyeig_destroy", "gsyeig_potrf", "gsyeig_sygst", "gsyeig_symv",
                 "gsyeig_trsm_back", "gsyeig_syev_lanczos", "gsyeig_tridiag_eig"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points(lib):
    from paper_1111_6374_gb300 import Opts

    o = Opts()
    assert lib.gsyeig_default_options(ctypes.byref(o)) == 0
    assert o.tol == 1e-12 and o.max_restarts == 2000 and o.krylov_dim == 0 and o.block == 0
    assert lib.gsyeig_default_options(None) == -1
    assert b"positive definite" in lib.gsyeig_strerror(1)
    assert lib.gsyeig_strerror(-3) == b"invalid argument"
    # NULL handle is rejected before any CUDA call
    assert lib.gsyeig_set_options(None, ctypes.byref(o)) == -1
    assert lib.gsyeig_solve(None, None, 1, None, 1, 4, 1, 0, None, None, 4, None) == -1
    assert lib.gsyeig_destroy(None) == -1
    assert lib.gsyeig_kernel_launches() >= 0


def test_library_is_built_for_sm_103a():
    from paper_1111_6374_gb300.build import ARCH, LIB

    assert "arch=compute_103a,code=sm_103a" in ARCH
    assert os.path.exists(LIB)


def test_colmajor_helpers_cpu():
    import torch

    from paper_1111_6374_gb300 import colmajor, colmajor_empty

    X = colmajor_empty(5, 3, device="cpu")
    assert X.shape == (5, 3) and X.stride() == (1, 5)
    T = torch.arange(12, dtype=torch.float64).reshape(4, 3)
    C = colmajor(T)
    assert C.stride(0) == 1 and torch.equal(C, T)


@pytest.mark.parametrize("struct", ["gsyeig_opts", "gsyeig_info"])
def test_binding_structs_match_the_header_layout(struct, tmp_path):
    """The ctypes mirrors of gsyeig_opts / gsyeig_info have the header's
    size and field offsets (compiled with the host C compiler)."""
    import shutil
    import subprocess

    from paper_1111_6374_gb300 import Info, Opts

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    py = {"gsyeig_opts": Opts, "gsyeig_info": Info}[struct]
    fields = [f for f, _ in py._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gsyeig.h"\nint main(void) {\n'
                   f'  printf("size %zu\\n", sizeof({struct}));\n'
                   + "".join(f'  printf("{f} %zu\\n", offsetof({struct}, {f}));\n' for f in fields)
                   + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    assert int(got["size"]) == ctypes.sizeof(py)
    for f in fields:
        assert int(got[f]) == getattr(py, f).offset, f
