"""The C-ABI library builds, loads and exports every symbol include/hz.h
declares; struct layouts agree between the header and the binding; the
host-side descriptor logic (no GPU compute) behaves as documented."""

import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2308_06152_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hz.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(hz_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists(_lib.LIB_PATH):
        pytest.skip("no nvcc to build libhz.so")
    path = build.build()
    return _lib.load_library(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("hz_workspace_bytes", "hz_setup", "hz_solve", "hz_solve_host",
                 "hz_apply", "hz_gradient", "hz_destroy", "hz_status_str"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


STRUCTS = [(_lib.HzDesc, "hz_desc"), (_lib.HzSolveInfo, "hz_solve_info"),
           (_lib.HzTuning, "hz_tuning")]


def test_struct_layout_matches_header(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hz.h"',
             "int main(void){"]
    for cls, cname in STRUCTS:
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        lines += [f'printf("%zu\\n", offsetof({cname}, {f}));'
                  for f, _ in cls._fields_]
    lines += ["return 0;}"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True,
                                          text=True).stdout.split()]
    k = 0
    for cls, cname in STRUCTS:
        assert out[k] == ctypes.sizeof(cls), cname
        k += 1
        for f, _ in cls._fields_:
            assert out[k] == getattr(cls, f).offset, (cname, f)
            k += 1


def _ws(lib, **kw):
    d = _lib.HzDesc()
    lib.hz_desc_default(ctypes.byref(d), kw.pop("nx", 33), kw.pop("ny", 33),
                        kw.pop("h", 1 / 32))
    for k, v in kw.items():
        setattr(d, k, v)
    n = ctypes.c_size_t(0)
    st = lib.hz_workspace_bytes(ctypes.byref(d), ctypes.byref(n))
    return st, n.value


def test_desc_defaults_are_the_papers(lib):
    d = _lib.HzDesc()
    lib.hz_desc_default(ctypes.byref(d), 81, 81, 1 / 80)
    assert (d.beta1, d.beta2, d.jacobi_omega) == (1.0, -0.5, 0.8)
    assert d.min_coarse_intervals == 2 and d.coarse_tol == 1e-6


def test_workspace_bytes_host_logic(lib):
    st, b1 = _ws(lib)
    assert st == 0 and b1 > 0
    st, b4 = _ws(lib, nrhs_max=4)
    assert st == 0 and b4 > 3 * b1 // 2
    assert _ws(lib, nx=2)[0] == 1                       # too small
    assert _ws(lib, nrhs_max=0)[0] == 1
    assert _ws(lib, bc=7)[0] == 1
    assert _ws(lib, nx=34, ny=34)[0] == 2                # cannot coarsen
    assert _ws(lib, nx=20, ny=20, zkind=0)[0] == 0       # plain CSLP is fine
    assert _ws(lib, nx=34, ny=34, zkind=0)[0] == 2       # 1156-node coarsest
    assert _ws(lib, nx=2301, ny=751, h=4.0)[0] == 2      # coarsest too large
    assert _ws(lib, nx=2305, ny=769, h=4.0)[0] == 0


def test_workspace_bytes_checks_method_choices(lib):
    """The coarse operator, outer iteration and preconditioner fields are
    validated on the host; TLKM needs deflation vectors, and each optional
    buffer only costs workspace when its choice is made."""
    _, base = _ws(lib)
    for ek in range(8):
        assert _ws(lib, ekind=ek)[0] == 0, ek
    assert _ws(lib, ekind=8)[0] == 1
    assert _ws(lib, outer_solver=1)[0] == 0
    assert _ws(lib, outer_solver=2)[0] == 1
    assert _ws(lib, preconditioner=1)[0] == 0
    assert _ws(lib, preconditioner=2)[0] == 1
    assert _ws(lib, preconditioner=1, zkind=0)[0] == 1
    assert _ws(lib, deflation_levels=2)[0] == 0
    assert _ws(lib, deflation_levels=2)[1] > base
    assert _ws(lib, deflation_levels=2, zkind=0)[0] == 1
    assert _ws(lib, deflation_levels=2, preconditioner=1)[0] == 1
    # multilevel deflation down to level D needs D coarsenings (33: 4)
    assert _ws(lib, deflation_levels=3)[0] == 0
    assert _ws(lib, deflation_levels=4)[1] > _ws(lib, deflation_levels=3)[1]
    assert _ws(lib, deflation_levels=5)[0] == 2
    assert _ws(lib, deflation_levels=24)[0] == 1
    assert _ws(lib, nx=5, ny=5, deflation_levels=2)[0] == 2   # one coarsening
    # the printed deflation scaling: two levels only, no extra workspace
    assert _ws(lib, deflation_scaling=1, ekind=3) == (0, _ws(lib, ekind=3)[1])
    assert _ws(lib, deflation_scaling=1, deflation_levels=2)[0] == 1
    assert _ws(lib, deflation_scaling=2)[0] == 1
    # FGMRES restart: 0 .. outer_maxit, not with GCR; no extra workspace
    assert _ws(lib, restart=5) == (0, base)
    assert _ws(lib, restart=-1)[0] == 1
    assert _ws(lib, restart=101)[0] == 1
    assert _ws(lib, restart=5, outer_solver=1)[0] == 1
    # GCR keeps a residual vector; TLKM a fine-grid scratch vector;
    # the stored Galerkin stencil is only planned for the Galerkin E
    assert _ws(lib, outer_solver=1)[1] > base
    assert _ws(lib, preconditioner=1)[1] > base
    assert _ws(lib, ekind=1)[1] < base


def test_tuning_defaults(lib):
    t = _lib.HzTuning()
    lib.hz_tuning_default(ctypes.byref(t))
    assert [getattr(t, f) for f, _ in t._fields_] == [0] * len(t._fields_)
    assert lib.hz_set_tuning(None, ctypes.byref(t)) == 1
    assert lib.hz_get_tuning(None, ctypes.byref(t)) == 1


def test_status_strings(lib):
    for code in range(9):
        assert lib.hz_status_str(code)
    assert lib.hz_status_str(0) == b"ok"
