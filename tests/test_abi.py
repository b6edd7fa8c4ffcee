"""Host-side checks of the C ABI library: it builds, loads and exports every entry
point include/krr.h declares, and the binding's struct layouts match the header.
No compute calls (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "krr.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(krr_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1905_10587_gb300 import build
    from paper_1905_10587_gb300 import _lib
    build()
    return _lib.load()


def test_header_declares_the_path():
    names = _declared()
    for must in ("krr_build_precond", "krr_solve", "krr_predict", "krr_kmvm", "krr_sketch",
                 "krr_qrcp", "krr_precond_apply", "krr_residual_hp", "krr_omega"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_declares_every_header_symbol():
    from paper_1905_10587_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == _declared()


def test_struct_layouts_match_header():
    from paper_1905_10587_gb300 import _lib
    assert C.sizeof(_lib.KrrOpts) == 4 * 4 + 8 * 2 + 4 * 2 + 8 + 4 * 4 + 4 * 8 + 8
    assert _lib.KrrSolveInfo.cond_estimate.offset == 288
    assert _lib.KrrOpts.inner_tol.offset == 16
    assert C.sizeof(_lib.KrrSolveInfo) == 16 + 8 * 16 + 16 + 4 + 4 * 8 + 4 + 8 * 8 + 4 * 7 + 4
    assert _lib.KrrSolveInfo.build_ms.offset == 16 + 8 * 16


def test_c_struct_layout_matches_binding(tmp_path):
    # compile the header with the host C compiler and compare sizes/offsets with ctypes
    import shutil
    import subprocess
    from paper_1905_10587_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "krr.h"\n'
        'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(krr_opts), '
        'offsetof(krr_opts, inner_tol), offsetof(krr_opts, residual), sizeof(krr_solve_info), '
        'offsetof(krr_solve_info, sweep_residual), offsetof(krr_solve_info, mvm_count), '
        'offsetof(krr_opts, recurrence) + 1000 * offsetof(krr_solve_info, cond_estimate));return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [C.sizeof(_lib.KrrOpts), _lib.KrrOpts.inner_tol.offset, _lib.KrrOpts.residual.offset,
            C.sizeof(_lib.KrrSolveInfo), _lib.KrrSolveInfo.sweep_residual.offset,
            _lib.KrrSolveInfo.mvm_count.offset,
            _lib.KrrOpts.recurrence.offset + 1000 * _lib.KrrSolveInfo.cond_estimate.offset]
    assert got == want


def test_default_opts_without_gpu(lib):
    from paper_1905_10587_gb300 import _lib
    o = _lib.KrrOpts()
    assert lib.krr_default_opts(C.byref(o)) == 0
    assert o.oversample == 5 and o.max_iter > 0 and 0 < o.inner_tol < 1
    assert lib.krr_default_opts(None) == 1
    assert lib.krr_last_error(None) == b"null context"
