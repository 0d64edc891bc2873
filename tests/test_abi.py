"""The C ABI library loads, exports every declared entry point, and its
structs have the layout the binding assumes.  No GPU needed."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "skr.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(skr_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def native():
    import __graft_entry__ as g
    g.build()
    from paper_2401_09516_gb300 import _native
    return _native


def test_every_declared_symbol_is_exported(native):
    lib = native.library()
    names = _declared()
    assert "skr_solve_sequence" in names and "skr_sort" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(native.exported_symbols()) <= set(names)


def test_struct_layout_matches_header(native):
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "skr.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(skr_system), sizeof(skr_options), sizeof(skr_result));
  printf("%zu %zu %zu %zu\n", offsetof(skr_system, coef), offsetof(skr_system, params),
         offsetof(skr_options, tol), offsetof(skr_options, stream));
  printf("%zu %zu\n", offsetof(skr_result, relres), offsetof(skr_result, seconds));
  printf("%zu %zu %zu %zu\n", offsetof(skr_options, warm_start), offsetof(skr_options, diagnostics),
         offsetof(skr_result, delta), offsetof(skr_options, pc_blocks));
  printf("%zu %zu %zu\n", offsetof(skr_system, rowptr), offsetof(skr_system, colind),
         offsetof(skr_options, recycle_out));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    vals = [int(v) for v in out]
    S, O, R = native.SkrSystem, native.SkrOptions, native.SkrResult
    assert vals[:3] == [ctypes.sizeof(S), ctypes.sizeof(O), ctypes.sizeof(R)]
    assert vals[3:7] == [S.coef.offset, S.params.offset, O.tol.offset, O.stream.offset]
    assert O.profile.offset == 52
    assert vals[7:9] == [R.relres.offset, R.seconds.offset]
    assert vals[9:13] == [O.warm_start.offset, O.diagnostics.offset, R.delta.offset, O.pc_blocks.offset]
    assert vals[13:16] == [S.rowptr.offset, S.colind.offset, O.recycle_out.offset]


def test_binding_constants_match_header(native):
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    defines = dict(re.findall(r"#define\s+(SKR_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", text))
    checked = 0
    for name, val in defines.items():
        if hasattr(native, name):
            assert getattr(native, name) == int(val), name
            checked += 1
    assert checked >= 20


def test_defaults_and_host_side_validation(native):
    o = native.skr_options_default()
    assert (o.m, o.k, o.maxit, o.max_refine) == (30, 10, 10000, 10)
    assert o.tol == 1e-8 and o.inner_tol == 1e-5 and o.pc_blocks == 1
    lib = native.library()
    # argument errors are reported before any device work
    assert lib.skr_sort(None, -1, 1, 0, 1, None, None) == native.SKR_ERR_INVALID_ARG
    assert "N < 0" in native.skr_last_error()
    assert lib.skr_sort(None, 0, 1, 0, 1, None, None) == native.SKR_OK
    assert lib.skr_solve_sequence(None, -2, None, None, 1, None, None, None) == native.SKR_ERR_INVALID_ARG
    assert lib.skr_sort_grouped(None, 5, 1, 0, 0, None, None, None, None) == native.SKR_ERR_INVALID_ARG
    assert "group_max" in native.skr_last_error()


def test_product_path_has_no_oracle_import():
    pkg = os.path.join(ROOT, "paper_2401_09516_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
