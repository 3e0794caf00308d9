"""The C-ABI library loads and exports every entry point declared in
include/pdst.h (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pdst.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pdst_[A-Za-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_11920_b300 import build, pdst
    build.build()
    return pdst.load()


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("pdst_build_G", "pdst_lsqr", "pdst_destroy", "pdst_G_export_csr",
                     "pdst_apply_G", "pdst_set_col_scaling", "pdst_last_error_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_signatures_cover_header(lib):
    from paper_2604_11920_b300 import pdst
    assert set(declared_functions()) <= set(pdst.SIGNATURES)


def test_struct_layouts_match_header(lib, tmp_path):
    """The ctypes structures have the sizes and offsets the C compiler gives
    the header's structs."""
    import subprocess
    from paper_2604_11920_b300 import pdst
    structs = {"pdst_grid": pdst.Grid, "pdst_build_opts": pdst.BuildOpts,
               "pdst_lsqr_opts": pdst.LsqrOpts, "pdst_lsqr_info": pdst.LsqrInfo,
               "pdst_batched_opts": pdst.BatchedOpts, "pdst_outer_opts": pdst.OuterOpts,
               "pdst_outer_info": pdst.OuterInfo}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pdst.h"', "int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)]).decode().splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, f"{cname}.{f}"


def test_version_and_error_string_without_gpu(lib):
    assert lib.pdst_version() >= 10000
    assert isinstance(lib.pdst_last_error_string(), bytes)


def test_null_arguments_rejected_on_host(lib):
    from paper_2604_11920_b300 import pdst
    out = ctypes.c_void_p()
    st = lib.pdst_build_G(None, 0, None, None, 1, None, None, None, ctypes.byref(out))
    assert st == 1 and b"grid" in lib.pdst_last_error_string()
    st = lib.pdst_lsqr(None, None, 1.0, 0.1, 10, 1e-6, None, None, None, None)
    assert st == 1
    g = pdst.Grid(4, 4, 2, 1.0, 2.0)
    st = lib.pdst_build_G(ctypes.byref(g), 0, None, None, 0, None, None, None, ctypes.byref(out))
    assert st == 1 and b"n_periods" in lib.pdst_last_error_string()
