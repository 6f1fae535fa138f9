"""The C ABI library (CPU side): it builds, loads, exports every entry point
declared in include/gbcg.h, and rejects malformed input before any GPU work."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1010_4639_gb300 as gb
from paper_1010_4639_gb300 import _lib

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gbcg.h")


def declared_symbols():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(gbcg_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    gb.build()
    return _lib.load()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("gbcg_create", "gbcg_spmv", "gbcg_solve", "gbcg_destroy", "gbcg_status_string", "gbcg_last_error"):
        assert name in syms
    assert sorted(_lib.EXPORTS) == syms


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code, name in enumerate(_lib.STATUS_NAMES):
        assert lib.gbcg_status_string(code).decode() == ("GBCG_OK" if code == 0 else "GBCG_ERR_" + name)
    assert lib.gbcg_status_string(99).decode() == "GBCG_UNKNOWN_STATUS"


def _create(lib, fmt, ptr, idx, val, base=0, n=None, nnz=None):
    ptr = np.asarray(ptr, np.int32)
    idx = np.asarray(idx, np.int32)
    val = np.asarray(val, np.float64)
    h = ctypes.c_void_p()
    n = len(ptr) - 1 if n is None else n
    nnz = len(idx) if nnz is None else nnz
    rc = lib.gbcg_create(ctypes.byref(h), fmt, n, nnz, ptr.ctypes.data_as(ctypes.c_void_p),
                         idx.ctypes.data_as(ctypes.c_void_p), val.ctypes.data_as(ctypes.c_void_p), base,
                         _lib.GBCG_HOST, None)
    return rc, lib.gbcg_last_error().decode()


@pytest.mark.parametrize("case", [
    ("unsorted columns", 0, [0, 2, 2], [1, 0], [1.0, 2.0], 0, "strictly increasing"),
    ("duplicate column", 0, [0, 2, 2], [0, 0], [1.0, 2.0], 0, "strictly increasing"),
    ("column out of range", 0, [0, 1], [5], [1.0], 0, "out of range"),
    ("negative column", 0, [0, 1], [-1], [1.0], 0, "out of range"),
    ("lower entry in upper storage", 1, [0, 1, 2], [0, 0], [1.0, 2.0], 0, "below the diagonal"),
    ("nan value", 0, [0, 1], [0], [float("nan")], 0, "non-finite"),
    ("decreasing ptr", 0, [0, 2, 1], [0, 1], [1.0, 1.0], 0, "ptr"),
    ("bad base", 0, [0, 1], [0], [1.0], 2, "index_base"),
    ("ptr[0] != base", 0, [1, 2], [0], [1.0], 0, "ptr[0]"),
    ("one-based index 0", 0, [1, 2], [0], [1.0], 1, "out of range"),
    ("bad format", 7, [0, 1], [0], [1.0], 0, "format"),
])
def test_create_rejects_malformed_input(lib, case):
    _, fmt, ptr, idx, val, base, needle = case
    rc, msg = _create(lib, fmt, ptr, idx, val, base)
    assert rc == 1, (rc, msg)
    assert needle in msg


def test_create_rejects_inconsistent_sizes(lib):
    rc, msg = _create(lib, 0, [0, 1, 2], [0, 1], [1.0, 1.0], nnz=3)
    assert rc == 1 and "nnz" in msg
    rc, msg = _create(lib, 0, [0, 1], [0], [1.0], n=-1)
    assert rc == 1
    h = ctypes.c_void_p()
    assert lib.gbcg_create(None, 0, 0, 0, None, None, None, 0, 0, None) == 1
    assert lib.gbcg_create(ctypes.byref(h), 0, 1, 1, None, None, None, 0, 0, None) == 1


def test_null_handle_calls(lib):
    assert lib.gbcg_spmv(None, None, None, None) == 1
    assert lib.gbcg_solve(None, None, None, 1e-10, 0, None, None, None) == 1
    assert lib.gbcg_destroy(None) == 0
    s = _lib.Stats()
    assert lib.gbcg_stats(None, ctypes.byref(s)) == 1


def test_python_binding_fails_loudly_without_library(tmp_path):
    with pytest.raises(ImportError):
        saved = _lib._lib
        _lib._lib = None
        try:
            _lib.load(str(tmp_path / "missing.so"))
        finally:
            _lib._lib = saved


def test_device_info_layout_and_decoder():
    """gbcg_device_info is 32 bytes (status, iterations, outer, pad, then the
    two residuals) and device_info() reads it field by field."""
    import struct

    import torch

    import paper_1010_4639_gb300 as gb
    assert _lib.DEVICE_INFO_BYTES == struct.calcsize("<iiiidd")
    raw = struct.pack("<iiiidd", 2, 17, 3, 0, 1.5e-3, 2.5e-11)
    info = gb.device_info(torch.frombuffer(bytearray(raw), dtype=torch.uint8))
    assert (info.status, info.iterations, info.outer) == ("NOT_SPD", 17, 3)
    assert info.rel_res_recursive == 1.5e-3 and info.rel_res_true == 2.5e-11


def test_solve_async_rejects_bad_arguments_without_a_gpu(lib):
    # argument checks run before any device work
    assert lib.gbcg_solve_async(None, None, None, 1e-10, 0, None, None, None) == 1
    assert b"null matrix handle" in lib.gbcg_last_error()


def test_both_bench_arms_share_the_workload_config():
    import argparse

    import bench
    import femgen
    g = femgen.PAPER_SIZE
    s = femgen.build_system(g)
    for fmt in ("csr", "sym", "csc"):
        args = argparse.Namespace(format=fmt, precision="fp32_ru")
        c = bench.workload_config(g, s, args, 1)
        assert c["n"] == s.n and c["nnz"] == s.nnz
        assert c["nnz_stored"] == (s.upper()[1].shape[0] if fmt == "sym" else s.nnz)
        assert f"{fmt} storage, fp32_ru, tol 1e-10" in c["workload"]
        assert c["l2"].startswith("matrix fits L2")


def test_header_is_plain_c_and_links(tmp_path):
    """include/gbcg.h compiles as C99 with warnings as errors, and a C program
    that calls the boundary links against the library (no GPU call is made:
    only argument checks run)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "gbcg.h"
int main(void) {
  gbcg_matrix_t A = NULL;
  gbcg_info info;
  gbcg_device_info* dinfo = NULL;
  int rc = gbcg_solve(A, NULL, NULL, 1e-10, 0, NULL, &info, NULL);
  int rc2 = gbcg_solve_async(A, NULL, NULL, 1e-10, 0, NULL, dinfo, NULL);
  printf("%d %d %s\n", rc, rc2, gbcg_status_string(rc));
  return (rc == GBCG_ERR_INVALID && rc2 == GBCG_ERR_INVALID) ? 0 : 1;
}
''')
    inc = os.path.join(os.path.dirname(__file__), "..", "include")
    libdir = os.path.dirname(_lib.LIB_PATH)
    exe = tmp_path / "use"
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", inc, str(src), "-L", libdir, "-lgbcg",
                    f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.split()[2] == "GBCG_ERR_INVALID"
