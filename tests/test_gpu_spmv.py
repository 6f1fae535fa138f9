"""GPU sparse products against the CPU oracle, element by element, through the C ABI.

Tolerance (double precision): |y_i - y_i^oracle| <= 1e-13 * (|A| |x|)_i, the
componentwise form of "relative error <= 1e-13 per entry": rows of a
stiffness matrix nearly cancel, so |y_i| itself can be far below the
rounding scale of its terms.  Each side's error is at most about
(row length) * 2^-53 * (|A||x|)_i, i.e. below 4e-15 here.  Single precision:
1e-5 * (|A32||x|)_i against the oracle's float product (each side within
~16 * 2^-24).
"""
import os

import numpy as np
import pytest

import femgen
import oracle
import paper_1010_4639_gb300 as gb
from gpu_cases import fem, random_general, random_spd, transpose_arrays

pytestmark = pytest.mark.gpu
TOL64 = 1e-13
TOL32 = 1e-5


@pytest.fixture(scope="module")
def torch():
    import torch
    gb.build()
    assert torch.cuda.is_available()
    return torch


def check(y, yref, scale, tol):
    err = np.abs(y - yref)
    bound = tol * scale
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, f"{bad.size} rows off, worst ratio {np.max(err / np.maximum(bound, 1e-300)):.3g}"


def gpu_spmv(torch, fmt, arrs, x, base=0, device_input=False):
    ptr, idx, val = arrs
    if base:
        ptr, idx = ptr + 1, idx + 1
    if device_input:
        args = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (ptr, idx, val)]
    else:
        args = [ptr, idx, val]
    with gb.Matrix(fmt, *args, index_base=base) as A:
        xd = torch.from_numpy(x).cuda()
        y1 = A.spmv(xd).cpu().numpy()
        y2 = A.spmv(xd).cpu().numpy()
        assert np.array_equal(y1, y2)  # deterministic: no floating-point atomics
        return y1, A.stats()


FEM_GRIDS = [(5, 5, 5), (9, 10, 11), (12, 12, 12), (31, 31, 32)]


@pytest.mark.parametrize("grid", FEM_GRIDS)
@pytest.mark.parametrize("fmt", ["csr", "sym", "csc"])
def test_fem_spmv_matches_oracle(torch, grid, fmt):
    s = fem(*grid)
    arrs = {"csr": (s.ptr, s.idx, s.val), "sym": s.upper(), "csc": s.csc()}[fmt]
    x = femgen.random_vector(s.n, 11)
    y, st = gpu_spmv(torch, fmt, arrs, x)
    check(y, oracle.spmv(fmt, *arrs, x), oracle.abs_spmv(fmt, *arrs, x), TOL64)
    assert st["nnz_full"] == s.nnz


@pytest.mark.parametrize("n,seed", [(1, 0), (33, 1), (200, 2), (1500, 3), (4097, 4)])
def test_general_csr_and_csc_edge_rows(torch, n, seed):
    empty = (0,) if n > 1 else ()
    ones = (n // 3,) if n > 2 else ()
    longr = (n // 2,) if n >= 200 else ()
    ptr, idx, val = random_general(n, n, min(0.5, 8.0 / n), seed, empty_rows=empty, one_rows=ones,
                                   long_rows=longr, long_len=1000)
    x = np.random.default_rng(seed).uniform(-1, 1, n)
    y, st = gpu_spmv(torch, "csr", (ptr, idx, val), x)
    check(y, oracle.spmv("csr", ptr, idx, val, x), oracle.abs_spmv("csr", ptr, idx, val, x), TOL64)
    if longr:
        assert st["long_rows"] >= 1
    # the same matrix handed over by columns
    cptr, cidx, cval = transpose_arrays(n, n, ptr, idx, val)
    y2, _ = gpu_spmv(torch, "csc", (cptr, cidx, cval), x)
    check(y2, oracle.spmv("csc", cptr, cidx, cval, x), oracle.abs_spmv("csc", cptr, cidx, cval, x), TOL64)


@pytest.mark.parametrize("n,seed,dense", [(2, 0, ()), (31, 1, ()), (700, 2, (5,)), (3000, 3, (100, 2999))])
def test_sym_upper_random_spd(torch, n, seed, dense):
    ptr, idx, val = random_spd(n, seed, density=min(0.3, 10.0 / n), dense_rows=dense)
    up = femgen.upper(n, ptr, idx, val)
    x = np.random.default_rng(seed).uniform(-1, 1, n)
    y, _ = gpu_spmv(torch, "sym", up, x)
    check(y, oracle.spmv("sym", *up, x), oracle.abs_spmv("sym", *up, x), TOL64)
    # and against the full storage of the same matrix
    yf, _ = gpu_spmv(torch, "csr", (ptr, idx, val), x)
    check(y, yf, oracle.abs_spmv("csr", ptr, idx, val, x), 2 * TOL64)


def test_one_based_and_device_input(torch):
    s = fem(8, 9, 10)
    x = femgen.random_vector(s.n, 3)
    for fmt, arrs in (("csr", (s.ptr, s.idx, s.val)), ("sym", s.upper())):
        ref = oracle.spmv(fmt, *arrs, x)
        sc = oracle.abs_spmv(fmt, *arrs, x)
        y1, _ = gpu_spmv(torch, fmt, arrs, x, base=1)
        y2, _ = gpu_spmv(torch, fmt, arrs, x, device_input=True)
        check(y1, ref, sc, TOL64)
        assert np.array_equal(y1, y2)


def test_empty_matrix_and_zero_rows(torch):
    with gb.Matrix("csr", np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0)) as A:
        assert A.n == 0
    ptr = np.zeros(41, np.int32)  # 40 rows, no entries
    with gb.Matrix("csr", ptr, np.zeros(0, np.int32), np.zeros(0)) as A:
        y = A.spmv(torch.ones(40, dtype=torch.float64, device="cuda"))
        assert not torch.any(y).item()


@pytest.mark.parametrize("fmt", ["csr", "sym", "csc"])
def test_fp32_product(torch, fmt):
    s = fem(13, 12, 11)
    arrs = {"csr": (s.ptr, s.idx, s.val), "sym": s.upper(), "csc": s.csc()}[fmt]
    x32 = femgen.random_vector(s.n, 5).astype(np.float32)
    v32 = arrs[2].astype(np.float32)
    ref = oracle.spmv_f32(fmt, arrs[0], arrs[1], v32, x32).astype(np.float64)
    sc = oracle.abs_spmv(fmt, arrs[0], arrs[1], v32.astype(np.float64), x32.astype(np.float64))
    with gb.Matrix(fmt, *arrs) as A:
        y = A.spmv_f32(torch.from_numpy(x32).cuda()).cpu().numpy().astype(np.float64)
    check(y, ref, sc, TOL32)


def test_full_size_128_all_formats(torch):
    # the 128^3 workload the benchmark times: every output row against the oracle
    s = fem(128, 128, 128)
    x = femgen.random_vector(s.n, 21)
    for fmt, arrs in (("csr", (s.ptr, s.idx, s.val)), ("sym", s.upper()), ("csc", s.csc())):
        y, st = gpu_spmv(torch, fmt, arrs, x)
        check(y, oracle.spmv(fmt, *arrs, x), oracle.abs_spmv(fmt, *arrs, x), TOL64)
        assert st["n"] == 2000376


@pytest.mark.parametrize("layout", ["tiles", "plan"])
def test_symmetric_layouts(torch, layout, monkeypatch):
    # both symmetric layouts (warp tiles with shared-memory accumulation, and
    # the transpose-plan gather kept for matrices whose tiles would not fit)
    monkeypatch.setenv("GBCG_SYM_LAYOUT", layout)
    for grid in [(9, 10, 11), (31, 31, 32)]:
        s = fem(*grid)
        up = s.upper()
        x = femgen.random_vector(s.n, 17)
        y, st = gpu_spmv(torch, "sym", up, x)
        assert st["layout"] == (2 if layout == "tiles" else 1)
        check(y, oracle.spmv("sym", *up, x), oracle.abs_spmv("sym", *up, x), TOL64)
        b = torch.from_numpy(s.b).cuda()
        with gb.Matrix("sym", *up) as A:
            xs, info = A.solve(b, tol=1e-10, maxit=10 * s.n)
            assert info.status == "OK"
            xi, info2 = A.solve(b, tol=1e-10, precision="fp32_ir", maxit=10 * s.n)
            assert info2.status == "OK"
        for sol in (xs, xi):
            r = s.b - oracle.spmv("csr", s.ptr, s.idx, s.val, sol.cpu().numpy())
            assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(s.b)


@pytest.mark.parametrize("fmt", ["csr", "csc"])
def test_narrow_and_wide_indices_agree(torch, fmt):
    """16-bit column offsets (chosen when every offset fits) and int32 column
    indices give the same products bit for bit (same sums, same order)."""
    s = fem(17, 15, 19)
    arrs = (s.ptr, s.idx, s.val) if fmt == "csr" else s.csc()
    x = torch.from_numpy(np.random.default_rng(9).uniform(-1, 1, s.n)).cuda()
    with gb.Matrix(fmt, *arrs) as N:
        assert N.stats()["index_bytes"] == 2
        yn, yn32 = N.spmv(x), N.spmv_f32(x.float())
    old = os.environ.get("GBCG_WIDE_INDEX")
    os.environ["GBCG_WIDE_INDEX"] = "1"
    try:
        W = gb.Matrix(fmt, *arrs)
    finally:
        if old is None:
            os.environ.pop("GBCG_WIDE_INDEX", None)
        else:
            os.environ["GBCG_WIDE_INDEX"] = old
    with W:
        assert W.stats()["index_bytes"] == 4
        assert torch.equal(W.spmv(x), yn) and torch.equal(W.spmv_f32(x.float()), yn32)


@pytest.mark.parametrize("ctas", [1, 3])
def test_one_shot_product_many_slices_per_warp(torch, ctas, monkeypatch):
    """Small grids give each warp more than 32 slices, so the one-shot
    product's slice-metadata window moves on while fills of the previous
    window are still in flight; mixed slice lengths (empty rows, rows past
    the stage size) cross the window edges too.  Double and single precision,
    16-bit offsets and int32 indices."""
    monkeypatch.setenv("GBCG_GRID", str(ctas))
    s = fem(31, 31, 32)
    ptr, idx, val = random_general(20000, 20000, 6.0 / 20000, 5, empty_rows=tuple(range(0, 20000, 97)),
                                   one_rows=tuple(range(3, 20000, 89)), long_rows=tuple(range(11, 20000, 1409)),
                                   long_len=300)
    cases = [("csr", (s.ptr, s.idx, s.val)), ("csc", s.csc()), ("csr", (ptr, idx, val))]
    for wide in ("0", "1"):
        monkeypatch.setenv("GBCG_WIDE_INDEX", wide)
        for fmt, arrs in cases:
            n = arrs[0].shape[0] - 1
            x = femgen.random_vector(n, 23)
            y, st = gpu_spmv(torch, fmt, arrs, x)
            assert st["grid_ctas"] == ctas and st["layout"] == 0
            check(y, oracle.spmv(fmt, *arrs, x), oracle.abs_spmv(fmt, *arrs, x), TOL64)
            x32 = x.astype(np.float32)
            v32 = arrs[2].astype(np.float32)
            with gb.Matrix(fmt, *arrs) as A:
                y32 = A.spmv_f32(torch.from_numpy(x32).cuda()).cpu().numpy().astype(np.float64)
            check(y32, oracle.spmv_f32(fmt, arrs[0], arrs[1], v32, x32).astype(np.float64),
                  oracle.abs_spmv(fmt, arrs[0], arrs[1], v32.astype(np.float64), x32.astype(np.float64)), TOL32)


def test_symmetry_check_in_debug_mode(torch, monkeypatch):
    """GBCG_CHECK_SYMMETRY=1: full CSR/CSC input must be symmetric, pattern
    and values bit for bit; off by default (the products are exact for any
    matrix)."""
    s = fem(5, 6, 7)
    ptr, idx, val = random_general(60, 60, 0.1, 3)
    with gb.Matrix("csr", ptr, idx, val):
        pass
    monkeypatch.setenv("GBCG_CHECK_SYMMETRY", "1")
    with gb.Matrix("csr", s.ptr, s.idx, s.val):
        pass
    with gb.Matrix("csc", *s.csc()):
        pass
    rows = np.repeat(np.arange(s.n), np.diff(s.ptr))
    k = int(np.nonzero(s.idx != rows)[0][0])  # an off-diagonal entry
    v = s.val.copy()
    v[k] = np.nextafter(v[k], np.inf)
    with pytest.raises(gb.GbcgError, match=f"not symmetric at entry \\({rows[k]}, {s.idx[k]}\\)"):
        gb.Matrix("csr", s.ptr, s.idx, v)
    with pytest.raises(gb.GbcgError, match="not symmetric"):
        gb.Matrix("csr", ptr, idx, val)
