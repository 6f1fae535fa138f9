"""Single-precision CG with double-precision reliable updates on the GPU
against the oracle's, through the C ABI.  Gates: true relative residual
(recomputed by the oracle's double-precision product) <= tol; iteration count
within 10% + 10 of the oracle's (single-precision iterations, reading of the
inner CG's gate); solved to 1e-12 on both sides, within 1e-8 of the oracle's
double-precision solution."""
import os

import numpy as np
import pytest

import femgen
import oracle
import paper_1010_4639_gb300 as gb
from gpu_cases import fem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    gb.build()
    assert torch.cuda.is_available()
    return torch


def arrays(s, fmt):
    return {"csr": (s.ptr, s.idx, s.val), "sym": s.upper(), "tiles": s.upper(), "csc": s.csc()}[fmt]


def oracle_fmt(fmt):
    return "sym" if fmt == "tiles" else fmt


def true_rel_res(s, x):
    return np.linalg.norm(s.b - oracle.spmv("csr", s.ptr, s.idx, s.val, x)) / np.linalg.norm(s.b)


def make(fmt, s):
    """"tiles": symmetric storage in the default (tiled) layout; "sym": the
    transpose-plan layout."""
    if fmt == "tiles":
        A = gb.Matrix("sym", *arrays(s, fmt))
        assert A.stats()["layout"] == 2
        return A
    if fmt != "sym":
        return gb.Matrix(fmt, *arrays(s, fmt))
    old = os.environ.get("GBCG_SYM_LAYOUT")
    os.environ["GBCG_SYM_LAYOUT"] = "plan"
    try:
        return gb.Matrix(fmt, *arrays(s, fmt))
    finally:
        if old is None:
            os.environ.pop("GBCG_SYM_LAYOUT", None)
        else:
            os.environ["GBCG_SYM_LAYOUT"] = old


@pytest.mark.parametrize("fmt,grid", [("csr", (31, 31, 32)), ("csc", (17, 15, 19)), ("sym", (31, 31, 32)),
                                      ("csr", (17, 15, 19)), ("tiles", (31, 31, 32)), ("tiles", (9, 10, 11))])
def test_reliable_updates_match_oracle(torch, fmt, grid):
    s = fem(*grid)
    b = torch.from_numpy(s.b).cuda()
    with make(fmt, s) as A:
        x, info = A.solve(b, tol=1e-10, maxit=10 * s.n, precision="fp32_ru")
        assert info.status == "OK", info
        ref = oracle.cg_ru(oracle_fmt(fmt), *arrays(s, fmt), s.b, tol=1e-10, maxit=10 * s.n)
        assert ref.status == "OK"
        assert true_rel_res(s, x.cpu().numpy()) <= 1e-10
        assert abs(info.iterations - ref.iterations) <= 0.10 * ref.iterations + 10, (info.iterations, ref.iterations)
        assert abs(info.outer - ref.restarts) <= 2, (info.outer, ref.restarts)
        x12, i12 = A.solve(b, tol=1e-12, maxit=10 * s.n, precision="fp32_ru")
        assert i12.status == "OK", i12
        ref12 = oracle.cg(oracle_fmt(fmt), *arrays(s, fmt), s.b, tol=1e-12, maxit=10 * s.n)
        assert np.linalg.norm(x12.cpu().numpy() - ref12.x) <= 1e-8 * np.linalg.norm(ref12.x)
        x2, _ = A.solve(b, tol=1e-10, maxit=10 * s.n, precision="fp32_ru")
        assert torch.equal(x, x2)


def test_reliable_updates_edge_cases(torch):
    s = fem(9, 8, 7)
    with gb.Matrix("csr", s.ptr, s.idx, s.val) as A:
        z = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        x, info = A.solve(z, torch.ones_like(z), precision="fp32_ru")
        assert info.status == "OK" and info.iterations == 0 and not torch.any(x).item()
        xs = torch.from_numpy(s.xstar).cuda()
        x, info = A.solve(A.spmv(xs), xs.clone(), tol=1e-8, precision="fp32_ru")
        assert info.status == "OK" and info.iterations == 0
        x, info = A.solve(torch.from_numpy(s.b).cuda(), tol=1e-30, maxit=4, precision="fp32_ru",
                          raise_on_error=False)
        assert info.status == "MAXIT" and info.iterations == 4
    with gb.Matrix("csr", s.ptr, s.idx, -s.val) as N:
        x, info = N.solve(torch.from_numpy(s.b).cuda(), precision="fp32_ru", raise_on_error=False)
        ref = oracle.cg_ru("csr", s.ptr, s.idx, -s.val, s.b)
        assert info.status == ref.status == "NOT_SPD" and info.iterations == 0


def test_reliable_updates_tiled_layout_edge_cases(torch):
    s = fem(9, 8, 7)
    with make("tiles", s) as A:
        z = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        x, info = A.solve(z, torch.ones_like(z), precision="fp32_ru")
        assert info.status == "OK" and info.iterations == 0 and not torch.any(x).item()
        xs = torch.from_numpy(s.xstar).cuda()
        x, info = A.solve(A.spmv(xs), xs.clone(), tol=1e-8, precision="fp32_ru")
        assert info.status == "OK" and info.iterations == 0
        x, info = A.solve(torch.from_numpy(s.b).cuda(), tol=1e-30, maxit=4, precision="fp32_ru",
                          raise_on_error=False)
        assert info.status == "MAXIT" and info.iterations == 4
    up = s.upper()
    with gb.Matrix("sym", up[0], up[1], -up[2]) as N:
        assert N.stats()["layout"] == 2
        x, info = N.solve(torch.from_numpy(s.b).cuda(), precision="fp32_ru", raise_on_error=False)
        ref = oracle.cg_ru("sym", up[0], up[1], -up[2], s.b)
        assert info.status == ref.status == "NOT_SPD" and info.iterations == 0


@pytest.mark.parametrize("ctas", ["1", "7"])
def test_reliable_updates_tiled_layout_grid_sizes(torch, ctas, monkeypatch):
    s = fem(17, 15, 19)
    monkeypatch.setenv("GBCG_GRID", ctas)
    with make("tiles", s) as A:
        assert A.stats()["grid_ctas"] == int(ctas)
        x, info = A.solve(torch.from_numpy(s.b).cuda(), tol=1e-10, maxit=10 * s.n, precision="fp32_ru")
    assert info.status == "OK", info
    assert true_rel_res(s, x.cpu().numpy()) <= 1e-10


@pytest.mark.parametrize("grid,ctas,precision", [((9, 10, 11), "7", "fp32_ru"), ((31, 31, 32), None, "fp32_ru"),
                                                 ((128, 128, 128), None, "fp32_ru"), ((9, 10, 11), "7", "fp64"),
                                                 ((64, 64, 64), None, "fp64"), ((31, 31, 32), None, "fp32_ir")])
def test_streamed_vector_passes(torch, grid, ctas, precision, monkeypatch):
    # the tiled solvers' vector passes either stream their vectors through
    # shared memory (bulk copies, 8 KB chunks per vector, four in flight; the
    # default once they outgrow the L2) or keep them in registers.  Each
    # thread visits the same rows in the same order either way, so the
    # iterates are bit for bit the same.  Ragged CTA ranges and a tail of
    # rows past the last 16-byte group (n = 990), one chunk per CTA (31^3),
    # chunks reusing buffers (128^3: 13 000 rows per CTA; 64^3 in double
    # precision: 1 600 rows per CTA, 1 024 per chunk)
    s = fem(*grid)
    if ctas:
        monkeypatch.setenv("GBCG_GRID", ctas)
    b = torch.from_numpy(s.b).cuda()
    out = {}
    for flag in ("0", "1"):
        monkeypatch.setenv("GBCG_STREAM_VEC", flag)
        with make("tiles", s) as A:
            x, info = A.solve(b, tol=1e-10, maxit=10 * s.n, precision=precision)
        assert info.status == "OK", info
        out[flag] = (x, info)
    (x0, i0), (x1, i1) = out["0"], out["1"]
    assert (i0.iterations, i0.outer) == (i1.iterations, i1.outer)
    assert torch.equal(x0, x1)
    assert true_rel_res(s, x1.cpu().numpy()) <= 1e-10
