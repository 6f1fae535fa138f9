"""GPU conjugate gradient (persistent kernel, FP64 and FP32-inner refinement)
against the CPU oracle, through the C ABI.

Gates (each summation order gives a different but equally valid CG run):
  - true relative residual ||b - A x|| / ||b||, recomputed by the oracle's
    double-precision product, <= tol;
  - iteration count within 5% + 5 of the oracle's;
  - solved to 1e-12 on both sides, ||x - x_oracle|| / ||x_oracle|| <= 1e-8.
"""
import os

import numpy as np
import pytest

import femgen
import oracle
import paper_1010_4639_gb300 as gb
from gpu_cases import fem, random_spd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    gb.build()
    assert torch.cuda.is_available()
    return torch


def arrays(s, fmt):
    return {"csr": (s.ptr, s.idx, s.val), "sym": s.upper(), "csc": s.csc()}[fmt]


def true_rel_res(s, x):
    r = s.b - oracle.spmv("csr", s.ptr, s.idx, s.val, x)
    return np.linalg.norm(r) / np.linalg.norm(s.b)


def gpu_solve(torch, s, fmt, tol, **kw):
    with gb.Matrix(fmt, *arrays(s, fmt)) as A:
        b = torch.from_numpy(s.b).cuda()
        x, info = A.solve(b, tol=tol, **kw)
        return x.cpu().numpy(), info


@pytest.mark.parametrize("grid", [(6, 7, 8), (12, 12, 12), (31, 31, 32)])
@pytest.mark.parametrize("fmt", ["sym", "csr", "csc"])
def test_fp64_cg_matches_oracle(torch, grid, fmt):
    s = fem(*grid)
    # at the paper's default bound N = n both sides stop together on the
    # smallest grid (floating-point CG there needs more than n steps)
    r0 = oracle.cg(fmt, *arrays(s, fmt), s.b, tol=1e-10)
    _, i0 = gpu_solve(torch, s, fmt, 1e-10, raise_on_error=False)
    assert (i0.status == "OK") == (r0.status == "OK")
    ref = oracle.cg(fmt, *arrays(s, fmt), s.b, tol=1e-10, maxit=10 * s.n)
    x, info = gpu_solve(torch, s, fmt, 1e-10, maxit=10 * s.n)
    assert info.status == "OK"
    assert true_rel_res(s, x) <= 1e-10
    assert abs(info.rel_res_true - true_rel_res(s, x)) <= 1e-3 * true_rel_res(s, x) + 1e-16
    assert abs(info.iterations - ref.iterations) <= 0.05 * ref.iterations + 5, (info.iterations, ref.iterations)
    ref12 = oracle.cg(fmt, *arrays(s, fmt), s.b, tol=1e-12, maxit=10 * s.n)
    x12, info12 = gpu_solve(torch, s, fmt, 1e-12, maxit=10 * s.n)
    assert info12.status == "OK" and ref12.status == "OK"
    assert np.linalg.norm(x12 - ref12.x) <= 1e-8 * np.linalg.norm(ref12.x)


@pytest.mark.parametrize("fmt", ["sym", "csr"])
def test_mixed_precision_refinement(torch, fmt):
    s = fem(31, 31, 32)
    x, info = gpu_solve(torch, s, fmt, 1e-10, precision="fp32_ir", inner_tol=1e-4)
    assert info.status == "OK"
    assert true_rel_res(s, x) <= 1e-10
    assert 2 <= info.outer <= 10
    ref12 = oracle.cg(fmt, *arrays(s, fmt), s.b, tol=1e-12)
    x12, info12 = gpu_solve(torch, s, fmt, 1e-12, precision="fp32_ir", inner_tol=1e-4)
    assert info12.status == "OK"
    assert np.linalg.norm(x12 - ref12.x) <= 1e-8 * np.linalg.norm(ref12.x)
    # the oracle's own refinement needs a similar amount of inner work
    ir = oracle.cg_ir(fmt, *arrays(s, fmt), s.b, tol=1e-10, inner_tol=1e-4)
    assert abs(info.iterations - ir.iterations) <= 0.1 * ir.iterations + 10


def test_edge_cases(torch):
    s = fem(9, 8, 7)
    with gb.Matrix("sym", *s.upper()) as A:
        z = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        x, info = A.solve(z, torch.ones_like(z))
        assert info.status == "OK" and info.iterations == 0 and not torch.any(x).item()   # b = 0 -> x = 0
        b = torch.from_numpy(s.b).cuda()
        x, info = A.solve(b, tol=1e-13, maxit=10 * s.n)
        x2, info2 = A.solve(b, x.clone(), tol=1e-10)                                         # x0 solves it
        assert info2.status == "OK" and info2.iterations == 0
        for prec in ("fp64", "fp32_ir"):
            _, inf3 = A.solve(b, tol=1e-30, maxit=5, precision=prec, raise_on_error=False)
            assert inf3.status == "MAXIT"
        xm, inf4 = A.solve(b, tol=1e-30, maxit=5, raise_on_error=False)
        ref = oracle.cg("sym", *s.upper(), s.b, tol=1e-30, maxit=5)
        assert inf4.iterations == ref.iterations == 5
        assert np.linalg.norm(xm.cpu().numpy() - ref.x) <= 1e-11 * np.linalg.norm(ref.x)
        bn = b.clone()
        bn[3] = float("nan")
        _, inf5 = A.solve(bn, raise_on_error=False)
        assert inf5.status == "NONFINITE"
    up = s.upper()
    with gb.Matrix("sym", up[0], up[1], -up[2]) as A:                                     # negative definite
        _, inf6 = A.solve(torch.from_numpy(s.b).cuda(), raise_on_error=False)
        assert inf6.status == "NOT_SPD" and inf6.iterations == 0
        _, inf7 = A.solve(torch.from_numpy(s.b).cuda(), precision="fp32_ir", raise_on_error=False)
        assert inf7.status == "NOT_SPD"


def test_host_memory_path_and_determinism(torch):
    s = fem(12, 11, 13)
    with gb.Matrix("sym", *s.upper()) as A:
        b = torch.from_numpy(s.b).cuda()
        x1, _ = A.solve(b)
        x2, _ = A.solve(b)
        assert torch.equal(x1, x2)                    # bitwise reproducible
        xh = np.zeros(s.n)
        xh, info = A.solve(s.b.copy(), xh)            # host b and x: copies inside the call
        assert info.status == "OK"
        assert np.array_equal(xh, x1.cpu().numpy())


@pytest.mark.parametrize("grid_ctas", ["1", "7", "64"])
def test_grid_sizes(torch, grid_ctas, monkeypatch):
    monkeypatch.setenv("GBCG_GRID", grid_ctas)
    s = fem(14, 13, 12)
    for fmt in ("sym", "csr"):
        x, info = gpu_solve(torch, s, fmt, 1e-10)
        assert info.status == "OK" and true_rel_res(s, x) <= 1e-10


def test_random_spd_with_long_rows(torch):
    ptr, idx, val = random_spd(3000, 9, density=0.003, dense_rows=(7, 1500))
    b = np.random.default_rng(1).uniform(-1, 1, 3000)
    ref = oracle.cg("csr", ptr, idx, val, b, tol=1e-12)
    for fmt, arrs in (("csr", (ptr, idx, val)), ("sym", femgen.upper(3000, ptr, idx, val))):
        with gb.Matrix(fmt, *arrs) as A:
            x, info = A.solve(torch.from_numpy(b).cuda(), tol=1e-12)
        assert info.status == "OK"
        assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


def test_wait_timeout_is_bounded_and_recoverable(torch):
    # One CTA never arrives at the barrier: the others must give up and report.
    assert gb.selftest_wait_timeout(ctas=0, timeout_ms=50) == 5      # GBCG_ERR_TIMEOUT
    assert gb.selftest_wait_timeout(ctas=4, timeout_ms=20) == 5
    s = fem(8, 8, 8)
    x, info = gpu_solve(torch, s, "sym", 1e-10)                        # context still usable
    assert info.status == "OK"


def test_misaligned_device_vectors_are_rejected(torch):
    # the kernels move vectors with 16-byte loads and bulk copies: an 8-byte
    # offset view is refused on the host with GBCG_ERR_INVALID, no launch
    s = fem(9, 8, 7)
    with gb.Matrix("sym", *s.upper()) as A:
        buf = torch.zeros(2 * s.n + 2, dtype=torch.float64, device="cuda")
        xo, yo = buf[1:s.n + 1], buf[s.n + 2:]
        assert xo.data_ptr() % 16 == 8
        with pytest.raises(gb.GbcgError, match="16-byte aligned"):
            A.spmv(xo, torch.empty_like(xo))
        with pytest.raises(gb.GbcgError, match="16-byte aligned"):
            A.solve(xo, yo)
        with pytest.raises(gb.GbcgError, match="16-byte aligned"):
            A.spmv_f32(torch.zeros(s.n, dtype=torch.float32, device="cuda"),
                       torch.empty(s.n + 2, dtype=torch.float32, device="cuda")[2:])
        # aligned views of the same buffer are accepted
        x, info = A.solve(torch.from_numpy(s.b).cuda(), buf[:s.n])
        assert info.status == "OK"
