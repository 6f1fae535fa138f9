"""gbcg_solve_async: the solve enqueued without host synchronisation, its
result written to device memory; and the same call captured into a CUDA
graph and replayed.  The iterates and the result fields must equal those of
gbcg_solve bit for bit (same kernels, same launch)."""
import numpy as np
import pytest

import femgen
import paper_1010_4639_gb300 as gb
from gpu_cases import fem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    gb.build()
    assert torch.cuda.is_available()
    return torch


def dinfo_buffer(torch):
    return torch.zeros(gb._lib.DEVICE_INFO_BYTES, dtype=torch.uint8, device="cuda")


def same_result(ia, isync):
    assert ia.status == isync.status
    assert ia.iterations == isync.iterations and ia.outer == isync.outer
    assert ia.rel_res_true == isync.rel_res_true


@pytest.mark.parametrize("fmt,precision,variant", [("csr", "fp64", "standard"), ("csr", "fp32_ru", "standard"),
                                                   ("csr", "fp64", "pipelined"), ("tiles", "fp32_ru", "standard"),
                                                   ("tiles", "fp64", "standard")])
def test_async_equals_sync(torch, fmt, precision, variant):
    s = fem(17, 15, 19)
    arrs = (s.ptr, s.idx, s.val) if fmt == "csr" else s.upper()
    with gb.Matrix("csr" if fmt == "csr" else "sym", *arrs) as A:
        b = torch.from_numpy(s.b).cuda()
        xs, isync = A.solve(b, tol=1e-10, precision=precision, variant=variant)
        x = torch.zeros_like(b)
        d = dinfo_buffer(torch)
        A.solve_async(b, x, d, tol=1e-10, precision=precision, variant=variant)
        torch.cuda.synchronize()
        assert torch.equal(x, xs)
        ia = gb.device_info(d)
        assert ia.status == "OK"
        same_result(ia, isync)


def test_async_statuses(torch):
    s = fem(9, 8, 7)
    d = dinfo_buffer(torch)
    b = torch.from_numpy(s.b).cuda()
    with gb.Matrix("csr", s.ptr, s.idx, s.val) as A:
        x = torch.zeros_like(b)
        A.solve_async(b, x, d, tol=1e-30, maxit=4)
        assert gb.device_info(d).status == "MAXIT" and gb.device_info(d).iterations == 4
        with pytest.raises(gb.GbcgError, match="host"):
            A.solve_async(b, x, d, precision="fp32_ir")
    with gb.Matrix("csr", s.ptr, s.idx, -s.val) as N:
        x = torch.zeros_like(b)
        N.solve_async(b, x, d, precision="fp32_ru")
        info = gb.device_info(d)
        assert info.status == "NOT_SPD" and info.iterations == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32_ru"])
def test_async_solve_in_a_cuda_graph(torch, precision):
    s = fem(17, 15, 19)
    s2 = fem(17, 15, 19, seed_x=7)  # same matrix, another right-hand side
    assert np.array_equal(s2.val, s.val)
    with gb.Matrix("csr", s.ptr, s.idx, s.val) as A:
        b = torch.from_numpy(s.b).cuda()
        x = torch.zeros_like(b)
        d = dinfo_buffer(torch)
        A.solve_async(b, x, d, tol=1e-10, precision=precision)  # kernels loaded before the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            x.zero_()
            A.solve_async(b, x, d, tol=1e-10, precision=precision, stream=torch.cuda.current_stream())
        for sys_, label in ((s, "first"), (s2, "second")):
            b.copy_(torch.from_numpy(sys_.b))
            g.replay()
            torch.cuda.synchronize()
            xs, isync = A.solve(torch.from_numpy(sys_.b).cuda(), tol=1e-10, precision=precision)
            assert torch.equal(x, xs), label
            same_result(gb.device_info(d), isync)
