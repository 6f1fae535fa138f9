"""gbcg_solve_csr_static, the entry point that allocates nothing.

Callers that cannot allocate device memory (inside an allocator's or memory
pool's own callback, in loops where an allocation would stall the device, or
in plug-ins whose host application owns all device memory) solve through this
call, whose scratch is a fixed device array inside the library.  Its result is
checked against the existing entry point (gbcg_create + gbcg_solve on the same
CSR matrix) at the tolerance the CG tests use, on two calls in a row -- the
second call must not be disturbed by what the first left in the shared
scratch.  This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1010_4639_gb300 as gb
from gpu_cases import fem
from paper_1010_4639_gb300 import _lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    gb.build()
    assert torch.cuda.is_available()
    return torch


def static_solve(torch, s, b, x, tol, maxit):
    lib = _lib.load()
    ptr, idx, val = (torch.from_numpy(a).cuda() for a in (s.ptr, s.idx, s.val))
    info = _lib.Info()
    rc = lib.gbcg_solve_csr_static(s.n, s.nnz, ptr.data_ptr(), idx.data_ptr(), val.data_ptr(), b.data_ptr(),
                                   x.data_ptr(), tol, maxit, ctypes.byref(info),
                                   torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return rc, info


@pytest.mark.parametrize("grid", [(12, 11, 13), (31, 31, 32)])
def test_static_solve_matches_allocating_entry_point(torch, grid):
    s = fem(*grid)
    b = torch.from_numpy(s.b).cuda()
    with gb.Matrix("csr", s.ptr, s.idx, s.val) as A:
        xh, ih = A.solve(b, tol=1e-12, maxit=10 * s.n)
    assert ih.status == "OK"
    xh = xh.cpu().numpy()
    for call in range(2):
        x = torch.zeros_like(b)
        rc, info = static_solve(torch, s, b, x, 1e-12, 10 * s.n)
        assert rc == 0, (call, rc, _lib.last_error())
        xs = x.cpu().numpy()
        res = np.linalg.norm(s.b - oracle.spmv("csr", s.ptr, s.idx, s.val, xs)) / np.linalg.norm(s.b)
        assert res <= 1e-12, (call, res)
        assert np.linalg.norm(xs - xh) <= 1e-8 * np.linalg.norm(xh), call
        assert abs(info.iterations - ih.iterations) <= 0.05 * ih.iterations + 5


def test_static_solve_rejects_sizes_beyond_the_scratch(torch):
    lib = _lib.load()
    info = _lib.Info()
    n = _lib.STATIC_MAX_N + 1
    rc = lib.gbcg_solve_csr_static(n, 0, None, None, None, None, None, 1e-10, 0, ctypes.byref(info), None)
    assert rc == 1
    assert "GBCG_STATIC_MAX_N" in _lib.last_error()
