"""The largest single system of the workload set (256^3 node grid, four
inclusions, 16.4M rows, 130M stored upper entries): the symmetric product in
double and single precision against the oracle on every row (tolerances as
in test_gpu_spmv).  Its solves are gated against the oracle's own solves in
test_gpu_golden."""
import numpy as np
import pytest

import femgen
import oracle
import paper_1010_4639_gb300 as gb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    gb.build()
    assert torch.cuda.is_available()
    return torch


@pytest.fixture(scope="module")
def system():
    return femgen.build_system(femgen.LARGEST)


def within(y, ref, scale, tol):
    bad = np.nonzero(np.abs(y - ref) > tol * scale)[0]
    assert bad.size == 0, f"{bad.size} rows off"


def test_largest_symmetric_products(torch, system):
    s = system
    up = s.upper()
    x = femgen.random_vector(s.n, 31)
    with gb.Matrix("sym", *up) as A:
        assert A.stats()["n"] == 16387064
        y = A.spmv(torch.from_numpy(x).cuda()).cpu().numpy()
        x32 = x.astype(np.float32)
        y32 = A.spmv_f32(torch.from_numpy(x32).cuda()).cpu().numpy().astype(np.float64)
    within(y, oracle.spmv("sym", *up, x), oracle.abs_spmv("sym", *up, x), 1e-13)
    v32 = up[2].astype(np.float32)
    within(y32, oracle.spmv_f32("sym", up[0], up[1], v32, x32).astype(np.float64),
           oracle.abs_spmv("sym", up[0], up[1], v32.astype(np.float64), x32.astype(np.float64)), 1e-5)
