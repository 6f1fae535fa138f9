"""Full-size solves against the CPU oracle's own solves of the same systems
(tests/golden, written by make_oracle_golden.py, which calls only femgen and
oracle/): the 128^3 system (2.0M rows) and the largest single system
(256^3, four inclusions, 16.4M rows, symmetric storage), in every precision
the benchmark times.

Gates (the paper's Section III listing; readings of the design notes):
  - status OK and the true relative residual ||b - A x|| / ||b||, formed by
    the oracle's own double-precision product, <= tol;
  - iterations against the oracle's count for the same method: within
    5% + 5 in double precision, 10% + 10 for single-precision iterations
    (summation order moves the step where the recurrence first reaches tol);
  - the solution against the double-precision oracle's, on its seeded
    sample positions: both solve A x = b to relative residual tol, so
    ||x - x_or|| <= ||A^-1|| (||r|| + ||r_or||) <= 2 kappa tol ||x_or||; the
    gate is 4 kappa_hat tol, kappa_hat the oracle's Ritz estimate (a lower
    bound of kappa) taken with a factor 2 of margin.
"""
import json
import os

import numpy as np
import pytest

import femgen
import oracle
import paper_1010_4639_gb300 as gb

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL = 1e-10


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def torch():
    import torch
    gb.build()
    assert torch.cuda.is_available()
    return torch


@pytest.fixture(scope="module")
def s128():
    return femgen.build_system(femgen.LARGE)


@pytest.fixture(scope="module")
def s256():
    return femgen.build_system(femgen.LARGEST)


def check(s, x, info, fp64_gold, method_gold, single):
    assert info.status == "OK", info
    r = s.b - oracle.spmv("csr", s.ptr, s.idx, s.val, x)
    assert np.linalg.norm(r) <= TOL * np.linalg.norm(s.b)
    it_or = method_gold["iterations"]
    slack = (0.10 * it_or + 10) if single else (0.05 * it_or + 5)
    assert abs(info.iterations - it_or) <= slack, (info.iterations, it_or)
    idx = np.asarray(fp64_gold["sample_index"])
    xo = np.asarray(fp64_gold["sample_x"])
    err = np.linalg.norm(x[idx] - xo) / np.linalg.norm(xo)
    assert err <= 4 * fp64_gold["kappa_hat"] * TOL, (err, fp64_gold["kappa_hat"])
    return err


@pytest.mark.parametrize("fmt", ["sym", "csr"])
def test_128_fp64(torch, s128, fmt):
    g = golden("oracle_128_sym.json")
    arrays = s128.upper() if fmt == "sym" else (s128.ptr, s128.idx, s128.val)
    with gb.Matrix(fmt, *arrays) as A:
        x, info = A.solve(torch.from_numpy(s128.b).cuda(), tol=TOL, precision="fp64")
    check(s128, x.cpu().numpy(), info, g, g, single=False)


@pytest.mark.parametrize("fmt", ["sym", "csr"])
def test_128_reliable_updates(torch, s128, fmt):
    arrays = s128.upper() if fmt == "sym" else (s128.ptr, s128.idx, s128.val)
    with gb.Matrix(fmt, *arrays) as A:
        x, info = A.solve(torch.from_numpy(s128.b).cuda(), tol=TOL, precision="fp32_ru")
    ru = golden(f"oracle_128_{fmt}_ru.json")
    check(s128, x.cpu().numpy(), info, golden("oracle_128_sym.json"), ru, single=True)
    assert abs(info.outer - ru["restarts"]) <= 2, (info.outer, ru["restarts"])


def test_128_restarted_refinement(torch, s128):
    with gb.Matrix("sym", *s128.upper()) as A:
        x, info = A.solve(torch.from_numpy(s128.b).cuda(), tol=TOL, precision="fp32_ir")
    assert info.status == "OK", info
    x = x.cpu().numpy()
    g = golden("oracle_128_sym.json")
    r = s128.b - oracle.spmv("csr", s128.ptr, s128.idx, s128.val, x)
    assert np.linalg.norm(r) <= TOL * np.linalg.norm(s128.b)
    idx = np.asarray(g["sample_index"])
    xo = np.asarray(g["sample_x"])
    assert np.linalg.norm(x[idx] - xo) / np.linalg.norm(xo) <= 4 * g["kappa_hat"] * TOL


def test_256_fp64_symmetric(torch, s256):
    g = golden("oracle_256_sym.json")
    with gb.Matrix("sym", *s256.upper()) as A:
        x, info = A.solve(torch.from_numpy(s256.b).cuda(), tol=TOL, precision="fp64")
    check(s256, x.cpu().numpy(), info, g, g, single=False)


def test_256_reliable_updates_symmetric(torch, s256):
    ru = golden("oracle_256_sym_ru.json")
    with gb.Matrix("sym", *s256.upper()) as A:
        x, info = A.solve(torch.from_numpy(s256.b).cuda(), tol=TOL, precision="fp32_ru")
    check(s256, x.cpu().numpy(), info, golden("oracle_256_sym.json"), ru, single=True)
    assert abs(info.outer - ru["restarts"]) <= 2, (info.outer, ru["restarts"])


def test_256_restarted_refinement_symmetric(torch, s256):
    g = golden("oracle_256_sym.json")
    with gb.Matrix("sym", *s256.upper()) as A:
        x, info = A.solve(torch.from_numpy(s256.b).cuda(), tol=TOL, precision="fp32_ir")
    assert info.status == "OK", info
    x = x.cpu().numpy()
    r = s256.b - oracle.spmv("csr", s256.ptr, s256.idx, s256.val, x)
    assert np.linalg.norm(r) <= TOL * np.linalg.norm(s256.b)
    idx = np.asarray(g["sample_index"])
    xo = np.asarray(g["sample_x"])
    assert np.linalg.norm(x[idx] - xo) / np.linalg.norm(xo) <= 4 * g["kappa_hat"] * TOL
