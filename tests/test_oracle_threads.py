"""The oracle's multi-threaded build gives the single-threaded build's bits.

The threaded build (oracle.c compiled with -fopenmp into a separate library)
times the CPU baseline on every host core and computes the large reference
solves of tests/golden.  It restructures the symmetric and column-storage
products output by output and splits the pairwise single-precision dot over
threads; each output still adds the same terms in the same order.  These
tests pin that: iterates, counts and residuals equal bit for bit, in every
storage format, for the double-precision CG and the reliable-update CG, on
grids large enough (n > 65536) that every threaded path runs.
"""
import numpy as np
import pytest

import femgen
import oracle


@pytest.fixture(scope="module")
def libs():
    return oracle.load(), oracle.load_threaded(4)


def _same(a, b):
    return (np.array_equal(a.x.view(np.uint64), b.x.view(np.uint64)) and a.iterations == b.iterations
            and a.restarts == b.restarts and a.status == b.status
            and np.float64(a.rel_res_true).tobytes() == np.float64(b.rel_res_true).tobytes())


def test_thread_counts(libs):
    one, many = libs
    assert oracle.threads(one) == 1
    assert oracle.threads(many) == 4


@pytest.mark.parametrize("grid,maxit", [((12, 13, 14), None), ((31, 31, 32), None), ((44, 43, 42), 300)])
@pytest.mark.parametrize("fmt", ["sym", "csr", "csc"])
def test_threaded_build_bitwise(libs, grid, maxit, fmt):
    one, many = libs
    s = femgen.build_system(femgen.Grid(*grid))
    arrs = {"sym": s.upper(), "csr": (s.ptr, s.idx, s.val), "csc": s.csc()}[fmt]
    tol = 1e-10 if maxit is None else 1e-30
    a = oracle.cg(fmt, *arrs, s.b, tol=tol, maxit=maxit, lib=one)
    b = oracle.cg(fmt, *arrs, s.b, tol=tol, maxit=maxit, lib=many)
    assert _same(a, b), (a.iterations, b.iterations)
    c = oracle.cg_ru(fmt, *arrs, s.b, tol=tol, maxit=maxit, lib=one)
    d = oracle.cg_ru(fmt, *arrs, s.b, tol=tol, maxit=maxit, lib=many)
    assert _same(c, d), (c.iterations, d.iterations)
    if maxit is not None:
        assert s.n > 65536 and c.restarts >= 1  # the threaded pairwise dot and an update ran


def test_threaded_build_from_nonzero_start(libs):
    one, many = libs
    s = femgen.build_system(femgen.Grid(10, 11, 12))
    up = s.upper()
    x0 = femgen.random_vector(s.n, 5)
    a = oracle.cg("sym", *up, s.b, x0=x0, tol=1e-12, lib=one)
    b = oracle.cg("sym", *up, s.b, x0=x0, tol=1e-12, lib=many)
    assert _same(a, b)
