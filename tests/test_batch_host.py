"""Batched systems on the CPU: the generator's block-diagonal batches, the
oracle's per-instance batch solve pinned against whole-matrix and dense
solves, and the batch C ABI's input checks (no GPU work)."""
import ctypes

import numpy as np
import pytest

import femgen
import oracle
import paper_1010_4639_gb300 as gb
from paper_1010_4639_gb300 import _lib

SMALL = [femgen.Grid(5, 6, 7, seed_mesh=11, seed_x=12), femgen.Grid(3, 5, 5, seed_mesh=13, seed_x=14),
         femgen.Grid(7, 5, 6, contrast=50.0, seed_mesh=15, seed_x=16), femgen.Grid(4, 4, 4, seed_mesh=17, seed_x=18)]


@pytest.fixture(scope="module")
def batch():
    return femgen.build_batch(SMALL, nrhs=3)


def dense(ptr, idx, val, n):
    A = np.zeros((n, n))
    for i in range(n):
        A[i, idx[ptr[i]:ptr[i + 1]]] = val[ptr[i]:ptr[i + 1]]
    return A


def test_batch_is_block_diagonal_with_manufactured_rhs(batch):
    assert batch.count == 4
    assert batch.n == sum(femgen.size(g)[0] for g in SMALL)
    assert batch.row_off[2] - batch.row_off[1] == 9  # 3 x 5 x 5 nodes: one interior layer of 3 x 3
    for i in range(batch.count):
        r0, r1 = batch.row_off[i], batch.row_off[i + 1]
        cols = batch.idx[batch.ptr[r0]:batch.ptr[r1]]
        assert np.all((cols >= r0) & (cols < r1))
        p, j, v = batch.instance(i)
        s = femgen.build_system(SMALL[i])
        assert np.array_equal(p, s.ptr) and np.array_equal(j, s.idx) and np.array_equal(v, s.val)
        A = dense(p, j, v, r1 - r0)
        np.testing.assert_allclose(A @ batch.Xstar[r0:r1], batch.B[r0:r1], rtol=0, atol=1e-12)
    # the columns of X* are distinct seeded draws
    assert not np.allclose(batch.Xstar[:, 0], batch.Xstar[:, 1])


def test_oracle_batch_equals_the_whole_block_diagonal_solve(batch):
    # one CG on the block-diagonal matrix converges to the concatenation of the
    # per-instance solutions: pins the instance slicing of the batch oracle
    X, res = oracle.batch_solve(batch.row_off, batch.ptr, batch.idx, batch.val, batch.B, tol=1e-13,
                                precision="fp64", maxit=10 * batch.n)
    for k in range(batch.B.shape[1]):
        whole = oracle.cg("csr", batch.ptr, batch.idx, batch.val, batch.B[:, k], tol=1e-13, maxit=10 * batch.n)
        assert whole.status == "OK"
        assert np.linalg.norm(X[:, k] - whole.x) <= 1e-9 * np.linalg.norm(whole.x)
    for i in range(batch.count):
        r0, r1 = batch.row_off[i], batch.row_off[i + 1]
        for k in range(batch.B.shape[1]):
            assert res[i][k].status == "OK"
            if r1 > r0:
                A = dense(*batch.instance(i), r1 - r0)
                xd = np.linalg.solve(A, batch.B[r0:r1, k])
                assert np.linalg.norm(X[r0:r1, k] - xd) <= 1e-8 * np.linalg.norm(xd)


def test_oracle_batch_mixed_precision_reaches_tol(batch):
    X, res = oracle.batch_solve(batch.row_off, batch.ptr, batch.idx, batch.val, batch.B, tol=1e-10,
                                precision="fp32_ir", maxit=10 * batch.n)
    for i in range(batch.count):
        r0, r1 = batch.row_off[i], batch.row_off[i + 1]
        p, j, v = batch.instance(i)
        for k in range(batch.B.shape[1]):
            assert res[i][k].status == "OK"
            if r1 > r0:
                r = batch.B[r0:r1, k] - oracle.spmv("csr", p, j, v, X[r0:r1, k])
                assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(batch.B[r0:r1, k])
                assert res[i][k].restarts >= 2  # 1e-4 inner passes: at least three to reach 1e-10


@pytest.fixture(scope="module")
def lib():
    gb.build()
    return _lib.load()


def _create(lib, row_off, ptr, idx, val, nrhs=8):
    row_off = np.asarray(row_off, np.int64)
    ptr = np.asarray(ptr, np.int32)
    idx = np.asarray(idx, np.int32)
    val = np.asarray(val, np.float64)
    h = ctypes.c_void_p()
    rc = lib.gbcg_batch_create(ctypes.byref(h), len(row_off) - 1, ctypes.c_void_p(row_off.ctypes.data),
                               ctypes.c_void_p(ptr.ctypes.data), ctypes.c_void_p(idx.ctypes.data),
                               ctypes.c_void_p(val.ctypes.data), nrhs, _lib.GBCG_HOST, 0, None)
    return rc, lib.gbcg_last_error().decode()


@pytest.mark.parametrize("case", [
    ("column in another instance", [0, 1, 2], [0, 1, 2], [0, 0], [1.0, 1.0], 8, "outside instance"),
    ("unsorted columns", [0, 2], [0, 2, 3], [1, 0, 1], [1.0, 1.0, 1.0], 8, "strictly increasing"),
    ("decreasing row offsets", [0, 2, 1], [0, 1, 2], [0, 1], [1.0, 1.0], 8, "row_off"),
    ("nonzero first offset", [1, 2], [0, 1, 2], [0, 1], [1.0, 1.0], 8, "row_off[0]"),
    ("nan value", [0, 1], [0, 1], [0], [float("nan")], 8, "non-finite"),
    ("too many right-hand sides", [0, 1], [0, 1], [0], [1.0], 9, "nrhs"),
    ("no right-hand side", [0, 1], [0, 1], [0], [1.0], 0, "nrhs"),
    ("decreasing ptr", [0, 2], [0, 2, 1], [0, 1], [1.0, 1.0], 8, "ptr"),
])
def test_batch_create_rejects_malformed_input(lib, case):
    _, row_off, ptr, idx, val, nrhs, needle = case
    rc, msg = _create(lib, row_off, ptr, idx, val, nrhs)
    assert rc == 1, (rc, msg)
    assert needle in msg


def test_batch_calls_reject_null_handles(lib):
    assert lib.gbcg_batch_solve(None, None, None, 1e-10, 0, None, None, None, None) == 1
    assert lib.gbcg_batch_autotune(None, 1, None, None) == 1
    assert lib.gbcg_batch_set_tuning(None, 1, None) == 1
    assert lib.gbcg_batch_destroy(None) == 0
