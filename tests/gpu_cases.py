"""Seeded test matrices shared by the GPU parity tests (inputs only)."""
from __future__ import annotations

import functools

import numpy as np
import scipy.sparse as sp

import femgen


@functools.lru_cache(maxsize=None)
def fem(nx, ny, nz, n_incl=1, contrast=1000.0, seed_mesh=0, seed_x=1):
    return femgen.build_system(femgen.Grid(nx, ny, nz, n_incl=n_incl, contrast=contrast, seed_mesh=seed_mesh,
                                           seed_x=seed_x))


def random_general(n, m, density, seed, empty_rows=(), one_rows=(), long_rows=(), long_len=1000):
    """Random non-symmetric CSR with edge-case rows; returns (ptr, idx, val)."""
    rng = np.random.default_rng(seed)
    nnz_target = int(n * m * density)
    rows = rng.integers(0, n, nnz_target)
    cols = rng.integers(0, m, nnz_target)
    A = sp.coo_matrix((rng.uniform(-1, 1, nnz_target), (rows, cols)), shape=(n, m)).tocsr().tolil()
    for r in empty_rows:
        A[r, :] = 0
    for r in one_rows:
        A[r, :] = 0
        A[r, int(rng.integers(0, m))] = rng.uniform(-1, 1)
    for r in long_rows:
        c = rng.choice(m, size=min(long_len, m), replace=False)
        A[r, c] = rng.uniform(-1, 1, c.size)
    A = A.tocsr()
    A.eliminate_zeros()
    A.sort_indices()
    return A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64)


def random_spd(n, seed, density=0.02, dense_rows=()):
    """Random sparse SPD (diagonally dominant) matrix as full CSR arrays."""
    rng = np.random.default_rng(seed)
    k = max(1, int(n * n * density / 2))
    r = rng.integers(0, n, k)
    c = rng.integers(0, n, k)
    A = sp.coo_matrix((rng.uniform(-1, 1, k), (r, c)), shape=(n, n)).tocsr()
    A = A + A.T
    for d in dense_rows:
        cols = rng.choice(n, size=min(n, 300), replace=False)
        B = sp.coo_matrix((rng.uniform(-1, 1, cols.size), (np.full(cols.size, d), cols)), shape=(n, n)).tocsr()
        A = A + B + B.T
    A = A.tocsr()
    A.setdiag(0)
    A.eliminate_zeros()
    A = A + sp.diags(np.asarray(abs(A).sum(axis=1)).ravel() + 1.0)
    A = A.tocsr()
    A.sort_indices()
    return A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64)


def transpose_arrays(n, m, ptr, idx, val):
    """CSC arrays of the CSR matrix (ptr, idx, val) of shape (n, m)."""
    A = sp.csr_matrix((val, idx, ptr), shape=(n, m)).tocsc()
    A.sort_indices()
    return A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64)
