"""Pins of the CPU oracle against facts that do not come from the oracle.

Every ``check_*`` function takes a loaded oracle library and raises
AssertionError when the oracle disagrees with what the paper or the
mathematics fixes.  ``test_oracle_pins.py`` runs them on the real oracle and
``test_oracle_mutants.py`` runs them on deliberately broken copies to show
that a plausible mistake (a dropped term, a wrong sign or index, a transposed
operand) is caught.

Sources of truth used here: dense brute-force products (numpy), dense
Cholesky solves (scipy), exact rational arithmetic (fractions), the
finite-termination and A-orthogonality properties of CG in exact arithmetic,
the monotone decrease of the A-norm of the error, and closed-form systems.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

import femgen
import oracle


# ----------------------------------------------------------------- inputs --
def random_csr(n, m, density, seed, empty_rows=(), long_row=None, long_len=0):
    """Random (non-symmetric) sparse matrix with sorted columns, as CSR arrays."""
    rng = np.random.default_rng(seed)
    dense = np.where(rng.random((n, m)) < density, rng.uniform(-1, 1, (n, m)), 0.0)
    for r in empty_rows:
        dense[r, :] = 0.0
    if long_row is not None:
        cols = rng.choice(m, size=min(long_len, m), replace=False)
        dense[long_row, cols] = rng.uniform(-1, 1, cols.size)
    A = sp.csr_matrix(dense)
    A.sort_indices()
    return A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64), dense


def spd_sparse(n, seed, density=0.2, shift=1.0):
    """Random sparse SPD matrix M M' + shift I, returned as (csr arrays, dense)."""
    rng = np.random.default_rng(seed)
    M = np.where(rng.random((n, n)) < density, rng.uniform(-1, 1, (n, n)), 0.0)
    A = M @ M.T + shift * np.eye(n)
    A = 0.5 * (A + A.T)
    S = sp.csr_matrix(A)
    S.sort_indices()
    return (S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64)), A


def fem_small(nx=8, ny=7, nz=9, **kw):
    return femgen.build_system(femgen.Grid(nx, ny, nz, **kw))


def dense_of(ptr, idx, val, n, m=None):
    m = n if m is None else m
    D = np.zeros((n, m))
    for i in range(n):
        for k in range(ptr[i], ptr[i + 1]):
            D[i, idx[k]] += val[k]
    return D


def componentwise(y, yref, scale, bound):
    err = np.abs(y - yref)
    lim = bound * scale + 1e-300
    assert np.all(err <= lim), f"max componentwise error {np.max(err / lim) * bound:.3e} > {bound}"


# ------------------------------------------------------------- products ----
def check_spmv_csr_bruteforce(lib):
    for seed, (n, m) in enumerate([(1, 1), (37, 37), (64, 50), (200, 200)]):
        ptr, idx, val, dense = random_csr(n, m, 0.1, seed, empty_rows=(0,) if n > 1 else (),
                                          long_row=n // 2, long_len=min(m, 40))
        x = np.random.default_rng(100 + seed).uniform(-1, 1, m)
        y = np.empty(n)
        lib.orc_spmv_csr(n, ptr.ctypes.data, idx.ctypes.data, val.ctypes.data, x.ctypes.data, y.ctypes.data)
        componentwise(y, dense @ x, np.abs(dense) @ np.abs(x), 1e-14)


def check_spmv_csc_bruteforce(lib):
    # CSC arrays of a non-symmetric A are the CSR arrays of A'.
    for seed, n in enumerate([1, 33, 150]):
        ptr, idx, val, denseT = random_csr(n, n, 0.12, 50 + seed, long_row=n - 1, long_len=n)
        dense = denseT.T
        x = np.random.default_rng(7 + seed).uniform(-1, 1, n)
        y = oracle.spmv("csc", ptr, idx, val, x, lib=lib)
        componentwise(y, dense @ x, np.abs(dense) @ np.abs(x), 1e-14)


def check_spmv_sym_bruteforce(lib):
    # Upper-triangle storage of a symmetric A (A = L + D + U, U' = L).
    for seed, n in enumerate([1, 2, 45, 160]):
        (ptr, idx, val), A = spd_sparse(n, 300 + seed, density=0.08)
        uptr, uidx, uval = femgen.upper(n, ptr, idx, val)
        x = np.random.default_rng(seed).uniform(-1, 1, n)
        y = oracle.spmv("sym", uptr, uidx, uval, x, lib=lib)
        componentwise(y, A @ x, np.abs(A) @ np.abs(x), 1e-14)
    s = fem_small(9, 8, 7)
    D = dense_of(s.ptr, s.idx, s.val, s.n)
    x = np.random.default_rng(3).uniform(-1, 1, s.n)
    uptr, uidx, uval = s.upper()
    for fmt, arrs in (("sym", (uptr, uidx, uval)), ("csr", (s.ptr, s.idx, s.val)), ("csc", s.csc())):
        y = oracle.spmv(fmt, *arrs, x, lib=lib)
        componentwise(y, D @ x, np.abs(D) @ np.abs(x), 1e-14)


def check_abs_spmv(lib):
    ptr, idx, val, dense = random_csr(40, 40, 0.2, 9)
    x = np.random.default_rng(1).uniform(-1, 1, 40)
    y = oracle.abs_spmv("csr", ptr, idx, val, x, lib=lib)
    assert np.allclose(y, np.abs(dense) @ np.abs(x), rtol=1e-14, atol=0)
    (ptr, idx, val), A = spd_sparse(30, 4)
    u = femgen.upper(30, ptr, idx, val)
    y = oracle.abs_spmv("sym", *u, x[:30], lib=lib)
    assert np.allclose(y, np.abs(A) @ np.abs(x[:30]), rtol=1e-14, atol=0)


def check_spmv_f32(lib):
    ptr, idx, val, dense = random_csr(80, 80, 0.1, 12)
    x = np.random.default_rng(2).uniform(-1, 1, 80).astype(np.float32)
    v32 = val.astype(np.float32)
    D32 = dense_of(ptr, idx, v32.astype(np.float64), 80)
    y = oracle.spmv_f32("csr", ptr, idx, v32, x, lib=lib).astype(np.float64)
    componentwise(y, D32 @ x.astype(np.float64), np.abs(D32) @ np.abs(x.astype(np.float64)), 1e-5)
    (p2, i2, v2), A = spd_sparse(60, 13, density=0.1)
    u = femgen.upper(60, p2, i2, v2)
    u32 = u[2].astype(np.float32)
    Au = dense_of(u[0], u[1], u32.astype(np.float64), 60)
    As = Au + np.triu(Au, 1).T
    xs = x[:60]
    y = oracle.spmv_f32("sym", u[0], u[1], u32, xs, lib=lib).astype(np.float64)
    componentwise(y, As @ xs.astype(np.float64), np.abs(As) @ np.abs(xs.astype(np.float64)), 1e-5)


def check_dot(lib):
    rng = np.random.default_rng(5)
    a = rng.uniform(-1, 1, 300)
    b = rng.uniform(-1, 1, 300)
    exact = sum(Fraction(float(u)) * Fraction(float(v)) for u, v in zip(a, b))
    assert abs(oracle.dot_long(a, b, lib=lib) - float(exact)) <= 1e-15 * float(np.abs(a) @ np.abs(b))
    assert abs(oracle.dot(a, b, lib=lib) - float(exact)) <= 300 * 1.2e-16 * float(np.abs(a) @ np.abs(b))


def check_dot_f32(lib):
    # the exact sum (rational arithmetic on the float inputs) within the
    # pairwise-summation bound (log2(n) + 8) u sum |a_i b_i|, u = 2^-24
    rng = np.random.default_rng(6)
    for n in (1, 7, 9, 300, 3001):
        a = rng.uniform(-1, 1, n).astype(np.float32)
        b = rng.uniform(-1, 1, n).astype(np.float32)
        exact = sum(Fraction(float(u)) * Fraction(float(v)) for u, v in zip(a, b))
        bound = (np.log2(n) + 8) * 2.0 ** -24 * float(np.abs(a.astype(np.float64)) @ np.abs(b.astype(np.float64)))
        assert abs(oracle.dot_f32(a, b, lib=lib) - float(exact)) <= bound, n
    # 2^20 copies of 0.1f: a left-to-right float sum drifts by about 1e-2
    # relative, the tree order stays within its log2(n) bound
    n = 1 << 20
    a = np.full(n, 0.1, dtype=np.float32)
    ones = np.ones(n, dtype=np.float32)
    exact = n * float(np.float32(0.1))
    assert abs(oracle.dot_f32(a, ones, lib=lib) - exact) <= (20 + 8) * 2.0 ** -24 * exact


# ---------------------------------------------------------------- CG -------
def check_cg_vs_cholesky(lib):
    for seed, n in enumerate([1, 3, 10, 25, 40]):
        (ptr, idx, val), A = spd_sparse(n, 10 + seed, density=0.3, shift=2.0)
        b = np.random.default_rng(seed).uniform(-1, 1, n)
        xc = sla.cho_solve(sla.cho_factor(A), b)
        for fmt, arrs in (("csr", (ptr, idx, val)), ("sym", femgen.upper(n, ptr, idx, val)),
                          ("csc", (ptr, idx, val))):
            r = oracle.cg(fmt, *arrs, b, tol=1e-14, maxit=10 * n + 10, lib=lib)
            assert r.status == "OK", r.status
            assert np.linalg.norm(r.x - xc) <= 1e-12 * np.linalg.norm(xc), (fmt, n)
            assert r.rel_res_true <= 1e-14


def check_cg_fem_vs_cholesky(lib):
    s = fem_small(7, 8, 6, contrast=1000.0)
    D = dense_of(s.ptr, s.idx, s.val, s.n)
    xc = sla.cho_solve(sla.cho_factor(D), s.b)
    r = oracle.cg("sym", *s.upper(), s.b, tol=1e-13, maxit=20 * s.n, lib=lib)
    assert r.status == "OK"
    assert np.linalg.norm(r.x - xc) / np.linalg.norm(xc) <= 1e-9
    # x* is the manufactured solution: b was assembled element by element from it
    assert np.linalg.norm(r.x - s.xstar) / np.linalg.norm(s.xstar) <= 1e-9


def check_cg_finite_termination(lib):
    # k distinct eigenvalues -> the exact solution after at most k steps.
    rng = np.random.default_rng(21)
    n = 60
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    eig = np.repeat([1.0, 2.0, 5.0, 9.0], n // 4)
    A = (Q * eig) @ Q.T
    A = 0.5 * (A + A.T)
    S = sp.csr_matrix(A)
    b = rng.uniform(-1, 1, n)
    r = oracle.cg("csr", S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data, b, tol=1e-11, lib=lib)
    assert r.status == "OK" and r.iterations <= 4, r.iterations
    # diagonal with 3 distinct values: exactly 3 steps
    d = np.repeat([3.0, 0.5, 7.0], 7)
    ptr = np.arange(22, dtype=np.int32)
    idx = np.arange(21, dtype=np.int32)
    bb = np.random.default_rng(2).uniform(0.5, 1.0, 21)
    r = oracle.cg("csr", ptr, idx, d, bb, tol=1e-13, lib=lib)
    assert r.status == "OK" and r.iterations == 3, r.iterations
    assert np.allclose(r.x, bb / d, rtol=1e-13, atol=0)
    # well-conditioned n = 12: at most n steps
    (p2, i2, v2), A2 = spd_sparse(12, 77, density=0.5, shift=3.0)
    r = oracle.cg("csr", p2, i2, v2, np.ones(12), tol=1e-12, lib=lib)
    assert r.status == "OK" and r.iterations <= 12


def check_cg_exact_first_steps(lib):
    # Exact rational CG on a 3x3 system: in exact arithmetic it terminates in
    # 3 steps; the floating-point iterates must follow the rational ones.
    A = [[Fraction(4), Fraction(1), Fraction(0)], [Fraction(1), Fraction(3), Fraction(1)],
         [Fraction(0), Fraction(1), Fraction(2)]]
    b = [Fraction(1), Fraction(2), Fraction(3)]

    def mv(M, v):
        return [sum(M[i][j] * v[j] for j in range(3)) for i in range(3)]

    def dt(u, v):
        return sum(a * c for a, c in zip(u, v))

    x = [Fraction(0)] * 3
    r = list(b)
    p = list(r)
    xs = []
    for _ in range(3):
        q = mv(A, p)
        a = dt(r, r) / dt(p, q)
        x = [xi + a * pi for xi, pi in zip(x, p)]
        rn = [ri - a * qi for ri, qi in zip(r, q)]
        be = dt(rn, rn) / dt(r, r)
        p = [ri + be * pi for ri, pi in zip(rn, p)]
        r = rn
        xs.append([float(v) for v in x])
    assert all(v == 0 for v in r)  # exact termination
    Ad = np.array([[float(v) for v in row] for row in A])
    S = sp.csr_matrix(Ad)
    res = oracle.cg("csr", S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data,
                    np.array([1.0, 2.0, 3.0]), tol=1e-15, maxit=3, history=3, lib=lib)
    assert res.iterations == 3
    for k in range(3):
        assert np.allclose(res.x_hist[k], xs[k], rtol=1e-13, atol=1e-15), k


def check_cg_a_orthogonality(lib):
    s = fem_small(10, 10, 10, contrast=10.0)
    D = dense_of(s.ptr, s.idx, s.val, s.n)
    r = oracle.cg("csr", s.ptr, s.idx, s.val, s.b, tol=1e-10, history=40, lib=lib)
    P = r.p_hist
    AP = P @ D
    G = AP @ P.T
    nrm = np.sqrt(np.diag(G))
    for i in range(P.shape[0]):
        for j in range(max(0, i - 2), i):
            assert abs(G[i, j]) / (nrm[i] * nrm[j]) <= 1e-8, (i, j, G[i, j] / (nrm[i] * nrm[j]))


def check_cg_error_a_norm_decreases(lib):
    s = fem_small(9, 9, 9, contrast=100.0)
    D = dense_of(s.ptr, s.idx, s.val, s.n)
    xe = sla.cho_solve(sla.cho_factor(D), s.b)
    r = oracle.cg("sym", *s.upper(), s.b, tol=1e-12, maxit=20 * s.n, history=2000, lib=lib)
    E = r.x_hist - xe
    en = np.sqrt(np.einsum("ki,ij,kj->k", E, D, E))
    e0 = np.sqrt(xe @ D @ xe)
    prev = e0
    for k, e in enumerate(en):
        assert e <= prev * (1 + 1e-9) + 1e-13 * e0, (k, e, prev)
        prev = e
    assert en[-1] <= 1e-9 * e0


def check_cg_tridiagonal_closed_form(lib):
    # -u'' = f on a uniform grid: tridiag(-1, 2, -1) x = b with x known.
    n = 50
    ptr = [0]
    idx, val = [], []
    for i in range(n):
        for j, v in ((i - 1, -1.0), (i, 2.0), (i + 1, -1.0)):
            if 0 <= j < n:
                idx.append(j)
                val.append(v)
        ptr.append(len(idx))
    ptr, idx, val = np.array(ptr, np.int32), np.array(idx, np.int32), np.array(val)
    t = np.arange(1, n + 1) / (n + 1)
    xs = np.sin(np.pi * t) + t ** 2
    b = 2 * xs - np.r_[xs[1:], 0.0] - np.r_[0.0, xs[:-1]]
    r = oracle.cg("csr", ptr, idx, val, b, tol=1e-13, lib=lib)
    assert r.status == "OK" and r.iterations <= n
    assert np.linalg.norm(r.x - xs) <= 1e-10 * np.linalg.norm(xs)
    # the eigenvalues of tridiag(-1,2,-1) are distinct: n steps suffice and
    # fewer than n cannot reach 1e-13 from a generic right-hand side
    assert r.iterations >= n // 2


def check_cg_edge_cases(lib):
    (ptr, idx, val), A = spd_sparse(20, 5, shift=1.0)
    b = np.random.default_rng(0).uniform(-1, 1, 20)
    r = oracle.cg("csr", ptr, idx, val, np.zeros(20), x0=np.ones(20), lib=lib)   # b = 0 -> x = 0
    assert r.status == "OK" and r.iterations == 0 and not np.any(r.x)
    xe = np.linalg.solve(A, b)
    r = oracle.cg("csr", ptr, idx, val, A @ np.ones(20), x0=np.ones(20), tol=1e-10, lib=lib)
    assert r.status == "OK" and r.iterations == 0                                  # x0 already solves it
    r = oracle.cg("csr", ptr, idx, val, b, tol=1e-30, maxit=3, lib=lib)
    assert r.status == "MAXIT" and r.iterations == 3
    neg = -val
    r = oracle.cg("csr", ptr, idx, neg, b, lib=lib)
    assert r.status == "NOT_SPD" and r.iterations == 0
    bad = val.copy()
    bad[0] = np.nan
    r = oracle.cg("csr", ptr, idx, bad, b, lib=lib)
    assert r.status == "NONFINITE"
    r = oracle.cg("csr", ptr, idx, val, b, tol=1e-12, lib=lib)
    assert np.linalg.norm(r.x - xe) <= 1e-10 * np.linalg.norm(xe)


# ------------------------------------------------------ pipelined CG ---
def check_pipelined_equals_cg_iterates(lib):
    # in exact arithmetic the single-reduction recurrences give the iterates
    # and step lengths of the Section III listing; on well-conditioned
    # systems the two agree to rounding over the first steps
    for seed, n in ((3, 30), (4, 45)):
        (ptr, idx, val), A = spd_sparse(n, 30 + seed, density=0.3, shift=3.0)
        b = np.random.default_rng(seed).uniform(-1, 1, n)
        a = oracle.cg("csr", ptr, idx, val, b, tol=0.0, maxit=8, history=8, lib=lib)
        q = oracle.cg("csr", ptr, idx, val, b, tol=0.0, maxit=8, history=8, lib=lib, pipelined=True)
        assert a.x_hist.shape == q.x_hist.shape == (8, n)
        np.testing.assert_allclose(q.x_hist, a.x_hist, rtol=0, atol=1e-11 * np.abs(a.x_hist).max())
        np.testing.assert_allclose(q.alpha, a.alpha, rtol=1e-10)
        np.testing.assert_allclose(q.beta[1:], a.beta[:-1], rtol=1e-9)   # beta of step k+1 pairs with CG's step k


def check_pipelined_vs_cholesky_and_edges(lib):
    for seed, n in enumerate([1, 3, 10, 25, 40]):
        (ptr, idx, val), A = spd_sparse(n, 10 + seed, density=0.3, shift=2.0)
        b = np.random.default_rng(seed).uniform(-1, 1, n)
        xc = sla.cho_solve(sla.cho_factor(A), b)
        for fmt, arrs in (("csr", (ptr, idx, val)), ("sym", femgen.upper(n, ptr, idx, val))):
            r = oracle.cg(fmt, *arrs, b, tol=1e-13, maxit=10 * n + 10, lib=lib, pipelined=True)
            assert r.status == "OK", (fmt, n, r.status)
            assert np.linalg.norm(r.x - xc) <= 1e-11 * np.linalg.norm(xc), (fmt, n)
    s = fem_small(7, 8, 6, contrast=1000.0)
    D = dense_of(s.ptr, s.idx, s.val, s.n)
    xc = sla.cho_solve(sla.cho_factor(D), s.b)
    r = oracle.cg("csr", s.ptr, s.idx, s.val, s.b, tol=1e-12, maxit=20 * s.n, lib=lib, pipelined=True)
    assert r.status == "OK" and r.rel_res_true <= 1e-12
    assert np.linalg.norm(r.x - xc) / np.linalg.norm(xc) <= 1e-8
    # diagonal with 3 distinct values: exactly 3 steps
    d = np.repeat([3.0, 0.5, 7.0], 7)
    ptr = np.arange(22, dtype=np.int32)
    idx = np.arange(21, dtype=np.int32)
    bb = np.random.default_rng(2).uniform(0.5, 1.0, 21)
    r = oracle.cg("csr", ptr, idx, d, bb, tol=1e-13, lib=lib, pipelined=True)
    assert r.status == "OK" and r.iterations == 3, r.iterations
    assert np.allclose(r.x, bb / d, rtol=1e-12, atol=0)
    (ptr, idx, val), A = spd_sparse(20, 5, shift=1.0)
    b = np.random.default_rng(0).uniform(-1, 1, 20)
    r = oracle.cg("csr", ptr, idx, val, np.zeros(20), x0=np.ones(20), lib=lib, pipelined=True)
    assert r.status == "OK" and r.iterations == 0 and not np.any(r.x)
    r = oracle.cg("csr", ptr, idx, val, b, tol=1e-30, maxit=3, lib=lib, pipelined=True)
    assert r.status == "MAXIT" and r.iterations == 3
    r = oracle.cg("csr", ptr, idx, -val, b, lib=lib, pipelined=True)
    assert r.status == "NOT_SPD" and r.iterations == 0


def check_cg_f32(lib):
    s = fem_small(8, 8, 8, contrast=10.0)
    u = s.upper()
    rhs = (s.b / np.linalg.norm(s.b)).astype(np.float32)
    d, it, bd = oracle.cg_f32("sym", u[0], u[1], u[2].astype(np.float32), rhs, 1e-4, 1000, lib=lib)
    assert not bd and it > 0
    D = dense_of(s.ptr, s.idx, s.val, s.n)
    res = np.linalg.norm(rhs.astype(np.float64) - D @ d.astype(np.float64))
    assert res <= 2e-4, res
    xe = np.linalg.solve(D, rhs.astype(np.float64))
    assert np.linalg.norm(d - xe) / np.linalg.norm(xe) <= 1e-2


def check_cg_ir(lib):
    s = fem_small(10, 9, 11, contrast=1000.0)
    D = dense_of(s.ptr, s.idx, s.val, s.n)
    xe = sla.cho_solve(sla.cho_factor(D), s.b)
    for fmt, arrs in (("csr", (s.ptr, s.idx, s.val)), ("sym", s.upper())):
        r = oracle.cg_ir(fmt, *arrs, s.b, tol=1e-10, inner_tol=1e-4, lib=lib)
        assert r.status == "OK", r.status
        true = np.linalg.norm(s.b - D @ r.x) / np.linalg.norm(s.b)
        assert true <= 1e-10 and abs(true - r.rel_res_true) <= 1e-3 * true + 1e-16
        assert np.linalg.norm(r.x - xe) / np.linalg.norm(xe) <= 1e-7
        assert 2 <= r.restarts <= 10


def check_cg_ru(lib):
    # single-precision iterations with double-precision reliable updates reach
    # double-precision accuracy: dense Cholesky at 1e-12, the manufactured x*
    s = fem_small(7, 8, 6, contrast=1000.0)
    D = dense_of(s.ptr, s.idx, s.val, s.n)
    xc = sla.cho_solve(sla.cho_factor(D), s.b)
    for fmt, arrs in (("csr", (s.ptr, s.idx, s.val)), ("sym", s.upper())):
        r = oracle.cg_ru(fmt, *arrs, s.b, tol=1e-12, maxit=40 * s.n, lib=lib)
        assert r.status == "OK" and r.rel_res_true <= 1e-12, (fmt, r.status, r.rel_res_true)
        assert np.linalg.norm(r.x - xc) / np.linalg.norm(xc) <= 1e-9
        true = np.linalg.norm(s.b - D @ r.x) / np.linalg.norm(s.b)
        assert true <= 1.01e-12
    # the Krylov space is kept: about the double-precision iteration count
    # (the refinement that restarts it needs ~50% more)
    s = fem_small(17, 15, 19)
    f = oracle.cg("csr", s.ptr, s.idx, s.val, s.b, tol=1e-10, maxit=40 * s.n, lib=lib)
    r = oracle.cg_ru("csr", s.ptr, s.idx, s.val, s.b, tol=1e-10, maxit=40 * s.n, lib=lib)
    assert r.status == "OK" and r.iterations <= 1.2 * f.iterations + 5, (r.iterations, f.iterations)
    # an update each time the recurrence residual has fallen by delta = 0.1
    # since the last one: about one per decade from ||r0|| to 1e-10 ||b||
    # (x0 = 0, so ||r0|| = ||b||), plus the confirming one
    assert 8 <= r.restarts <= 14, r.restarts
    # three distinct eigenvalues, exact in float: three steps, then updates
    d = np.repeat([2.0, 0.5, 4.0], 5)
    ptr = np.arange(16, dtype=np.int32)
    idx = np.arange(15, dtype=np.int32)
    bb = np.tile([1.0, 2.0, 3.0, -1.0, 5.0], 3)
    r = oracle.cg_ru("csr", ptr, idx, d, bb, tol=1e-14, lib=lib)
    assert r.status == "OK" and r.iterations <= 9, r.iterations
    np.testing.assert_allclose(r.x, bb / d, rtol=1e-13)  # cond 8 x residual 1e-14
    # edge cases
    (ptr, idx, val), A = spd_sparse(20, 5, shift=1.0)
    b = np.random.default_rng(0).uniform(-1, 1, 20)
    r = oracle.cg_ru("csr", ptr, idx, val, np.zeros(20), x0=np.ones(20), lib=lib)
    assert r.status == "OK" and r.iterations == 0 and not np.any(r.x)
    r = oracle.cg_ru("csr", ptr, idx, -val, b, lib=lib)
    assert r.status == "NOT_SPD" and r.iterations == 0
    r = oracle.cg_ru("csr", ptr, idx, val, b, tol=1e-30, maxit=3, lib=lib)
    assert r.status == "MAXIT" and r.iterations == 3


# ------------------------------------------------------- differentiation ---
def _diff_case(g):
    s = femgen.build_system(g)
    el = femgen.elements(g)
    xt = femgen.random_vector(s.n, 77)
    return s, el, xt


def _dense(ptr, idx, val, n):
    A = np.zeros((n, n))
    for i in range(n):
        A[i, idx[ptr[i]:ptr[i + 1]]] = val[ptr[i]:ptr[i + 1]]
    return A


def check_grad_dense_reference(lib):
    # L = ||x - xt||^2, A x = b: dense solves give lambda = A^-1 2(x - xt) and
    # the full dL/dA = -lambda x'; every stored form must be that matrix (or its
    # symmetric fold) at the stored positions, dL/db = lambda, and the element
    # gradient the sum of Kh_e against dL/dA over the element's unknowns
    g = femgen.Grid(6, 6, 6, contrast=30.0, seed_mesh=5, seed_x=6)
    s, el, xt = _diff_case(g)
    A = _dense(s.ptr, s.idx, s.val, s.n)
    x = np.linalg.solve(A, s.b)
    lam = np.linalg.solve(A, 2.0 * (x - xt))
    GA = -np.outer(lam, x)
    rows = np.repeat(np.arange(s.n), np.diff(s.ptr))
    g_csr = oracle.grad_values("csr", s.ptr, s.idx, lam, x, lib=lib)
    np.testing.assert_allclose(g_csr, GA[rows, s.idx], rtol=1e-13, atol=1e-13 * np.abs(GA).max())
    g_csc = oracle.grad_values("csc", s.ptr, s.idx, lam, x, lib=lib)  # columns of A (= rows: symmetric)
    np.testing.assert_allclose(g_csc, GA[s.idx, rows], rtol=1e-13, atol=1e-13 * np.abs(GA).max())
    up, ui, uv = s.upper()
    urows = np.repeat(np.arange(s.n), np.diff(up))
    fold = np.where(urows == ui, GA[urows, ui], GA[urows, ui] + GA[ui, urows])
    g_sym = oracle.grad_values("sym", up, ui, lam, x, lib=lib)
    np.testing.assert_allclose(g_sym, fold, rtol=1e-13, atol=1e-13 * np.abs(GA).max())
    # element gradient: sum_ab Kh_ab GA[u_a, u_b] over unknown vertices
    nodes = el.nodes
    ok = nodes >= 0
    safe = np.where(ok, nodes, 0)
    Gsub = GA[safe[:, :, None], safe[:, None, :]] * (ok[:, :, None] & ok[:, None, :])
    gc_ref = np.einsum("eab,eab->e", el.kh, Gsub)
    for storage, (pp, ii, gv) in (("csr", (s.ptr, s.idx, g_csr)), ("sym", (up, ui, g_sym))):
        pos, w = femgen.element_map(el, pp, ii, storage=storage)
        gc = oracle.element_grad(pos, w, gv, lib=lib)
        np.testing.assert_allclose(gc, gc_ref, rtol=1e-10, atol=1e-12 * np.abs(gc_ref).max())


def check_assemble_reproduces_the_generator(lib):
    g = femgen.Grid(7, 6, 5, contrast=100.0, seed_mesh=8, seed_x=9)
    s, el, _ = _diff_case(g)
    for storage, (pp, ii, vv) in (("csr", (s.ptr, s.idx, s.val)), ("sym", s.upper())):
        pos, w = femgen.element_map(el, pp, ii, storage=storage)
        tptr, te, tw = femgen.assembly_map(pos, w, len(ii))
        val = oracle.assemble(tptr, te, tw, el.coef, lib=lib)
        np.testing.assert_allclose(val, vv, rtol=1e-12, atol=1e-13 * np.abs(vv).max())


def check_grad_finite_differences(lib):
    # central differences of L through the oracle's own solves (to 1e-14),
    # step 1e-6, along random directions in b, in the stored upper values
    # (a symmetric perturbation of A) and in the element coefficients
    g = femgen.Grid(6, 6, 7, contrast=20.0, seed_mesh=3, seed_x=4)
    s, el, xt = _diff_case(g)
    up, ui, uv = s.upper()
    pos, w = femgen.element_map(el, up, ui, storage="sym")
    tptr, te, tw = femgen.assembly_map(pos, w, len(ui))
    coef = el.coef.copy()
    val = oracle.assemble(tptr, te, tw, coef, lib=lib)
    L, x, lam, gb, gv = oracle.loss_gradients("sym", up, ui, val, s.b, xt, tol=1e-14, lib=lib)
    gc = oracle.element_grad(pos, w, gv, lib=lib)

    def loss(v, b):
        r = oracle.cg("sym", up, ui, v, b, tol=1e-14, maxit=40 * s.n, lib=lib)
        return float(np.dot(r.x - xt, r.x - xt))

    rng = np.random.default_rng(11)
    h = 1e-6
    for _ in range(3):
        d = rng.standard_normal(s.n)
        fd = (loss(val, s.b + h * d) - loss(val, s.b - h * d)) / (2 * h)
        assert abs(fd - gb @ d) <= 1e-6 * abs(fd) + 1e-9, ("b", fd, gb @ d)
        dv = rng.standard_normal(len(ui)) * np.abs(val)
        fd = (loss(val + h * dv, s.b) - loss(val - h * dv, s.b)) / (2 * h)
        assert abs(fd - gv @ dv) <= 1e-5 * abs(fd) + 1e-9, ("values", fd, gv @ dv)
        dc = rng.standard_normal(coef.shape[0]) * coef
        vp = oracle.assemble(tptr, te, tw, coef + h * dc, lib=lib)
        vm = oracle.assemble(tptr, te, tw, coef - h * dc, lib=lib)
        fd = (loss(vp, s.b) - loss(vm, s.b)) / (2 * h)
        assert abs(fd - gc @ dc) <= 1e-5 * abs(fd) + 1e-9, ("coefficients", fd, gc @ dc)


def check_lanczos_extremes(lib):
    """The Ritz values from the CG step lengths (oracle.lanczos_extremes) are
    the extreme eigenvalues of A, to the accuracy of a converged run: against
    numpy's dense symmetric eigensolver on a FEM grid and on a random SPD
    matrix, and exactly (in exact arithmetic) on a diagonal with known
    spectrum."""
    import oracle

    fem = fem_small(9, 8, 7)
    (sp_ptr, sp_idx, sp_val), _ = spd_sparse(60, 4)
    for ptr, idx, val, sym in (fem.upper() + (True,), (sp_ptr, sp_idx, sp_val, False)):
        n = len(ptr) - 1
        fmt = "sym" if sym else "csr"
        A = dense_of(ptr, idx, val, n)
        if sym:
            A = A + np.triu(A, 1).T
        b = np.random.default_rng(2).uniform(-1, 1, n)
        r = oracle.cg(fmt, ptr, idx, val, b, tol=1e-13, maxit=20 * n, scalar_history=20 * n, lib=lib)
        lo, hi = oracle.lanczos_extremes(r.alpha, r.beta)
        w = np.linalg.eigvalsh(A)
        # Ritz values lie inside the spectrum ...
        assert lo >= w[0] * (1 - 1e-12) and hi <= w[-1] * (1 + 1e-12), (lo, w[0], hi, w[-1])
        # ... and a run to 1e-13 has found the ends: to 1e-6 on the FEM grid
        # (well separated ends), to 1% on the random matrix (whose smallest
        # eigenvalues cluster at the shift, where the run stops first)
        rt = 1e-6 if sym else 1e-2
        assert abs(lo - w[0]) <= rt * w[0] and abs(hi - w[-1]) <= rt * w[-1], (lo, w[0], hi, w[-1])
    # diag(1, 2, ..., 10): CG terminates in 10 steps, T_10 has exactly A's spectrum
    n = 10
    ptr, idx, val = np.arange(n + 1), np.arange(n), np.arange(1.0, n + 1)
    r = oracle.cg("csr", ptr, idx, val, np.ones(n), tol=1e-15, maxit=n, scalar_history=n, lib=lib)
    lo, hi = oracle.lanczos_extremes(r.alpha, r.beta)
    assert abs(lo - 1.0) < 1e-10 and abs(hi - 10.0) < 1e-9, (lo, hi)


ALL_CHECKS = [
    check_spmv_csr_bruteforce, check_spmv_csc_bruteforce, check_spmv_sym_bruteforce, check_abs_spmv,
    check_spmv_f32, check_dot, check_dot_f32, check_cg_vs_cholesky, check_cg_fem_vs_cholesky,
    check_cg_finite_termination, check_cg_exact_first_steps, check_cg_a_orthogonality,
    check_cg_error_a_norm_decreases, check_cg_tridiagonal_closed_form, check_cg_edge_cases,
    check_cg_f32, check_cg_ir, check_cg_ru, check_grad_dense_reference, check_assemble_reproduces_the_generator,
    check_grad_finite_differences, check_pipelined_equals_cg_iterates, check_pipelined_vs_cholesky_and_edges,
    check_lanczos_extremes,
]
