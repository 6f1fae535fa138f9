"""The synthetic FEM input generator against closed forms and FEM invariants."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import femgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_table1.json")

# the 7 positive offsets of the Kuhn pattern (the other 7 are their negatives)
POS_OFFSETS = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]


def analytic_counts(nx, ny, nz, dirichlet=True):
    m = np.array([nx, ny, nz]) - (2 if dirichlet else 0)
    n = int(np.prod(m))
    off = sum(int(np.prod(m - np.array(o))) for o in POS_OFFSETS)
    return n, n + 2 * off, n + off   # rows, full nnz, stored upper-triangle nnz


@pytest.mark.parametrize("dims", [(3, 3, 3), (4, 5, 6), (12, 12, 12), (31, 31, 32), (17, 9, 40)])
def test_counts_match_closed_form(dims):
    g = femgen.Grid(*dims)
    s = femgen.build_system(g)
    n, nnz, nnz_u = analytic_counts(*dims)
    assert (s.n, s.nnz) == (n, nnz)
    assert int(s.upper()[0][-1]) == nnz_u


def test_large_sizes_closed_form():
    assert femgen.size(femgen.LARGE) == analytic_counts(128, 128, 128)[:2] == (2000376, 29626126)
    assert analytic_counts(256, 256, 256) == (16387064, 244260622, 130323843)
    assert analytic_counts(31, 31, 32) == (25230, 358152, 191691)


def test_structure_and_symmetry():
    s = femgen.build_system(femgen.Grid(9, 10, 11, contrast=1000.0))
    A = sp.csr_matrix((s.val, s.idx, s.ptr), shape=(s.n, s.n))
    assert (A != A.T).nnz == 0                   # exact symmetry (row-centric assembly)
    assert np.all(A.diagonal() > 0)
    for i in range(s.n):                          # sorted, unique columns
        c = s.idx[s.ptr[i]:s.ptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    np.linalg.cholesky(A.toarray())               # SPD after Dirichlet elimination
    rel = np.abs(A @ s.xstar - s.b) / (np.abs(A) @ np.abs(s.xstar))
    assert rel.max() <= 1e-14                     # b = A x*, assembled element by element


def test_neumann_row_sums_vanish():
    # Without elimination every row of a stiffness matrix sums to zero
    # (the barycentric gradients of an element sum to zero).
    for dims in [(5, 6, 7), (10, 10, 10)]:
        s = femgen.build_system(femgen.Grid(*dims, dirichlet=False, contrast=1000.0))
        A = sp.csr_matrix((s.val, s.idx, s.ptr), shape=(s.n, s.n))
        rs = np.abs(np.asarray(A.sum(axis=1)).ravel())
        scale = np.asarray(abs(A).sum(axis=1)).ravel()
        assert np.max(rs / scale) <= 1e-14


def test_unjittered_unit_laplacian_stencil():
    # Kuhn split of a unit cube, no jitter, coefficient 1: the 7-point
    # Laplacian stencil scaled by h (6h on the diagonal, -h on the axis
    # neighbours), zero on the diagonal edges.
    g = femgen.Grid(6, 6, 6, jitter=0.0, n_incl=0)
    s = femgen.build_system(g)
    A = sp.csr_matrix((s.val, s.idx, s.ptr), shape=(s.n, s.n)).toarray()
    h = 1.0 / 5
    i = (1 - 1) + 4 * ((2 - 1) + 4 * (2 - 1))     # node (1,2,2), interior
    assert A[i, i] == pytest.approx(6 * h, rel=1e-14)
    assert A[i, i + 1] == pytest.approx(-h, rel=1e-14)
    assert A[i, i + 4] == pytest.approx(-h, rel=1e-14)
    assert A[i, i + 16] == pytest.approx(-h, rel=1e-14)
    assert abs(A[i, i + 1 + 4]) <= 1e-16 and abs(A[i, i + 1 + 4 + 16]) <= 1e-16


def test_orientation_and_inclusions():
    for g in [femgen.PAPER_SIZE, femgen.Grid(20, 20, 20, n_incl=4, seed_mesh=7)]:
        assert femgen.min_volume(g) > 0.0        # every jittered tetrahedron positive
        assert femgen.inclusion_tets(g) > 0
        bx = femgen.boxes(g)
        assert bx.shape == (g.n_incl, 6)
        ext = bx[:, 3:] - bx[:, :3]
        assert np.all((bx[:, :3] >= 0) & (bx[:, :3] <= 0.6) & (ext >= 0.2) & (ext <= 0.4))


def test_deterministic():
    g = femgen.Grid(11, 12, 13, seed_mesh=3, seed_x=4)
    a, b = femgen.build_system(g), femgen.build_system(g)
    for f in ("ptr", "idx", "val", "b", "xstar"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    c = femgen.build_system(femgen.Grid(11, 12, 13, seed_mesh=5, seed_x=4))
    assert not np.array_equal(a.val, c.val)


def test_paper_scale_matches_printed_matrix():
    # Section III: 30 880 rows, 449 798 non-zeros (~14.57 per row).
    paper = json.load(open(GOLDEN))["matrix"]
    s = femgen.build_system(femgen.PAPER_SIZE)
    assert abs(s.n / paper["rows"] - 1) < 0.2
    assert abs((s.nnz / s.n) / (paper["nonzeros"] / paper["rows"]) - 1) < 0.05


def test_batched_instances_ranges():
    inst = femgen.batched_instances(256)
    assert len(inst) == 256
    dims = np.array([(g.nx, g.ny, g.nz) for g in inst])
    assert dims.min() >= 12 and dims.max() <= 40
    c = np.array([g.contrast for g in inst])
    assert c.min() >= 10 and c.max() <= 1e4
    assert len({(g.seed_mesh, g.seed_x) for g in inst}) == 256


def test_batched_instances_are_positively_oriented():
    # +-0.2h jitter per coordinate can invert a Kuhn tetrahedron: the
    # original draw of instance 159 (mesh seed 318) does, and its stiffness
    # matrix then has a negative diagonal entry; the batch redraws that mesh
    inst = femgen.batched_instances(256)
    bad = femgen.Grid(34, 21, 27, contrast=inst[159].contrast, seed_mesh=318, seed_x=319)
    assert femgen.min_volume(bad) < 0.0
    s = femgen.build_system(bad)
    diag = np.array([s.val[s.ptr[i] + np.searchsorted(s.idx[s.ptr[i]:s.ptr[i + 1]], i)] for i in range(s.n)])
    assert diag.min() < 0.0
    assert inst[159].seed_mesh == 318 + 512
    assert all(femgen.min_volume(g) > 0.0 for g in inst)
