"""Seeded synthetic FEM inputs: stiffness matrices of jittered P1 tetrahedral
meshes with high-contrast box inclusions, the stand-in for the paper's
electrical-machine matrix (Section III: a 30 880-row SPD matrix with 449 798
non-zeros, about 14.6 per row).

This module produces inputs only.  It holds none of the solver's arithmetic
(no sparse products, no conjugate-gradient steps) and is shared by the CPU
oracle, the tests and the benchmark; it imports neither of them.

The C source (``femgen.c``) is compiled on first use with ``gcc`` into
``_femgen.so`` next to this file (``build()`` does it explicitly).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "femgen.c")
_SO = os.path.join(_HERE, "_femgen.so")
_lib = None


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("n_incl", ctypes.c_int32), ("dirichlet", ctypes.c_int32), ("pad_", ctypes.c_int32),
        ("jitter", ctypes.c_double), ("contrast", ctypes.c_double),
        ("seed_mesh", ctypes.c_uint64), ("seed_x", ctypes.c_uint64),
    ]


@dataclass(frozen=True)
class Grid:
    """One synthetic system: node grid, inclusions, contrast and seeds."""
    nx: int
    ny: int
    nz: int
    n_incl: int = 1
    contrast: float = 1000.0
    jitter: float = 0.2
    seed_mesh: int = 0
    seed_x: int = 1
    dirichlet: bool = True

    def params(self) -> Params:
        return Params(self.nx, self.ny, self.nz, self.n_incl, 1 if self.dirichlet else 0, 0,
                      float(self.jitter), float(self.contrast), int(self.seed_mesh), int(self.seed_x))


# Workloads shaped like the paper's (Section III) at the sizes the benchmark uses.
PAPER_SIZE = Grid(31, 31, 32)                               # ~25K rows, the paper's scale
LARGE = Grid(128, 128, 128)                                  # ~2.0M rows, ~29.6M nnz
DIFF = Grid(64, 64, 64)                                      # ~238K rows
LARGEST = Grid(256, 256, 256, n_incl=4)                      # ~16.4M rows, ~244M nnz


def batched_instances(count: int = 256, seed: int = 0):
    """Uneven batch: grid edges uniform in [12, 40] per axis, contrast
    log-uniform in [10, 1e4], seeds derived from the instance id.

    Independent +-0.2h jitter of every coordinate can invert a Kuhn
    tetrahedron (rarely: one instance in the first 256), which makes the
    stiffness matrix indefinite; such an instance is redrawn with the next
    mesh seed (2 i + 512 a for attempt a) until every element is positively
    oriented."""
    lib = _load()
    out = []
    for i in range(count):
        u = [lib.femgen_uniform(ctypes.c_uint64(seed + 1000003), ctypes.c_uint64(4 * i + d)) for d in range(4)]
        nx, ny, nz = (12 + min(28, int(v * 29)) for v in u[:3])
        contrast = float(10.0 ** (1.0 + 3.0 * u[3]))
        for a in range(64):
            g = Grid(nx, ny, nz, n_incl=1, contrast=contrast, seed_mesh=2 * i + 512 * a, seed_x=2 * i + 1)
            if min_volume(g) > 0.0:
                break
        else:  # pragma: no cover
            raise RuntimeError(f"no positively oriented mesh for batch instance {i}")
        out.append(g)
    return out


def _compile(dst: str = _SO) -> str:
    flags = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11"]
    try:
        subprocess.run(flags + ["-fopenmp", _SRC, "-o", dst, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(flags + [_SRC, "-o", dst, "-lm"], check=True)
    return dst


def build() -> str:
    """Compile the generator (idempotent when the library is newer than the source)."""
    if not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        _compile()
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.POINTER(Params)
        i64p = ctypes.POINTER(ctypes.c_int64)
        vp = ctypes.c_void_p
        lib.femgen_size.argtypes = [P, i64p, i64p]
        lib.femgen_build.argtypes = [P, vp, vp, vp, vp, vp]
        lib.femgen_elements.argtypes = [P, vp, vp, vp]
        lib.femgen_boxes.argtypes = [P, vp]
        lib.femgen_min_volume.argtypes = [P]
        lib.femgen_min_volume.restype = ctypes.c_double
        lib.femgen_count_inclusion_tets.argtypes = [P]
        lib.femgen_count_inclusion_tets.restype = ctypes.c_int64
        lib.femgen_upper.argtypes = [ctypes.c_int64, vp, vp, vp, vp, vp, vp]
        lib.femgen_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.femgen_uniform.restype = ctypes.c_double
        _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def size(g: Grid) -> tuple[int, int]:
    lib = _load()
    n, nnz = ctypes.c_int64(), ctypes.c_int64()
    if lib.femgen_size(ctypes.byref(g.params()), ctypes.byref(n), ctypes.byref(nnz)):
        raise ValueError(f"invalid grid {g}")
    return n.value, nnz.value


@dataclass
class System:
    """A generated SPD system in full CSR (0-based, sorted columns)."""
    grid: Grid
    n: int
    ptr: np.ndarray     # int32[n+1]
    idx: np.ndarray     # int32[nnz]
    val: np.ndarray     # float64[nnz]
    b: np.ndarray       # float64[n], element-assembled A @ xstar
    xstar: np.ndarray   # float64[n], U(-1, 1)

    @property
    def nnz(self) -> int:
        return int(self.idx.shape[0])

    def upper(self):
        """(ptr, idx, val) of the stored upper triangle, diagonal included."""
        return upper(self.n, self.ptr, self.idx, self.val)

    def csc(self):
        """(colptr, rowidx, val) of the same matrix in CSC.  The matrix is
        exactly symmetric, so its CSC arrays are its CSR arrays."""
        return self.ptr, self.idx, self.val


def build_system(g: Grid) -> System:
    lib = _load()
    n, nnz = size(g)
    ptr = np.empty(n + 1, dtype=np.int32)
    idx = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    b = np.empty(n, dtype=np.float64)
    xs = np.empty(n, dtype=np.float64)
    rc = lib.femgen_build(ctypes.byref(g.params()), _ptr(ptr), _ptr(idx), _ptr(val), _ptr(b), _ptr(xs))
    if rc:
        raise ValueError(f"femgen_build failed ({rc}) for {g}")
    return System(g, n, ptr, idx, val, b, xs)


def upper(n: int, ptr: np.ndarray, idx: np.ndarray, val: np.ndarray):
    """Upper triangle (j >= i) of a sorted-column CSR matrix: index selection only."""
    lib = _load()
    uptr = np.empty(n + 1, dtype=np.int32)
    lib.femgen_upper(n, _ptr(ptr), _ptr(idx), _ptr(val), _ptr(uptr), None, None)
    m = int(uptr[-1])
    uidx = np.empty(m, dtype=np.int32)
    uval = np.empty(m, dtype=np.float64)
    lib.femgen_upper(n, _ptr(ptr), _ptr(idx), _ptr(val), _ptr(uptr), _ptr(uidx), _ptr(uval))
    return uptr, uidx, uval


def boxes(g: Grid) -> np.ndarray:
    lib = _load()
    out = np.empty((max(g.n_incl, 1), 6), dtype=np.float64)
    lib.femgen_boxes(ctypes.byref(g.params()), _ptr(out))
    return out[: g.n_incl]


def min_volume(g: Grid) -> float:
    return float(_load().femgen_min_volume(ctypes.byref(g.params())))


def inclusion_tets(g: Grid) -> int:
    return int(_load().femgen_count_inclusion_tets(ctypes.byref(g.params())))


def uniform(seed: int, counter: int) -> float:
    return float(_load().femgen_uniform(ctypes.c_uint64(seed), ctypes.c_uint64(counter)))


@dataclass
class BatchSystem:
    """Independent systems as one block-diagonal CSR with global columns:
    instance i owns rows row_off[i]..row_off[i+1]; B = A X* column by column,
    (n, nrhs) row-major."""
    grids: list
    row_off: np.ndarray   # int64[count+1]
    ptr: np.ndarray       # int32[n+1]
    idx: np.ndarray       # int32[nnz], global columns
    val: np.ndarray       # float64[nnz]
    B: np.ndarray         # float64[n, nrhs]
    Xstar: np.ndarray     # float64[n, nrhs]

    @property
    def count(self) -> int:
        return int(self.row_off.shape[0]) - 1

    @property
    def n(self) -> int:
        return int(self.row_off[-1])

    @property
    def nnz(self) -> int:
        return int(self.idx.shape[0])

    def instance(self, i: int):
        """(ptr, idx, val) of instance i alone, 0-based local columns."""
        r0, r1 = int(self.row_off[i]), int(self.row_off[i + 1])
        k0, k1 = int(self.ptr[r0]), int(self.ptr[r1])
        return ((self.ptr[r0:r1 + 1] - k0).astype(np.int32), (self.idx[k0:k1] - r0).astype(np.int32),
                self.val[k0:k1])


def build_batch(grids, nrhs: int = 8) -> BatchSystem:
    """Block-diagonal batch of the generator's systems with nrhs manufactured
    solutions per instance: x*_k ~ U(-1, 1) seeded by the instance's seed_x and
    k, b_k = A x*_k (sparse product of the generated matrix, input generation)."""
    import scipy.sparse as sp

    ptrs, idxs, vals, Bs, Xs = [], [], [], [], []
    row_off = [0]
    nnz_off = 0
    for g in grids:
        s = build_system(g)
        r0 = row_off[-1]
        ptrs.append(s.ptr[:-1].astype(np.int64) + nnz_off)
        idxs.append(s.idx.astype(np.int64) + r0)
        vals.append(s.val)
        X = np.stack([random_vector(s.n, 1_000_000 + 8 * g.seed_x + k) for k in range(nrhs)], axis=1) \
            if s.n else np.zeros((0, nrhs))
        A = sp.csr_matrix((s.val, s.idx, s.ptr), shape=(s.n, s.n))
        Bs.append(np.asarray(A @ X).reshape(s.n, nrhs))
        Xs.append(X.reshape(s.n, nrhs))
        nnz_off += s.nnz
        row_off.append(r0 + s.n)
    ptr = np.concatenate(ptrs + [np.array([nnz_off], dtype=np.int64)])
    if nnz_off >= 2 ** 31:
        raise ValueError("batch has more than 2^31 - 1 entries")
    return BatchSystem(list(grids), np.array(row_off, dtype=np.int64), ptr.astype(np.int32),
                       np.concatenate(idxs).astype(np.int32), np.concatenate(vals),
                       np.ascontiguousarray(np.concatenate(Bs, axis=0)),
                       np.ascontiguousarray(np.concatenate(Xs, axis=0)))


@dataclass
class Elements:
    """Tetrahedra of a generated system: unknown index of each vertex (-1 for
    an eliminated Dirichlet node), unit-coefficient element matrix
    Kh = |V| G G' (4 x 4) and coefficient; A = sum_e coef_e Kh_e restricted to
    the unknowns."""
    nodes: np.ndarray   # int32[E, 4]
    kh: np.ndarray      # float64[E, 4, 4]
    coef: np.ndarray    # float64[E]

    @property
    def count(self) -> int:
        return int(self.coef.shape[0])


def elements(g: Grid) -> Elements:
    lib = _load()
    ne = 6 * (g.nx - 1) * (g.ny - 1) * (g.nz - 1)
    nodes = np.empty((ne, 4), dtype=np.int32)
    kh = np.empty((ne, 4, 4), dtype=np.float64)
    coef = np.empty(ne, dtype=np.float64)
    if lib.femgen_elements(ctypes.byref(g.params()), _ptr(nodes), _ptr(kh), _ptr(coef)):
        raise ValueError(f"invalid grid {g}")
    return Elements(nodes, kh, coef)


def element_map(el: Elements, ptr: np.ndarray, idx: np.ndarray, storage: str = "csr"):
    """Positions of the element matrices in a stored matrix.

    Returns (pos int32[E, m], w float64[E, m]): entry k of element e adds
    coef_e * w[e, k] to the stored value at pos[e, k] (-1: none).  "csr" (full
    storage, or CSC of the symmetric matrix): m = 16, every vertex pair (a, b).
    "sym" (upper triangle and diagonal): m = 10, the pairs a <= b, placed at
    the stored entry (min(i, j), max(i, j)).  The assembly A = sum_e coef_e Kh_e
    is then val[p] = sum over (e, k) with pos[e, k] = p of coef_e w[e, k].
    """
    E = el.count
    pairs = [(a, b) for a in range(4) for b in range(4)] if storage == "csr" else \
        [(a, b) for a in range(4) for b in range(a, 4)]
    m = len(pairs)
    pos = np.full((E, m), -1, dtype=np.int64)
    w = np.zeros((E, m))
    ptr = np.asarray(ptr, dtype=np.int64)
    idx = np.asarray(idx, dtype=np.int64)
    for k, (a, b) in enumerate(pairs):
        i = el.nodes[:, a].astype(np.int64)
        j = el.nodes[:, b].astype(np.int64)
        ok = (i >= 0) & (j >= 0)
        r = np.where(ok, np.minimum(i, j) if storage == "sym" else i, 0)
        c = np.where(ok, np.maximum(i, j) if storage == "sym" else j, 0)
        # position of column c in row r: rows hold sorted columns
        lo = ptr[r]
        hi = ptr[r + 1]
        p = lo.copy()
        step = hi - lo
        while np.any(step > 0):  # vectorised lower bound
            half = step // 2
            mid = p + half
            go = (step > 0) & (idx[np.minimum(mid, len(idx) - 1)] < c)
            p = np.where(go, mid + 1, p)
            step = np.where(go, step - half - 1, half)
        found = ok & (p < hi) & (idx[np.minimum(p, len(idx) - 1)] == c)
        if np.any(ok & ~found):
            raise ValueError("an element pair is missing from the stored pattern")
        pos[:, k] = np.where(found, p, -1)
        w[:, k] = np.where(found, el.kh[:, a, b], 0.0)
    return pos.astype(np.int32), w


def assembly_map(pos: np.ndarray, w: np.ndarray, nnz: int):
    """The element map by stored position: (tptr int64[nnz+1], telem int32,
    tw float64) with the contributions (element, weight) of position p at
    tptr[p]..tptr[p+1], elements increasing."""
    E, m = pos.shape
    p = pos.reshape(-1).astype(np.int64)
    e = np.repeat(np.arange(E, dtype=np.int64), m)
    ww = w.reshape(-1)
    keep = p >= 0
    p, e, ww = p[keep], e[keep], ww[keep]
    order = np.lexsort((e, p))
    p, e, ww = p[order], e[order], ww[order]
    tptr = np.zeros(nnz + 1, dtype=np.int64)
    np.add.at(tptr, p + 1, 1)
    return np.cumsum(tptr), e.astype(np.int32), np.ascontiguousarray(ww)


def random_vector(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Seeded U(lo, hi) vector (numpy's PCG64, seeded; inputs only)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=n)
