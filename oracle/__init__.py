"""CPU oracle for the sparse conjugate-gradient solver -- TEST INFRASTRUCTURE.

Only the tests, the smoke check and the benchmark's CPU-baseline leg load this
package; the library never does.  It wraps ``oracle.c`` (plain C, IEEE double,
compiled with ``-ffp-contract=off``), which restates the paper's CG listing
(Section III), its symmetric-storage product (A = L + D + U with U' = L,
Section III) and its single-precision variant (Section IV).  It shares no code
with the CUDA path.

Parity status per function (what pins it; see ``tests/test_oracle_pins.py``):
  spmv (CSR, symmetric upper, CSC)  -- dense brute force, format equivalence
  cg (also pipelined=True)            -- dense Cholesky, finite termination,
                                         A-orthogonality, A-norm monotonicity,
                                         closed-form diagonal/tridiagonal cases
  cg_f32 / cg_ir / cg_ru              -- true residual in double, error vs x*, exact
                                         float-representable special cases
  dot_long                            -- exact rational arithmetic
  dot_f32                             -- exact sum within the pairwise bound
  grad_values / element_grad /        -- central finite differences of the
  assemble                               loss through oracle solves, dense
                                         reference gradients, the generator's
                                         assembled matrix
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_oracle.so")
# The same source compiled with -fopenmp: a separate library whose CG loops
# run on several host threads and give the single-threaded library's bits
# (oracle.c, "multi-threaded build").  Used for the timed CPU baseline on every
# host core and for the large reference solves of tests/golden.
_SO_OMP = os.path.join(_HERE, "_oracle_omp.so")
_lib = None
_lib_omp = None

CSR, SYM_UPPER, CSC = 0, 1, 2
FORMATS = {"csr": CSR, "sym": SYM_UPPER, "sym_upper": SYM_UPPER, "csc": CSC}
STATUS = {0: "OK", 1: "INVALID", 2: "NOT_SPD", 3: "MAXIT", 4: "NONFINITE"}


class Info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("status", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("rel_res_recursive", ctypes.c_double), ("rel_res_true", ctypes.c_double)]


class History(ctypes.Structure):
    _fields_ = [("cap", ctypes.c_int32), ("count", ctypes.c_int32),
                ("p", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("alpha", ctypes.c_void_p), ("beta", ctypes.c_void_p)]


def compile_oracle(src: str = _SRC, dst: str = _SO, openmp: bool = False) -> str:
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11",
                    *(["-fopenmp"] if openmp else []), src, "-o", dst, "-lm"], check=True)
    return dst


def build() -> str:
    """Compiles both builds of the oracle (single- and multi-threaded)."""
    for so, omp in ((_SO, False), (_SO_OMP, True)):
        if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
            compile_oracle(dst=so, openmp=omp)
    return _SO


def load_threaded(threads: int | None = None):
    """The multi-threaded build (same bits as ``load()``'s); ``threads``
    sets its thread count (default: every host core)."""
    global _lib_omp
    if _lib_omp is None:
        build()
        _lib_omp = load(_SO_OMP)
    _lib_omp.orc_set_threads(int(threads or os.cpu_count() or 1))
    return _lib_omp


def threads(lib=None) -> int:
    """Threads the given build runs its CG loops on (1 for the plain build)."""
    return int((lib or load()).orc_threads())


def load(path: str | None = None):
    """Load the oracle library (``path`` lets tests load a deliberately broken copy)."""
    global _lib
    if path is None and _lib is not None:
        return _lib
    so = path or build()
    lib = ctypes.CDLL(so)
    vp, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    for name in ("orc_spmv_csr", "orc_spmv_sym_upper", "orc_spmv_csc"):
        getattr(lib, name).argtypes = [i64, vp, vp, vp, vp, vp]
    lib.orc_spmv.argtypes = [ctypes.c_int, i64, vp, vp, vp, vp, vp]
    lib.orc_spmv_f32.argtypes = [ctypes.c_int, i64, vp, vp, vp, vp, vp]
    lib.orc_abs_spmv.argtypes = [ctypes.c_int, i64, vp, vp, vp, vp, vp]
    lib.orc_dot.argtypes = [i64, vp, vp]
    lib.orc_dot.restype = d
    lib.orc_dot_long.argtypes = [i64, vp, vp]
    lib.orc_dot_long.restype = d
    lib.orc_dot_f32.argtypes = [i64, vp, vp]
    lib.orc_dot_f32.restype = ctypes.c_float
    lib.orc_cg.argtypes = [ctypes.c_int, i64, vp, vp, vp, vp, vp, d, i32,
                           ctypes.POINTER(Info), ctypes.POINTER(History)]
    lib.orc_cg_f32.argtypes = [ctypes.c_int, i64, vp, vp, vp, vp, vp, ctypes.c_float, i32,
                               ctypes.POINTER(i32)]
    lib.orc_cg_f32.restype = i32
    lib.orc_cg_ir.argtypes = [ctypes.c_int, i64, vp, vp, vp, vp, vp, d, i32, d, i32,
                              ctypes.POINTER(Info)]
    lib.orc_grad_values.argtypes = [ctypes.c_int, i64, vp, vp, vp, vp, vp]
    lib.orc_cg_ru.argtypes = [ctypes.c_int, i64, vp, vp, vp, vp, vp, d, i32, d, ctypes.POINTER(Info)]
    lib.orc_cg_pipelined.argtypes = [ctypes.c_int, i64, vp, vp, vp, vp, vp, d, i32,
                                     ctypes.POINTER(Info), ctypes.POINTER(History)]
    lib.orc_element_grad.argtypes = [i64, i32, vp, vp, vp, vp]
    lib.orc_assemble.argtypes = [i64, vp, vp, vp, vp, vp]
    lib.orc_threads.restype = i32
    lib.orc_set_threads.argtypes = [i32]
    if path is None:
        _lib = lib
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _fmt(fmt) -> int:
    return FORMATS[fmt] if isinstance(fmt, str) else int(fmt)


def _arrays(ptr, idx, val, vdtype=np.float64):
    return (np.ascontiguousarray(ptr, dtype=np.int32), np.ascontiguousarray(idx, dtype=np.int32),
            np.ascontiguousarray(val, dtype=vdtype))


def spmv(fmt, ptr, idx, val, x, lib=None) -> np.ndarray:
    """y = A x for A given as CSR, symmetric upper (D + U by rows) or CSC."""
    lib = lib or load()
    ptr, idx, val = _arrays(ptr, idx, val)
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = ptr.shape[0] - 1
    y = np.empty(n, dtype=np.float64)
    lib.orc_spmv(_fmt(fmt), n, _p(ptr), _p(idx), _p(val), _p(x), _p(y))
    return y


def spmv_f32(fmt, ptr, idx, val32, x32, lib=None) -> np.ndarray:
    lib = lib or load()
    ptr, idx, val32 = _arrays(ptr, idx, val32, np.float32)
    x32 = np.ascontiguousarray(x32, dtype=np.float32)
    n = ptr.shape[0] - 1
    y = np.empty(n, dtype=np.float32)
    lib.orc_spmv_f32(_fmt(fmt), n, _p(ptr), _p(idx), _p(val32), _p(x32), _p(y))
    return y


def abs_spmv(fmt, ptr, idx, val, x, lib=None) -> np.ndarray:
    """|A| |x|: the scale of the componentwise rounding bound of y = A x."""
    lib = lib or load()
    ptr, idx, val = _arrays(ptr, idx, val)
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = ptr.shape[0] - 1
    y = np.empty(n, dtype=np.float64)
    lib.orc_abs_spmv(_fmt(fmt), n, _p(ptr), _p(idx), _p(val), _p(x), _p(y))
    return y


def dot(a, b, lib=None) -> float:
    lib = lib or load()
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return float(lib.orc_dot(a.shape[0], _p(a), _p(b)))


def dot_long(a, b, lib=None) -> float:
    lib = lib or load()
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return float(lib.orc_dot_long(a.shape[0], _p(a), _p(b)))


def dot_f32(a, b, lib=None) -> float:
    """Single-precision dot product of the single-precision CG (tree order)."""
    lib = lib or load()
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    return float(lib.orc_dot_f32(a.shape[0], _p(a), _p(b)))


@dataclass
class Result:
    x: np.ndarray
    iterations: int
    restarts: int
    status: str
    rel_res_recursive: float
    rel_res_true: float
    p_hist: np.ndarray | None = None
    x_hist: np.ndarray | None = None
    alpha: np.ndarray | None = None
    beta: np.ndarray | None = None


def cg(fmt, ptr, idx, val, b, x0=None, tol=1e-10, maxit=None, history=0, lib=None, pipelined=False,
       scalar_history=0) -> Result:
    """Plain double-precision CG (Section III listing; readings in oracle.c);
    pipelined=True: the single-reduction form of the same iteration.
    history=h records p, x, alpha and beta of the first h iterations;
    scalar_history=h only alpha and beta (no n-sized copies)."""
    lib = lib or load()
    ptr, idx, val = _arrays(ptr, idx, val)
    n = ptr.shape[0] - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    maxit = n if maxit is None else int(maxit)
    info = Info()
    hist = None
    ph = xh = al = be = None
    if history:
        ph = np.zeros((history, n))
        xh = np.zeros((history, n))
        al = np.zeros(history)
        be = np.zeros(history)
        hist = History(history, 0, ph.ctypes.data, xh.ctypes.data, al.ctypes.data, be.ctypes.data)
    elif scalar_history:
        al = np.zeros(scalar_history)
        be = np.zeros(scalar_history)
        hist = History(scalar_history, 0, None, None, al.ctypes.data, be.ctypes.data)
    fn = lib.orc_cg_pipelined if pipelined else lib.orc_cg
    fn(_fmt(fmt), n, _p(ptr), _p(idx), _p(val), _p(b), _p(x), float(tol), maxit,
       ctypes.byref(info), ctypes.byref(hist) if hist is not None else None)
    res = Result(x, info.iterations, info.restarts, STATUS[info.status], info.rel_res_recursive,
                 info.rel_res_true)
    if history:
        c = hist.count
        res.p_hist, res.x_hist, res.alpha, res.beta = ph[:c], xh[:c], al[:c], be[:c]
    elif scalar_history:
        c = hist.count
        res.alpha, res.beta = al[:c], be[:c]
    return res


def lanczos_extremes(alpha, beta):
    """Extreme eigenvalue estimates of A from the CG step lengths of one run
    (no restart): the Lanczos tridiagonal T with T_00 = 1/alpha_0,
    T_kk = 1/alpha_k + beta_{k-1}/alpha_{k-1}, T_{k,k+1} = sqrt(beta_k)/alpha_k
    (the CG-Lanczos relation).  Its eigenvalues are Ritz values of A, so
    lambda_max(T) <= lambda_max(A) and lambda_min(T) >= lambda_min(A)."""
    from scipy.linalg import eigvalsh_tridiagonal

    alpha = np.asarray(alpha, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    m = alpha.shape[0]
    d = 1.0 / alpha
    d[1:] += beta[:m - 1] / alpha[:m - 1]
    e = np.sqrt(beta[:m - 1]) / alpha[:m - 1]
    w = eigvalsh_tridiagonal(d, e)
    return float(w[0]), float(w[-1])


def cg_f32(fmt, ptr, idx, val32, rhs32, tol, maxit, lib=None):
    """Single-precision CG from d = 0; returns (d, iterations, breakdown)."""
    lib = lib or load()
    ptr, idx, val32 = _arrays(ptr, idx, val32, np.float32)
    rhs32 = np.ascontiguousarray(rhs32, dtype=np.float32)
    n = ptr.shape[0] - 1
    d = np.zeros(n, dtype=np.float32)
    bd = ctypes.c_int32()
    it = lib.orc_cg_f32(_fmt(fmt), n, _p(ptr), _p(idx), _p(val32), _p(rhs32), _p(d), float(tol), int(maxit),
                        ctypes.byref(bd))
    return d, int(it), bool(bd.value)


def cg_ir(fmt, ptr, idx, val, b, x0=None, tol=1e-10, maxit=None, inner_tol=1e-4, max_outer=30,
          lib=None) -> Result:
    """Single-precision inner CG with double-precision iterative refinement."""
    lib = lib or load()
    ptr, idx, val = _arrays(ptr, idx, val)
    n = ptr.shape[0] - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    maxit = 10 * max(n, 1) if maxit is None else int(maxit)
    info = Info()
    lib.orc_cg_ir(_fmt(fmt), n, _p(ptr), _p(idx), _p(val), _p(b), _p(x), float(tol), maxit,
                  float(inner_tol), int(max_outer), ctypes.byref(info))
    return Result(x, info.iterations, info.restarts, STATUS[info.status], info.rel_res_recursive,
                  info.rel_res_true)


def batch_solve(row_off, ptr, idx, val, B, X0=None, tol=1e-10, maxit=None, precision="fp32_ir", inner_tol=1e-4,
                max_outer=30, lib=None):
    """Independent systems of a block-diagonal CSR (instance i: rows
    row_off[i]..row_off[i+1], global columns), each right-hand side solved on
    its own by ``cg_ir`` (precision "fp32_ir"), ``cg_ru`` ("fp32_ru") or ``cg``
    ("fp64").  Returns
    (X, results) with results[i][k] the Result of instance i, column k."""
    lib = lib or load()
    row_off = np.asarray(row_off, dtype=np.int64)
    B = np.asarray(B, dtype=np.float64)
    X = np.zeros_like(B) if X0 is None else np.array(X0, dtype=np.float64, copy=True)
    results = []
    for i in range(row_off.shape[0] - 1):
        r0, r1 = int(row_off[i]), int(row_off[i + 1])
        k0, k1 = int(ptr[r0]), int(ptr[r1])
        p_i = np.asarray(ptr[r0:r1 + 1], dtype=np.int64) - k0
        i_i = np.asarray(idx[k0:k1], dtype=np.int64) - r0
        v_i = val[k0:k1]
        row = []
        for k in range(B.shape[1]):
            m = maxit if maxit is not None else max(r1 - r0, 1)
            if precision == "fp64":
                res = cg("csr", p_i, i_i, v_i, B[r0:r1, k], X[r0:r1, k], tol=tol, maxit=m, lib=lib)
            elif precision == "fp32_ru":
                res = cg_ru("csr", p_i, i_i, v_i, B[r0:r1, k], X[r0:r1, k], tol=tol, maxit=m, lib=lib)
            else:
                res = cg_ir("csr", p_i, i_i, v_i, B[r0:r1, k], X[r0:r1, k], tol=tol, maxit=m, inner_tol=inner_tol,
                            max_outer=max_outer, lib=lib)
            X[r0:r1, k] = res.x
            row.append(res)
        results.append(row)
    return X, results


def cg_ru(fmt, ptr, idx, val, b, x0=None, tol=1e-10, maxit=None, delta=0.1, lib=None) -> Result:
    """Single-precision CG with double-precision reliable updates (restarts =
    number of updates)."""
    lib = lib or load()
    ptr, idx, val = _arrays(ptr, idx, val)
    n = ptr.shape[0] - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    maxit = 10 * max(n, 1) if maxit is None else int(maxit)
    info = Info()
    lib.orc_cg_ru(_fmt(fmt), n, _p(ptr), _p(idx), _p(val), _p(b), _p(x), float(tol), maxit, float(delta),
                  ctypes.byref(info))
    return Result(x, info.iterations, info.restarts, STATUS[info.status], info.rel_res_recursive,
                  info.rel_res_true)


# ------------------------------------------------------------ differentiation
def grad_values(fmt, ptr, idx, lam, x, lib=None) -> np.ndarray:
    """dL/d(stored values) from the adjoint lambda = A^-1 dL/dx and x."""
    lib = lib or load()
    ptr = np.ascontiguousarray(ptr, dtype=np.int32)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = np.empty(idx.shape[0])
    lib.orc_grad_values(_fmt(fmt), ptr.shape[0] - 1, _p(ptr), _p(idx), _p(lam), _p(x), _p(g))
    return g


def element_grad(pos, w, g, lib=None) -> np.ndarray:
    """dL/dcoef per element from the stored-value gradient g (chain rule
    through the assembly map)."""
    lib = lib or load()
    pos = np.ascontiguousarray(pos, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = np.empty(pos.shape[0])
    lib.orc_element_grad(pos.shape[0], pos.shape[1], _p(pos), _p(w), _p(g), _p(out))
    return out


def assemble(tptr, telem, tw, coef, lib=None) -> np.ndarray:
    """Stored values sum_e coef_e w from the assembly map by position."""
    lib = lib or load()
    tptr = np.ascontiguousarray(tptr, dtype=np.int64)
    telem = np.ascontiguousarray(telem, dtype=np.int32)
    tw = np.ascontiguousarray(tw, dtype=np.float64)
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    out = np.empty(tptr.shape[0] - 1)
    lib.orc_assemble(out.shape[0], _p(tptr), _p(telem), _p(tw), _p(coef), _p(out))
    return out


def loss_gradients(fmt, ptr, idx, val, b, xt, tol=1e-13, maxit=None, lib=None):
    """L = ||x - xt||^2 with A x = b (double-precision CG): returns
    (L, x, lambda, dL/db, dL/dval) through the adjoint solve A lambda = 2 (x - xt)."""
    lib = lib or load()
    n = np.asarray(ptr).shape[0] - 1
    m = maxit if maxit is not None else 20 * max(n, 1)
    fw = cg(fmt, ptr, idx, val, b, tol=tol, maxit=m, lib=lib)
    gx = 2.0 * (fw.x - xt)
    adj = cg(fmt, ptr, idx, val, gx, tol=tol, maxit=m, lib=lib)
    L = float(np.dot(fw.x - xt, fw.x - xt))
    return L, fw.x, adj.x, adj.x.copy(), grad_values(fmt, ptr, idx, adj.x, fw.x, lib=lib)
