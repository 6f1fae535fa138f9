"""GB300-native sparse conjugate-gradient solver (Python binding).

Solves A x = b for sparse symmetric positive-definite A by the conjugate
gradient iteration of Section III of "Parallel Sparse Matrix Solver on the GPU
Applied to Simulation of Electrical Machines", with A given as CSR, symmetric
CSR (upper triangle and diagonal) or CSC.  The names mirror the C ABI in
``include/gbcg.h``: ``Matrix`` wraps ``gbcg_create``/``gbcg_destroy``,
``Matrix.spmv`` wraps ``gbcg_spmv``, ``Matrix.solve`` wraps ``gbcg_solve``.

PyTorch provides device memory and streams; every computation runs in the
library's own sm_103a kernels.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import GbcgError

FORMATS = {"csr": _lib.GBCG_CSR, "sym": _lib.GBCG_SYM_CSR_UPPER, "sym_upper": _lib.GBCG_SYM_CSR_UPPER,
           "csc": _lib.GBCG_CSC}
PRECISIONS = {"fp64": _lib.GBCG_FP64, "fp32_ir": _lib.GBCG_FP32_IR, "ir": _lib.GBCG_FP32_IR,
              "fp32_ru": _lib.GBCG_FP32_RU}
VARIANTS = {"standard": _lib.GBCG_STANDARD, "pipelined": _lib.GBCG_PIPELINED}


def build(verbose: bool = False) -> str:
    """Compile libgbcg.so for sm_103a in-tree."""
    from .builder import build as _build
    return _build(verbose=verbose)


def _torch():
    import torch
    return torch


def _is_tensor(a) -> bool:
    try:
        torch = _torch()
    except ImportError:  # pragma: no cover
        return False
    return isinstance(a, torch.Tensor)


def _stream_handle(stream=None):
    torch = _torch()
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _host_stream(stream):
    if stream is not None:
        return _stream_handle(stream)
    try:
        torch = _torch()
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:  # pragma: no cover
        pass
    return ctypes.c_void_p(0)


@dataclass
class SolveInfo:
    iterations: int
    outer: int
    status: str
    rel_res_recursive: float
    rel_res_true: float
    ms: float
    kernel_ms: float = 0.0
    kernel_launches: int = 0
    launches: int = 0


class Matrix:
    """A sparse SPD matrix resident on the GPU (``gbcg_create``).

    ``ptr``/``idx``/``val`` are numpy arrays (host) or CUDA tensors (device):
    int32 offsets, int32 indices, float64 values, ``index_base`` 0 or 1.
    """

    def __init__(self, fmt, ptr, idx, val, index_base: int = 0, stream=None):
        lib = _lib.load()
        self._lib = lib
        self.format = FORMATS[fmt] if isinstance(fmt, str) else int(fmt)
        self._h = ctypes.c_void_p()
        if _is_tensor(ptr):
            torch = _torch()
            ptr = ptr.to(torch.int32).contiguous()
            idx = idx.to(torch.int32).contiguous()
            val = val.to(torch.float64).contiguous()
            self.n = int(ptr.numel()) - 1
            nnz = int(idx.numel())
            mem = _lib.GBCG_DEVICE if ptr.is_cuda else _lib.GBCG_HOST
            args = (ptr.data_ptr(), idx.data_ptr(), val.data_ptr())
            keep = (ptr, idx, val)
        else:
            ptr = np.ascontiguousarray(ptr, dtype=np.int32)
            idx = np.ascontiguousarray(idx, dtype=np.int32)
            val = np.ascontiguousarray(val, dtype=np.float64)
            self.n = int(ptr.shape[0]) - 1
            nnz = int(idx.shape[0])
            mem = _lib.GBCG_HOST
            args = (ptr.ctypes.data, idx.ctypes.data, val.ctypes.data)
            keep = (ptr, idx, val)
        rc = lib.gbcg_create(ctypes.byref(self._h), self.format, self.n, nnz, *[ctypes.c_void_p(a) for a in args],
                             int(index_base), mem, _host_stream(stream))
        del keep
        _lib.check(rc, "gbcg_create")
        self.nnz = nnz

    # ------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.gbcg_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # pragma: no cover
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> int:
        return int(self._h.value or 0)

    def stats(self) -> dict:
        s = _lib.Stats()
        _lib.check(self._lib.gbcg_stats(self._h, ctypes.byref(s)), "gbcg_stats")
        return {name: getattr(s, name) for name, _ in _lib.Stats._fields_}

    def update_values(self, val, stream=None):
        """Replace the stored values (same pattern, same order as at creation):
        a float64 CUDA tensor or a numpy array (``gbcg_update_values``)."""
        if _is_tensor(val):
            torch = _torch()
            val = val.to(torch.float64).contiguous()
            if val.numel() != self.nnz:
                raise ValueError(f"expected {self.nnz} values")
            mem = _lib.GBCG_DEVICE if val.is_cuda else _lib.GBCG_HOST
            stream_h = _stream_handle(stream) if val.is_cuda else _host_stream(stream)
            ptr = val.data_ptr()
        else:
            val = np.ascontiguousarray(val, dtype=np.float64)
            if val.shape[0] != self.nnz:
                raise ValueError(f"expected {self.nnz} values")
            mem, stream_h, ptr = _lib.GBCG_HOST, _host_stream(stream), val.ctypes.data
        _lib.check(self._lib.gbcg_update_values(self._h, ctypes.c_void_p(ptr), mem, stream_h), "gbcg_update_values")
        if mem == _lib.GBCG_HOST:
            _torch().cuda.synchronize()

    # ------------------------------------------------------------ product
    def spmv(self, x, y=None, stream=None):
        """y = A x (float64 CUDA tensors)."""
        torch = _torch()
        if y is None:
            y = torch.empty(self.n, dtype=torch.float64, device=x.device)
        _check_vec(x, torch.float64, self.n, "x")
        _check_vec(y, torch.float64, self.n, "y")
        _lib.check(self._lib.gbcg_spmv(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                       _stream_handle(stream)), "gbcg_spmv")
        return y

    def spmv_f32(self, x, y=None, stream=None):
        """y = A32 x with the single-precision copy of the values (float32 CUDA tensors)."""
        torch = _torch()
        if y is None:
            y = torch.empty(self.n, dtype=torch.float32, device=x.device)
        _check_vec(x, torch.float32, self.n, "x")
        _check_vec(y, torch.float32, self.n, "y")
        _lib.check(self._lib.gbcg_spmv_f32(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                           _stream_handle(stream)), "gbcg_spmv_f32")
        return y

    # ------------------------------------------------------------ solve
    def solve(self, b, x=None, tol: float = 1e-10, maxit: int = 0, precision: str = "fp64",
              inner_tol: float = 0.0, max_outer: int = 30, wait_timeout_ms: int = 1000,
              max_restarts: int = 3, variant: str = "standard", stream=None, raise_on_error: bool = True):
        """Conjugate gradient for A x = b (``gbcg_solve``).

        ``precision``: "fp64", "fp32_ir" (refinement; ``inner_tol`` the inner
        tolerance, default 1e-4) or "fp32_ru" (reliable updates; ``inner_tol``
        the residual reduction between updates, default 0.1); 0 = default.

        ``b`` and ``x`` are float64 CUDA tensors, or numpy arrays (host
        memory; the copies happen inside the call).  ``x`` holds x0 on entry
        (zeros if None) and the solution on return.  Returns (x, SolveInfo).
        """
        opts = _lib.Opts(PRECISIONS[precision], int(max_outer), float(inner_tol), int(wait_timeout_ms),
                         int(max_restarts), VARIANTS[variant], 0)
        info = _lib.Info()
        if _is_tensor(b):
            torch = _torch()
            if x is None:
                x = torch.zeros_like(b)
            if b.is_cuda:
                _check_vec(b, torch.float64, self.n, "b")
                _check_vec(x, torch.float64, self.n, "x")
                stream_h = _stream_handle(stream)
            else:
                b = b.contiguous()
                stream_h = _host_stream(stream)
            bp, xp = b.data_ptr(), x.data_ptr()
        else:
            b = np.ascontiguousarray(b, dtype=np.float64)
            x = np.zeros(self.n) if x is None else x
            if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous):
                raise ValueError("x must be a contiguous float64 numpy array")
            stream_h = _host_stream(stream)
            bp, xp = b.ctypes.data, x.ctypes.data
        rc = self._lib.gbcg_solve(self._h, ctypes.c_void_p(bp), ctypes.c_void_p(xp), float(tol), int(maxit),
                                  ctypes.byref(opts), ctypes.byref(info), stream_h)
        res = SolveInfo(info.iterations, info.outer, _lib.STATUS_NAMES[info.status] if rc == info.status else
                        _lib.STATUS_NAMES[rc], info.rel_res_recursive, info.rel_res_true, info.ms,
                        info.kernel_ms, info.kernel_launches, info.launches)
        if rc != 0 and raise_on_error and rc not in (3,):
            raise GbcgError(rc, "gbcg_solve", _lib.last_error())
        return x, res

    def solve_async(self, b, x, dinfo, tol: float = 1e-10, maxit: int = 0, precision: str = "fp64",
                    inner_tol: float = 0.0, wait_timeout_ms: int = 1000, max_restarts: int = 3,
                    variant: str = "standard", stream=None):
        """``gbcg_solve_async``: the solve enqueued on ``stream`` with no host
        synchronisation (capturable into a CUDA graph).  ``b``, ``x``: float64
        CUDA tensors of length n (x holds x0); ``dinfo``: a CUDA uint8 tensor
        of ``DEVICE_INFO_BYTES`` that receives the result (read it with
        ``device_info``).  Precisions "fp64" and "fp32_ru"."""
        torch = _torch()
        _check_vec(b, torch.float64, self.n, "b")
        _check_vec(x, torch.float64, self.n, "x")
        if not (dinfo.is_cuda and dinfo.dtype == torch.uint8 and dinfo.numel() >= _lib.DEVICE_INFO_BYTES
                and dinfo.is_contiguous() and dinfo.data_ptr() % 8 == 0):
            raise ValueError(f"dinfo must be a contiguous, 8-byte aligned CUDA uint8 tensor of "
                             f"{_lib.DEVICE_INFO_BYTES} bytes")
        opts = _lib.Opts(PRECISIONS[precision], 0, float(inner_tol), int(wait_timeout_ms), int(max_restarts),
                         VARIANTS[variant], 0)
        _lib.check(self._lib.gbcg_solve_async(self._h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                              float(tol), int(maxit), ctypes.byref(opts),
                                              ctypes.c_void_p(dinfo.data_ptr()), _stream_handle(stream)),
                   "gbcg_solve_async")
        return x


def device_info(dinfo) -> SolveInfo:
    """Decodes the result ``Matrix.solve_async`` wrote (copies 32 bytes to the host)."""
    raw = bytes(dinfo[:_lib.DEVICE_INFO_BYTES].cpu().numpy().tobytes())
    status, iterations, outer, _ = np.frombuffer(raw[:16], dtype=np.int32)
    rec, true = np.frombuffer(raw[16:32], dtype=np.float64)
    return SolveInfo(int(iterations), int(outer), _lib.STATUS_NAMES[int(status)], float(rec), float(true), 0.0)


BATCH_INFO_DTYPE = np.dtype([("iterations", np.int32), ("outer", np.int32), ("status", np.int32),
                             ("pad_", np.int32), ("rel_res_true", np.float64)])


def _tuning_dict(t) -> dict:
    return {"threads": t.threads, "cluster": t.cluster, "rows_per_warp": list(t.rows_per_warp),
            "clusters": t.clusters, "from_cache": bool(t.from_cache), "candidates": t.candidates,
            "probe_ms": t.probe_ms}


class Batch:
    """Independent SPD systems of uneven size with up to eight right-hand
    sides each, solved in one persistent launch (``gbcg_batch_create``).

    ``row_off`` (count + 1 int64 row offsets) is a host array; ``ptr``/``idx``/
    ``val`` form one 0-based CSR of the block-diagonal matrix with global
    column numbers (numpy arrays or CUDA tensors).
    """

    def __init__(self, row_off, ptr, idx, val, nrhs: int = 8, tune: bool = True, stream=None):
        lib = _lib.load()
        self._lib = lib
        self._h = ctypes.c_void_p()
        row_off = np.ascontiguousarray(row_off, dtype=np.int64)
        self.count = int(row_off.shape[0]) - 1
        self.n = int(row_off[-1])
        self.nrhs = int(nrhs)
        self.row_off = row_off
        if _is_tensor(ptr):
            torch = _torch()
            ptr = ptr.to(torch.int32).contiguous()
            idx = idx.to(torch.int32).contiguous()
            val = val.to(torch.float64).contiguous()
            mem = _lib.GBCG_DEVICE if ptr.is_cuda else _lib.GBCG_HOST
            args = (ptr.data_ptr(), idx.data_ptr(), val.data_ptr())
        else:
            ptr = np.ascontiguousarray(ptr, dtype=np.int32)
            idx = np.ascontiguousarray(idx, dtype=np.int32)
            val = np.ascontiguousarray(val, dtype=np.float64)
            mem = _lib.GBCG_HOST
            args = (ptr.ctypes.data, idx.ctypes.data, val.ctypes.data)
        keep = (row_off, ptr, idx, val)
        rc = lib.gbcg_batch_create(ctypes.byref(self._h), self.count, ctypes.c_void_p(row_off.ctypes.data),
                                   *[ctypes.c_void_p(a) for a in args], self.nrhs, mem, int(bool(tune)),
                                   _host_stream(stream))
        del keep
        _lib.check(rc, "gbcg_batch_create")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.gbcg_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # pragma: no cover
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def stats(self) -> dict:
        s = _lib.BatchStats()
        _lib.check(self._lib.gbcg_batch_stats(self._h, ctypes.byref(s)), "gbcg_batch_stats")
        return {"n": s.n, "nnz": s.nnz, "device_bytes": s.device_bytes, "iter_bytes_fp32": s.iter_bytes_fp32,
                "iter_bytes_fp64": s.iter_bytes_fp64, "count": s.count, "nrhs": s.nrhs,
                "threads": list(s.threads), "cluster": list(s.cluster),
                "rows_per_warp": [list(r) for r in s.rows_per_warp]}

    def autotune(self, precision: str = "fp32_ir", stream=None) -> dict:
        t = _lib.BatchTuning()
        _lib.check(self._lib.gbcg_batch_autotune(self._h, PRECISIONS[precision], ctypes.byref(t),
                                                 _host_stream(stream)), "gbcg_batch_autotune")
        return _tuning_dict(t)

    def set_tuning(self, precision: str, threads: int, cluster: int, rows_per_warp):
        rpw = list(rows_per_warp) if not isinstance(rows_per_warp, int) else [rows_per_warp] * 8
        t = _lib.BatchTuning(int(threads), int(cluster), (ctypes.c_int32 * 8)(*rpw))
        _lib.check(self._lib.gbcg_batch_set_tuning(self._h, PRECISIONS[precision], ctypes.byref(t)),
                   "gbcg_batch_set_tuning")

    def instance_times(self):
        """(start/end ns [count, 2], inner products [count], residual products [count]) of the last solve."""
        t = np.zeros((self.count, 2), dtype=np.int64)
        p = np.zeros(self.count, dtype=np.int32)
        o = np.zeros(self.count, dtype=np.int32)
        _lib.check(self._lib.gbcg_batch_instance_times(self._h, ctypes.c_void_p(t.ctypes.data),
                                                       ctypes.c_void_p(p.ctypes.data),
                                                       ctypes.c_void_p(o.ctypes.data)), "gbcg_batch_instance_times")
        return t, p, o

    def selftest_group_timeout(self, timeout_ms: int = 50, stream=None) -> int:
        """Bounded-wait self-test of the multi-cluster groups; returns the status code (5 expected)."""
        return self._lib.gbcg_batch_selftest_group_timeout(self._h, int(timeout_ms), _host_stream(stream))

    def solve(self, b, x=None, tol: float = 1e-10, maxit: int = 0, precision: str = "fp32_ir",
              inner_tol: float = 0.0, max_outer: int = 0, fixed_order: bool = False, max_group: int = 0,
              force_group: int = 0, wait_timeout_ms: int = 0, stream=None, raise_on_error: bool = True):
        """Solve every instance for every right-hand side (``gbcg_batch_solve``).

        ``b``, ``x``: (n, nrhs) float64, both CUDA tensors or both numpy
        arrays; ``x`` holds x0 (zeros if None) and receives the solutions.
        Returns (x, infos, report): infos a (count, nrhs) structured array
        (iterations, outer, status, rel_res_true), report a dict.
        """
        opts = _lib.BatchOpts(PRECISIONS[precision], int(max_outer), float(inner_tol), int(bool(fixed_order)),
                              int(max_group), int(force_group), int(wait_timeout_ms))
        infos = np.zeros((self.count, self.nrhs), dtype=BATCH_INFO_DTYPE)
        rep = _lib.BatchReport()
        shape = (self.n, self.nrhs)
        if _is_tensor(b):
            torch = _torch()
            if x is None:
                x = torch.zeros(shape, dtype=torch.float64, device=b.device)
            for t, name in ((b, "b"), (x, "x")):
                if t.dtype != torch.float64 or tuple(t.shape) != shape or not t.is_contiguous():
                    raise ValueError(f"{name} must be a contiguous float64 tensor of shape {shape}")
            stream_h = _stream_handle(stream) if b.is_cuda else _host_stream(stream)
            bp, xp = b.data_ptr(), x.data_ptr()
        else:
            b = np.ascontiguousarray(b, dtype=np.float64).reshape(shape)
            x = np.zeros(shape) if x is None else x
            if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous and x.shape == shape):
                raise ValueError(f"x must be a contiguous float64 numpy array of shape {shape}")
            stream_h = _host_stream(stream)
            bp, xp = b.ctypes.data, x.ctypes.data
        rc = self._lib.gbcg_batch_solve(self._h, ctypes.c_void_p(bp), ctypes.c_void_p(xp), float(tol), int(maxit),
                                        ctypes.byref(opts), ctypes.c_void_p(infos.ctypes.data), ctypes.byref(rep),
                                        stream_h)
        if rc != 0 and raise_on_error and rc not in (2, 3, 4):
            raise GbcgError(rc, "gbcg_batch_solve", _lib.last_error())
        report = {name: getattr(rep, name) for name, _ in _lib.BatchReport._fields_}
        report["status"] = _lib.STATUS_NAMES[rc] if 0 <= rc < len(_lib.STATUS_NAMES) else str(rc)
        return x, infos, report


def _check_vec(t, dtype, n, name):
    if not t.is_cuda or t.dtype != dtype or t.numel() != n or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} CUDA tensor of length {n}")


def _cuda_arg(t, dtype, name):
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous {dtype} CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def grad_values(fmt, ptr, idx, lam, x, index_base: int = 0, out=None, stream=None):
    """dL/d(stored values) = the sampled outer product of the adjoint lambda and
    x on the pattern (``gbcg_grad_values``); CUDA tensors."""
    torch = _torch()
    f = FORMATS[fmt] if isinstance(fmt, str) else int(fmt)
    n, nnz = ptr.numel() - 1, idx.numel()
    if out is None:
        out = torch.empty(nnz, dtype=torch.float64, device=lam.device)
    args = [_cuda_arg(ptr, torch.int32, "ptr"), _cuda_arg(idx, torch.int32, "idx"), int(index_base),
            _cuda_arg(lam, torch.float64, "lambda"), _cuda_arg(x, torch.float64, "x"),
            _cuda_arg(out, torch.float64, "out")]
    _lib.check(_lib.load().gbcg_grad_values(f, n, nnz, *args, _stream_handle(stream)), "gbcg_grad_values")
    return out


def element_grad(pos, w, grad, out=None, stream=None):
    """dL/dcoef per element through the assembly map (``gbcg_element_grad``);
    pos int32 [E, m], w float64 [E, m], grad float64 [nnz]."""
    torch = _torch()
    ne, m = pos.shape
    if out is None:
        out = torch.empty(ne, dtype=torch.float64, device=grad.device)
    _lib.check(_lib.load().gbcg_element_grad(ne, m, _cuda_arg(pos, torch.int32, "pos"),
                                             _cuda_arg(w, torch.float64, "w"), _cuda_arg(grad, torch.float64, "grad"),
                                             _cuda_arg(out, torch.float64, "out"), _stream_handle(stream)),
               "gbcg_element_grad")
    return out


def assemble(tptr, telem, tw, coef, out=None, stream=None):
    """Stored values from element coefficients (``gbcg_assemble``)."""
    torch = _torch()
    nnz = tptr.numel() - 1
    if out is None:
        out = torch.empty(nnz, dtype=torch.float64, device=coef.device)
    _lib.check(_lib.load().gbcg_assemble(nnz, _cuda_arg(tptr, torch.int64, "tptr"),
                                         _cuda_arg(telem, torch.int32, "telem"), _cuda_arg(tw, torch.float64, "tw"),
                                         _cuda_arg(coef, torch.float64, "coef"), _cuda_arg(out, torch.float64, "out"),
                                         _stream_handle(stream)), "gbcg_assemble")
    return out


class Ablation:
    """The paper's 2010 solver structure on device CSR arrays, a measurement
    baseline (``gbcg_ablation_spmv`` / ``gbcg_ablation_solve``): "csr" =
    the thread-per-row kernel, "sym" = SCSR + SCSC with atomics."""

    def __init__(self, fmt, ptr, idx, val, device=None):
        torch = _torch()
        dev = torch.device("cuda") if device is None else torch.device(device)
        self.format = FORMATS[fmt]
        self.ptr = torch.from_numpy(np.ascontiguousarray(ptr, dtype=np.int32)).to(dev)
        self.idx = torch.from_numpy(np.ascontiguousarray(idx, dtype=np.int32)).to(dev)
        self.val = torch.from_numpy(np.ascontiguousarray(val, dtype=np.float64)).to(dev)
        self.n = int(self.ptr.numel()) - 1
        self._lib = _lib.load()

    def _pat(self):
        return (ctypes.c_void_p(self.ptr.data_ptr()), ctypes.c_void_p(self.idx.data_ptr()),
                ctypes.c_void_p(self.val.data_ptr()))

    def spmv(self, x, y=None, stream=None):
        torch = _torch()
        if y is None:
            y = torch.empty(self.n, dtype=torch.float64, device=x.device)
        _lib.check(self._lib.gbcg_ablation_spmv(self.format, self.n, *self._pat(), ctypes.c_void_p(x.data_ptr()),
                                                ctypes.c_void_p(y.data_ptr()), _stream_handle(stream)),
                   "gbcg_ablation_spmv")
        return y

    def solve(self, b, x=None, tol: float = 1e-10, maxit: int = 0, stream=None):
        torch = _torch()
        if x is None:
            x = torch.zeros_like(b)
        info = _lib.Info()
        rc = self._lib.gbcg_ablation_solve(self.format, self.n, *self._pat(), ctypes.c_void_p(b.data_ptr()),
                                           ctypes.c_void_p(x.data_ptr()), float(tol), int(maxit), ctypes.byref(info),
                                           _stream_handle(stream))
        if rc not in (0, 2, 3, 4):
            raise GbcgError(rc, "gbcg_ablation_solve", _lib.last_error())
        return x, SolveInfo(info.iterations, info.outer, _lib.STATUS_NAMES[rc], info.rel_res_recursive,
                            info.rel_res_true, info.ms, info.kernel_ms, info.kernel_launches, info.launches)


def selftest_wait_timeout(ctas: int = 0, timeout_ms: int = 50, stream=None) -> int:
    """Runs the bounded-wait self-test (``gbcg_selftest_wait_timeout``); returns its status code."""
    return _lib.load().gbcg_selftest_wait_timeout(int(ctas), int(timeout_ms), _stream_handle(stream))


def measure_fp64_fma_rate(stream=None) -> float:
    """FP64 FMAs per second of the device (``gbcg_measure_fp64_fma_rate``; measurement only)."""
    out = ctypes.c_double(0.0)
    _lib.check(_lib.load().gbcg_measure_fp64_fma_rate(ctypes.byref(out), _stream_handle(stream)),
               "gbcg_measure_fp64_fma_rate")
    return out.value


from .autograd import Assembly, SparseSolve  # noqa: E402

__all__ = ["Matrix", "Batch", "SparseSolve", "Assembly", "Ablation", "grad_values", "element_grad", "assemble", "SolveInfo", "GbcgError", "build", "selftest_wait_timeout", "measure_fp64_fma_rate", "FORMATS", "PRECISIONS"]
