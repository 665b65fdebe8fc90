"""mspv: sparse matrix-vector multiply over COO / CSR / DIA and conjugate gradient on
GB300 (sm_103a), after "Morpheus unleashed" (arXiv 2304.09511).

A thin binding over libmspv.so (include/mspv.h): every step runs in the library's
CUDA kernels; this module only marshals arguments. PyTorch provides device memory
and the current CUDA stream.

    import paper_2304_09511_gb300 as mspv
    A = mspv.Matrix.from_coo(n, n, rows, cols, vals)        # canonical COO on the GPU
    D = A.convert("dia")                                     # or "csr"; value_type="f32"/"bf16"
    y = D.spmv(x)                                            # x: CUDA float64 tensor
    res = D.cg(b, tol=1e-10, maxit=1000)                     # res.x, res.iters, res.relres
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import MspvError, FORMATS, VALUE_TYPES, load

__all__ = ["Matrix", "CgResult", "MspvError", "load", "csr_vector_width", "fp64_fma_rate", "stream_handle",
           "spmv_coo_noalloc", "selector_train", "selector_predict", "NUM_FEATURES",
           "SELECTOR_PARAMS"]

NUM_FEATURES = _lib.NUM_FEATURES
SELECTOR_PARAMS = _lib.SELECTOR_PARAMS

_FMT_NAMES = {v: k for k, v in FORMATS.items()}
_VT_NAMES = {v: k for k, v in VALUE_TYPES.items()}


def stream_handle(stream=None) -> int:
    """cudaStream_t of a torch stream (default: torch's current stream), as an int."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(a):
    """(address, on_device) of a numpy array or torch tensor, contiguous."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data, 0
    return int(a.data_ptr()), 1 if a.is_cuda else 0


def spmv_coo_noalloc(nrows: int, ncols: int, rows, cols, vals, x, y, stream=None):
    """y = A x for row-sorted COO triplets already on the device (int32 rows/cols,
    float64 vals, CUDA tensors), without any device allocation by the library: the
    kernel's scratch is a fixed array compiled into libmspv.so (at most 201,326,592
    entries). For callers that cannot allocate device memory. Synchronises the stream
    once to validate the indices."""
    for t, dt in ((rows, "int32"), (cols, "int32"), (vals, "float64")):
        if not (t.is_cuda and str(t.dtype).endswith(dt) and t.is_contiguous()):
            raise TypeError("triplets must be contiguous CUDA tensors (int32, int32, float64)")
    _check_vec(x, ncols)
    _check_vec(y, nrows)
    _lib.check(load().mspv_spmv_coo_noalloc(nrows, ncols, int(rows.numel()), rows.data_ptr(),
                                            cols.data_ptr(), vals.data_ptr(), x.data_ptr(),
                                            y.data_ptr(), stream_handle(stream)))
    return y


def fp64_fma_rate(iters: int = 4096, repeats: int = 3, stream=None) -> float:
    """FP64 FMA rate of the current device in TFLOP/s (the FP64 roofline's peak)."""
    out = ctypes.c_double(0.0)
    _lib.check(load().mspv_fp64_fma_rate(int(iters), int(repeats), stream_handle(stream), ctypes.byref(out)))
    return out.value


def csr_vector_width(row_mean: float, row_std: float = 0.0, row_max: int = 0) -> int:
    return int(load().mspv_csr_vector_width(row_mean, row_std, row_max))


@dataclass
class CgResult:
    x: object
    status: int
    iters: int
    relres: float
    outer_iters: int = 0

    @property
    def converged(self) -> bool:
        return self.status == _lib.OK


class Matrix:
    """A handle on a sparse matrix held by libmspv (device memory owned by the handle)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)
        self._shape = None   # (nrows, ncols), fixed for the handle's life; read once

    # -- lifecycle ---------------------------------------------------------------
    @classmethod
    def from_coo(cls, nrows: int, ncols: int, rows, cols, vals, stream=None) -> "Matrix":
        """Triplets as numpy arrays (host) or torch tensors (host or CUDA); int32 indices,
        float64 values. The handle holds the canonical form (sorted, duplicates summed)."""
        lib = load()
        rows, cols, vals = _as_contig(rows, np.int32), _as_contig(cols, np.int32), _as_contig(vals, np.float64)
        n = int(rows.shape[0])
        if not (int(cols.shape[0]) == n == int(vals.shape[0])):
            raise ValueError("rows, cols and vals must have the same length")
        (pr, dr), (pc, dc), (pv, dv) = _ptr(rows), _ptr(cols), _ptr(vals)
        if not (dr == dc == dv):
            raise ValueError("triplet arrays must all be on the host or all on the device")
        out = ctypes.c_void_p()
        s = stream_handle(stream) if dr else 0
        _lib.check(lib.mspv_create_coo(nrows, ncols, n, pr or None, pc or None, pv or None, dr, s,
                                       ctypes.byref(out)))
        return cls(out.value)

    def convert(self, fmt: str, value_type: str = "f64", stream=None) -> "Matrix":
        lib = load()
        out = ctypes.c_void_p()
        _lib.check(lib.mspv_convert(self._h, FORMATS[fmt], VALUE_TYPES[value_type],
                                    _stream_or_null(stream), ctypes.byref(out)))
        return Matrix(out.value)

    def close(self):
        if self._h is not None and self._h.value:
            load().mspv_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- description ---------------------------------------------------------------
    @property
    def info(self) -> dict:
        inf = _lib.MatrixInfo()
        _lib.check(load().mspv_info(self._h, ctypes.byref(inf)))
        d = {name: getattr(inf, name) for name, _ in _lib.MatrixInfo._fields_}
        d["format"] = _FMT_NAMES[d["format"]]
        d["value_type"] = _VT_NAMES[d["value_type"]]
        return d

    @property
    def shape(self):
        if self._shape is None:
            i = self.info
            self._shape = (i["nrows"], i["ncols"])
        return self._shape

    def export(self) -> dict:
        """Stored structure copied to host numpy arrays (values widened to float64)."""
        inf = self.info
        fmt, nnz, nr = inf["format"], inf["nnz"], inf["nrows"]
        if fmt == "coo":
            a0, a1, nv = np.empty(max(nnz, 1), np.int32), np.empty(max(nnz, 1), np.int32), nnz
        elif fmt == "csr":
            a0, a1, nv = np.empty(nr + 1, np.int32), np.empty(max(nnz, 1), np.int32), nnz
        else:
            a0, a1, nv = np.empty(max(inf["ndiags"], 1), np.int32), None, inf["ndiags"] * inf["npad"]
        v = np.empty(max(nv, 1), np.float64)
        _lib.check(load().mspv_export(self._h, a0.ctypes.data, None if a1 is None else a1.ctypes.data,
                                      v.ctypes.data, _stream_or_null(None)))
        if fmt == "coo":
            return {"rows": a0[:nnz], "cols": a1[:nnz], "vals": v[:nv]}
        if fmt == "csr":
            return {"irp": a0, "cols": a1[:nnz], "vals": v[:nv]}
        return {"doff": a0[:inf["ndiags"]], "vals": v[:nv], "npad": inf["npad"]}

    # -- compute ---------------------------------------------------------------------
    def spmv(self, x, y=None, stream=None):
        """y = A x on the device (float64 CUDA tensors). Asynchronous on the stream."""
        import torch
        nr, nc = self.shape
        _check_vec(x, nc)
        if y is None:
            y = torch.empty(nr, dtype=torch.float64, device=x.device)
        _check_vec(y, nr)
        _lib.check(load().mspv_spmv(self._h, x.data_ptr(), y.data_ptr(), stream_handle(stream)))
        return y

    def cg(self, b, x=None, tol: float = 1e-10, maxit: int = 1000, stream=None) -> CgResult:
        """Unpreconditioned CG from x (zeros if None); x is overwritten in place."""
        import torch
        n = self.shape[0]
        _check_vec(b, n)
        if x is None:
            x = torch.zeros(n, dtype=torch.float64, device=b.device)
        _check_vec(x, n)
        it = ctypes.c_int32(0)
        rr = ctypes.c_double(0.0)
        st = load().mspv_cg_solve(self._h, b.data_ptr(), x.data_ptr(), float(tol), int(maxit),
                                  stream_handle(stream), ctypes.byref(it), ctypes.byref(rr))
        _lib.check(st, allow=(_lib.ENOTCONV, _lib.EBREAKDOWN))
        return CgResult(x, st, it.value, rr.value)

    def spmv_f32(self, x, y=None, stream=None):
        """y = A x in FP32 arithmetic for FP32/BF16-valued handles (float32 CUDA tensors,
        16-byte aligned)."""
        import torch
        nr, nc = self.shape
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float32 and x.numel() == nc):
            raise TypeError("x must be a CUDA float32 tensor with ncols entries")
        if y is None:
            y = torch.empty(nr, dtype=torch.float32, device=x.device)
        _lib.check(load().mspv_spmv_f32(self._h, x.data_ptr(), y.data_ptr(), stream_handle(stream)))
        return y

    def spmv_add(self, x, y, stream=None):
        """y += A x (device float64 tensors); returns y."""
        _check_vec(x, self.shape[1])
        _check_vec(y, self.shape[0])
        _lib.check(load().mspv_spmv_add(self._h, x.data_ptr(), y.data_ptr(), stream_handle(stream)))
        return y

    def split_columns(self, ncols_local: int, stream=None):
        """(local, remote): entries with column < ncols_local, and the rest with columns
        renumbered from 0; both new COO handles."""
        lo, re = ctypes.c_void_p(), ctypes.c_void_p()
        _lib.check(load().mspv_split_columns(self._h, int(ncols_local), stream_handle(stream),
                                             ctypes.byref(lo), ctypes.byref(re)))
        return Matrix(lo.value), Matrix(re.value)

    def features(self, stream=None) -> np.ndarray:
        """The ten FP32 sparsity features of the stored structure (mspv_features)."""
        out = np.zeros(NUM_FEATURES, dtype=np.float32)
        _lib.check(load().mspv_features(self._h, out.ctypes.data, stream_handle(stream)))
        return out

    def tune_format(self, reps: int = 10, stream=None):
        """Run-first tuner: (best format name, {format: ms per SpMV}); inf where DIA is not
        built (not square, or over its fill cap)."""
        ms = np.zeros(3, dtype=np.float64)
        best = ctypes.c_int(0)
        _lib.check(load().mspv_tune_format(self._h, int(reps), stream_handle(stream), ms.ctypes.data,
                                           ctypes.byref(best)))
        return _FMT_NAMES[best.value], {_FMT_NAMES[k]: float(ms[k]) for k in range(3)}

    def select_format(self, params=None, stream=None) -> str:
        """Format chosen by the MLP `params` (float32[SELECTOR_PARAMS]), or by the run-first
        tuner when params is None."""
        best = ctypes.c_int(0)
        pp = None
        if params is not None:
            params = _params_array(params)
            pp = params.ctypes.data
        _lib.check(load().mspv_select_format(self._h, pp, stream_handle(stream), ctypes.byref(best)))
        return _FMT_NAMES[best.value]

    def cg_ir(self, low: "Matrix", b, x=None, tol: float = 1e-10, inner_tol: float = 1e-6,
              max_outer: int = 50, maxit_inner: int = 10000, inner_fp32: int = 0,
              stream=None) -> CgResult:
        """Iterative refinement: FP64 residuals on self, inner CG on `low` (e.g. BF16 values),
        in FP64 arithmetic (inner_fp32=0), in FP32 arithmetic (1), or one FP32 CG with
        reliable updates (2; see cg_ru)."""
        import torch
        n = self.shape[0]
        _check_vec(b, n)
        if x is None:
            x = torch.zeros(n, dtype=torch.float64, device=b.device)
        _check_vec(x, n)
        oi, ii, rr = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0.0)
        st = load().mspv_cg_solve_ir(self._h, low._h, b.data_ptr(), x.data_ptr(), float(tol),
                                     float(inner_tol), int(max_outer), int(maxit_inner), int(inner_fp32),
                                     stream_handle(stream), ctypes.byref(oi), ctypes.byref(ii),
                                     ctypes.byref(rr))
        _lib.check(st, allow=(_lib.ENOTCONV, _lib.EBREAKDOWN))
        return CgResult(x, st, ii.value, rr.value, outer_iters=oi.value)

    def cg_ru(self, low: "Matrix", b, x=None, tol: float = 1e-10, delta: float = 0.0,
              max_updates: int = 100, maxit: int = 10000, stream=None) -> CgResult:
        """Mixed precision with reliable updates: one FP32 CG on `low` (FP32 or BF16 values)
        whose residual is replaced by the FP64 residual of self when it has fallen by `delta`
        (0 = the library's default for the value type). iters counts FP32 iterations and
        outer_iters the updates."""
        return self.cg_ir(low, b, x, tol=tol, inner_tol=delta, max_outer=max_updates, maxit_inner=maxit,
                          inner_fp32=2, stream=stream)


def _params_array(params) -> np.ndarray:
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.shape != (SELECTOR_PARAMS,):
        raise ValueError(f"selector parameters must have {SELECTOR_PARAMS} entries")
    return p


def _features_array(X) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float32)
    if X.ndim != 2 or X.shape[1] != NUM_FEATURES:
        raise ValueError(f"features must be an (N, {NUM_FEATURES}) array")
    return X


def selector_train(X, y, epochs: int = 200, lr: float = 1e-3, seed: int = 0, stream=None) -> np.ndarray:
    """Train the format-selector MLP on the GPU (mspv_selector_train); returns the
    float32[SELECTOR_PARAMS] parameter vector."""
    X = _features_array(X)
    y = np.ascontiguousarray(y, dtype=np.int32)
    if y.shape != (X.shape[0],):
        raise ValueError("one label per feature row")
    out = np.zeros(SELECTOR_PARAMS, dtype=np.float32)
    _lib.check(load().mspv_selector_train(X.ctypes.data, y.ctypes.data, int(X.shape[0]), int(epochs),
                                          float(lr), int(seed), out.ctypes.data, stream_handle(stream)))
    return out


def selector_predict(params, X, stream=None) -> np.ndarray:
    """Predicted format index (0 COO, 1 CSR, 2 DIA) per feature row (mspv_selector_predict)."""
    params = _params_array(params)
    X = _features_array(X)
    out = np.zeros(X.shape[0], dtype=np.int32)
    _lib.check(load().mspv_selector_predict(params.ctypes.data, X.ctypes.data, int(X.shape[0]),
                                            out.ctypes.data, stream_handle(stream)))
    return out


def _as_contig(a, dtype):
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=dtype)
    import torch
    tdt = {np.int32: torch.int32, np.float64: torch.float64}[dtype]
    return a.to(tdt).contiguous()


def _check_vec(v, n):
    import torch
    if not isinstance(v, torch.Tensor) or not v.is_cuda or v.dtype != torch.float64:
        raise TypeError("vectors must be CUDA float64 tensors")
    if v.numel() != n or not v.is_contiguous():
        raise ValueError(f"vector must be contiguous with {n} entries (got {v.numel()})")


def _stream_or_null(stream):
    try:
        import torch
        if torch.cuda.is_available():
            return stream_handle(stream)
    except Exception:
        pass
    return None
