"""FP64 CPU oracle for the SpMV / CG hot path of arXiv 2304.09511.

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It loads ``liboracle.so``,
compiled from ``oracle.c`` (plain C11, ``-ffp-contract=off``), and shares no code
with the CUDA library in ``paper_2304_09511_gb300``.

Functions and the passages they follow:
  canonicalize   COO storage, Sec. II-B-1 (stable (row, col) sort, duplicates summed
                 in input order)
  coo_to_csr     CSR, Sec. II-B-2
  coo_to_dia     DIA, Sec. II-B-3 (diagonal-major AV[j*npad + i], npad = ceil(n/32)*32)
  spmv_coo/csr/dia   Algorithms 1, 2, 3
  round_values   FP32 / BF16 storage rounding (round to nearest even from FP64)
  cg             unpreconditioned CG as run in the paper's HPCG experiments (Sec. VI)
  cg_ir          FP64 iterative refinement around a low-precision inner CG (not in
                 the paper; pinned by the dense stationary recursion
                 x += Alo^-1 (b - A64 x) step by step, its contraction bound and its
                 final FP64 residual)
  cg_ru          one low-precision CG with reliable updates of its residual from
                 FP64 (not in the paper; pinned by finite termination, by equality
                 with cg when both matrices are equal, and by its final residual)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

COO, CSR, DIA = 0, 1, 2
F64, F32, BF16 = 0, 1, 2
OK, NOTCONV, BREAKDOWN = 0, 1, 2
_FMT = {"coo": COO, "csr": CSR, "dia": DIA}
_VT = {"f64": F64, "f32": F32, "bf16": BF16}


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, no -march, no fast-math)."""
    stale = (not os.path.exists(_LIB)
             or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                        "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")


def build_timing(force: bool = False) -> str:
    """Compile the CPU-baseline timing copy, liboracle_omp.so: the same source with -O3 and
    OpenMP (row loops of the CSR / DIA SpMV and CG's vector loops on all host cores, dot
    products as reductions). Not used for parity. No -march flag: the library builds the
    same on x86-64 and AArch64 hosts."""
    stale = (not os.path.exists(_LIB_OMP)
             or os.path.getmtime(_LIB_OMP) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB_OMP + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O3", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                        "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


class timing_build:
    """Context manager: the oracle functions run on the OpenMP timing copy inside it."""

    def __enter__(self):
        global _lib
        self._saved = _lib
        _lib = _configure(ctypes.CDLL(build_timing()))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def threads() -> int:
    """Threads the loaded oracle library uses (1 for the parity build)."""
    return int(_L().orc_threads())


class _Mat(ctypes.Structure):
    _fields_ = [("fmt", ctypes.c_int32), ("nrows", ctypes.c_int32), ("ncols", ctypes.c_int32),
                ("nnz", ctypes.c_int64), ("ai", ctypes.c_void_p), ("aj", ctypes.c_void_p),
                ("irp", ctypes.c_void_p), ("av", ctypes.c_void_p), ("ndiags", ctypes.c_int32),
                ("doff", ctypes.c_void_p), ("npad", ctypes.c_int32)]


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


def _configure(lib):
    i32, i64, dbl, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    sig = {
        "orc_coo_canonicalize": (i64, [i32, i32, i64, vp, vp, vp, vp, vp, vp]),
        "orc_coo_to_csr": (None, [i32, i64, vp, vp]),
        "orc_csr_to_coo": (None, [i32, vp, vp]),
        "orc_dia_offsets": (i32, [i32, i64, vp, vp, vp]),
        "orc_coo_to_dia": (None, [i32, i64, vp, vp, vp, i32, vp, i32, vp]),
        "orc_dia_to_coo": (i64, [i32, i32, vp, i32, vp, vp, vp, vp]),
        "orc_spmv_coo": (None, [i32, i64, vp, vp, vp, vp, vp]),
        "orc_spmv_csr": (None, [i32, vp, vp, vp, vp, vp]),
        "orc_spmv_dia": (None, [i32, i32, vp, i32, vp, vp, vp]),
        "orc_round_values": (None, [i64, vp, i32, vp]),
        "orc_cg": (i32, [vp, vp, vp, dbl, i32, vp, vp, vp, vp, vp]),
        "orc_cg_ir": (i32, [vp, vp, vp, vp, dbl, dbl, i32, i32, vp, vp, vp]),
        "orc_cg_ru": (i32, [vp, vp, vp, vp, dbl, dbl, i32, i32, vp, vp, vp]),
        "orc_threads": (i32, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def npad_of(n: int) -> int:
    """Padded row count of the DIA value array: n rounded up to a multiple of 32."""
    return ((n + 31) // 32) * 32


class Matrix:
    """A matrix held by the oracle in one format; arrays are numpy, FP64 values."""

    def __init__(self, fmt, nrows, ncols, nnz, ai=None, aj=None, irp=None, av=None,
                 doff=None, npad=0):
        self.fmt, self.nrows, self.ncols, self.nnz = fmt, int(nrows), int(ncols), int(nnz)
        self.ai, self.aj, self.irp, self.av, self.doff, self.npad = ai, aj, irp, av, doff, int(npad)

    @property
    def ndiags(self) -> int:
        return 0 if self.doff is None else int(self.doff.size)

    def _struct(self) -> _Mat:
        return _Mat(self.fmt, self.nrows, self.ncols, self.nnz, _p(self.ai), _p(self.aj),
                    _p(self.irp), _p(self.av), self.ndiags, _p(self.doff), self.npad)


def canonicalize(nrows, ncols, rows, cols, vals) -> Matrix:
    """Canonical COO: stable sort by (row, col), duplicates summed in input order."""
    rows, cols, vals = _i32(rows), _i32(cols), _f64(vals)
    nnz = rows.size
    o_r = np.empty(max(nnz, 1), np.int32)
    o_c = np.empty(max(nnz, 1), np.int32)
    o_v = np.empty(max(nnz, 1), np.float64)
    m = _L().orc_coo_canonicalize(nrows, ncols, nnz, _p(rows), _p(cols), _p(vals),
                                  _p(o_r), _p(o_c), _p(o_v))
    if m < 0:
        raise ValueError("oracle: index out of range or allocation failure")
    return Matrix(COO, nrows, ncols, m, ai=o_r[:m].copy(), aj=o_c[:m].copy(), av=o_v[:m].copy())


def coo_to_csr(A: Matrix) -> Matrix:
    irp = np.empty(A.nrows + 1, np.int32)
    _L().orc_coo_to_csr(A.nrows, A.nnz, _p(A.ai), _p(irp))
    return Matrix(CSR, A.nrows, A.ncols, A.nnz, aj=A.aj.copy(), irp=irp, av=A.av.copy())


def csr_to_coo(A: Matrix) -> Matrix:
    rows = np.empty(max(A.nnz, 1), np.int32)
    _L().orc_csr_to_coo(A.nrows, _p(A.irp), _p(rows))
    return Matrix(COO, A.nrows, A.ncols, A.nnz, ai=rows[:A.nnz].copy(), aj=A.aj.copy(),
                  av=A.av.copy())


def coo_to_dia(A: Matrix) -> Matrix:
    if A.nrows != A.ncols:
        raise ValueError("oracle: DIA needs a square matrix")
    n = A.nrows
    doff = np.empty(max(2 * n - 1, 1), np.int32)
    nd = _L().orc_dia_offsets(n, A.nnz, _p(A.ai), _p(A.aj), _p(doff))
    doff = doff[:nd].copy()
    npad = npad_of(n)
    av = np.empty(max(nd * npad, 1), np.float64)
    _L().orc_coo_to_dia(n, A.nnz, _p(A.ai), _p(A.aj), _p(A.av), nd, _p(doff), npad, _p(av))
    return Matrix(DIA, n, n, A.nnz, av=av[:nd * npad].copy(), doff=doff, npad=npad)


def dia_to_coo(A: Matrix) -> Matrix:
    cap = max(A.ndiags * A.nrows, 1)
    r = np.empty(cap, np.int32)
    c = np.empty(cap, np.int32)
    v = np.empty(cap, np.float64)
    m = _L().orc_dia_to_coo(A.nrows, A.ndiags, _p(A.doff), A.npad, _p(A.av), _p(r), _p(c), _p(v))
    return Matrix(COO, A.nrows, A.ncols, m, ai=r[:m].copy(), aj=c[:m].copy(), av=v[:m].copy())


def split_columns(A: Matrix, ncols_local: int):
    """Local/remote split of a canonical COO matrix (the per-process split of the paper's
    distributed HPCG, Sec. VI): local = the entries with column < ncols_local, remote = the
    others with ncols_local subtracted from their columns; entry order is kept, so both
    stay canonical. A x = local x[:ncols_local] + remote x[ncols_local:]."""
    if A.fmt != COO:
        raise ValueError("oracle: split a COO matrix")
    m = A.aj < ncols_local
    loc = Matrix(COO, A.nrows, ncols_local, int(m.sum()), ai=A.ai[m].copy(), aj=A.aj[m].copy(),
                 av=A.av[m].copy())
    rem = Matrix(COO, A.nrows, A.ncols - ncols_local, int((~m).sum()), ai=A.ai[~m].copy(),
                 aj=(A.aj[~m] - ncols_local).astype(np.int32), av=A.av[~m].copy())
    return loc, rem


def round_values(vals, value_type: str) -> np.ndarray:
    v = _f64(vals)
    out = np.empty_like(v)
    _L().orc_round_values(v.size, _p(v), _VT[value_type], _p(out))
    return out


def with_values(A: Matrix, value_type: str) -> Matrix:
    """The same matrix with its stored values rounded to FP32 or BF16 (held as FP64)."""
    return Matrix(A.fmt, A.nrows, A.ncols, A.nnz, ai=A.ai, aj=A.aj, irp=A.irp,
                  av=round_values(A.av, value_type), doff=A.doff, npad=A.npad)


def convert(A: Matrix, fmt: str) -> Matrix:
    if fmt == "coo":
        return A
    return coo_to_csr(A) if fmt == "csr" else coo_to_dia(A)


def spmv(A: Matrix, x) -> np.ndarray:
    x = _f64(x)
    y = np.empty(max(A.nrows, 1), np.float64)
    L = _L()
    if A.fmt == COO:
        L.orc_spmv_coo(A.nrows, A.nnz, _p(A.ai), _p(A.aj), _p(A.av), _p(x), _p(y))
    elif A.fmt == CSR:
        L.orc_spmv_csr(A.nrows, _p(A.irp), _p(A.aj), _p(A.av), _p(x), _p(y))
    else:
        L.orc_spmv_dia(A.nrows, A.ndiags, _p(A.doff), A.npad, _p(A.av), _p(x), _p(y))
    return y[:A.nrows]


def cg(A: Matrix, b, x0=None, tol=1e-10, maxit=1000, xstar=None):
    """Returns (x, status, iters, relres, res_hist, aerr_hist)."""
    n = A.nrows
    b = _f64(b)
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    hist = np.zeros(maxit + 1)
    aerr = np.zeros(maxit + 1) if xstar is not None else None
    xs = None if xstar is None else _f64(xstar)
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    m = A._struct()
    st = _L().orc_cg(ctypes.addressof(m), _p(b), _p(x), tol, maxit, ctypes.addressof(it),
                     ctypes.addressof(rr), _p(hist), _p(xs), _p(aerr))
    k = it.value
    return (x, st, k, rr.value, hist[:k + 1], None if aerr is None else aerr[:k + 1])


def cg_ir(A64: Matrix, Alo: Matrix, b, x0=None, tol=1e-10, inner_tol=1e-6, max_outer=50,
          maxit_inner=10000):
    """Returns (x, status, outer_iters, inner_iters_total, relres)."""
    n = A64.nrows
    b = _f64(b)
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    oi = ctypes.c_int32(0)
    ii = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    m64, mlo = A64._struct(), Alo._struct()
    st = _L().orc_cg_ir(ctypes.addressof(m64), ctypes.addressof(mlo), _p(b), _p(x), tol,
                        inner_tol, max_outer, maxit_inner, ctypes.addressof(oi),
                        ctypes.addressof(ii), ctypes.addressof(rr))
    return x, st, oi.value, ii.value, rr.value


def cg_ru(A64: Matrix, Alo: Matrix, b, x0=None, tol=1e-10, delta=1e-2, max_updates=100,
          maxit=10000):
    """Returns (x, status, updates, iters, relres)."""
    n = A64.nrows
    b = _f64(b)
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    nu = ctypes.c_int32(0)
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    m64, mlo = A64._struct(), Alo._struct()
    st = _L().orc_cg_ru(ctypes.addressof(m64), ctypes.addressof(mlo), _p(b), _p(x), tol, delta,
                        max_updates, maxit, ctypes.addressof(nu),
                        ctypes.addressof(it), ctypes.addressof(rr))
    return x, st, nu.value, it.value, rr.value
