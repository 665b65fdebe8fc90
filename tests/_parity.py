"""Shared helpers for the GPU parity tests (CUDA path vs the CPU oracle)."""
import numpy as np

U = 2.0 ** -53


def spmv_tolerance(O, x, oracle):
    """Per-row bound tol_i * sum_j |a_ij x_j| with tol_i = max(1e-13, 2 (k_i + 2) u) for a
    row of k_i stored entries: two summation orders of the same k products (with or
    without fused multiply-adds) each lie within gamma_{k+1} sum |a x| of the exact
    value. 1e-13 is the floor stated for FP64 SpMV parity."""
    absA = oracle.Matrix(O.fmt, O.nrows, O.ncols, O.nnz, ai=O.ai, aj=O.aj, irp=O.irp,
                         av=np.abs(O.av), doff=O.doff, npad=O.npad)
    scale = oracle.spmv(absA, np.abs(x))
    if O.fmt == oracle.DIA:
        k = np.full(O.nrows, max(O.ndiags, 1))
    elif O.fmt == oracle.CSR:
        k = np.diff(O.irp)
    else:
        k = np.bincount(O.ai, minlength=O.nrows)[:O.nrows]
    tol = np.maximum(1e-13, 2.0 * (k + 2) * U)
    return tol * scale


def assert_spmv_parity(y_gpu, O, x, oracle):
    want = oracle.spmv(O, x)
    bound = spmv_tolerance(O, x, oracle)
    err = np.abs(y_gpu - want)
    unwritten = np.nonzero(np.isnan(y_gpu) & ~np.isnan(want))[0]
    assert unwritten.size == 0, f"{unwritten.size} rows NaN on the GPU, first {unwritten[0]}"
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, (f"{bad.size} rows out of tolerance; first row {bad[0]}: "
                           f"gpu {y_gpu[bad[0]]!r} oracle {want[bad[0]]!r} bound {bound[bad[0]]:.3e}")


def assert_structure_equal(M, O, oracle):
    """Bit-exact comparison of the handle's stored structure with the oracle's."""
    e = M.export()
    if O.fmt == oracle.COO:
        assert np.array_equal(e["rows"], O.ai)
        assert np.array_equal(e["cols"], O.aj)
        assert np.array_equal(e["vals"].view(np.uint64), O.av.view(np.uint64))
    elif O.fmt == oracle.CSR:
        assert np.array_equal(e["irp"], O.irp)
        assert np.array_equal(e["cols"], O.aj)
        assert np.array_equal(e["vals"].view(np.uint64), O.av.view(np.uint64))
    else:
        assert e["npad"] == O.npad
        assert np.array_equal(e["doff"], O.doff)
        assert np.array_equal(e["vals"].view(np.uint64), O.av.view(np.uint64))
