"""Host-side checks of the C ABI that need no GPU: the library builds and loads,
exports every entry point include/mspv.h declares, and rejects bad arguments on the
host before any device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2304_09511_gb300 import build_lib
    build_lib.build()
    import paper_2304_09511_gb300 as mspv
    return mspv.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mspv.h")).read()
    return re.findall(r"MSPV_API\s+[^;(]*?\b(mspv_\w+)\s*\(", src)


def test_header_declares_the_boundary():
    names = set(declared_functions())
    for required in ("mspv_create_coo", "mspv_convert", "mspv_spmv", "mspv_cg_solve",
                     "mspv_destroy", "mspv_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2304_09511_gb300 import _lib
    assert set(declared_functions()) == set(_lib.SIGNATURES)


def test_status_strings(lib):
    from paper_2304_09511_gb300 import _lib
    for code, name in enumerate(_lib.STATUS_NAMES):
        assert lib.mspv_status_string(code).decode() == name
    assert lib.mspv_version() >= 100


@pytest.mark.parametrize("mean,expect", [(0.0, 4), (1.0, 4), (27.0, 4), (48.0, 4), (60.0, 8), (96.0, 8),
                                         (150.0, 16), (192.5, 32), (20000.0, 32)])
def test_csr_vector_width_heuristic(lib, mean, expect, monkeypatch):
    monkeypatch.delenv("MSPV_CSR_VEC", raising=False)
    assert lib.mspv_csr_vector_width(mean, 0.0, 0) == expect


def test_csr_vector_width_override(lib, monkeypatch):
    monkeypatch.setenv("MSPV_CSR_VEC", "8")
    assert lib.mspv_csr_vector_width(27.0, 0.0, 27) == 8
    monkeypatch.setenv("MSPV_CSR_VEC", "0")
    assert lib.mspv_csr_vector_width(900.0, 0.0, 900) == 0
    monkeypatch.setenv("MSPV_CSR_VEC", "7")   # not a power of two: ignored
    assert lib.mspv_csr_vector_width(27.0, 0.0, 27) == 4


def _create(lib, nrows, ncols, rows, cols, vals, nnz=None):
    n = len(rows) if nnz is None else nnz
    R = (ctypes.c_int32 * max(len(rows), 1))(*rows)
    C = (ctypes.c_int32 * max(len(cols), 1))(*cols)
    V = (ctypes.c_double * max(len(vals), 1))(*vals)
    out = ctypes.c_void_p(1234)
    st = lib.mspv_create_coo(nrows, ncols, n, R, C, V, 0, None, ctypes.byref(out))
    return st, out.value


def test_create_rejects_bad_host_triplets(lib):
    from paper_2304_09511_gb300 import _lib
    st, h = _create(lib, 3, 3, [0, 3], [0, 0], [1.0, 2.0])
    assert st == _lib.EINVAL and h is None
    assert b"outside" in lib.mspv_last_error()
    st, _ = _create(lib, 3, 3, [0, 1], [0, -1], [1.0, 2.0])
    assert st == _lib.EINVAL
    st, _ = _create(lib, -1, 3, [], [], [])
    assert st == _lib.EINVAL
    st, _ = _create(lib, 0, 0, [0], [0], [1.0])
    assert st == _lib.EINVAL
    st, _ = _create(lib, 3, 3, [0], [0], [1.0], nnz=1 << 31)
    assert st == _lib.ETOOBIG
    assert lib.mspv_create_coo(3, 3, 0, None, None, None, 0, None, None) == _lib.EINVAL


def test_null_handles_are_rejected(lib):
    from paper_2304_09511_gb300 import _lib
    out = ctypes.c_void_p()
    assert lib.mspv_convert(None, 1, 0, None, ctypes.byref(out)) == _lib.EINVAL
    assert lib.mspv_spmv(None, None, None, None) == _lib.EINVAL
    assert lib.mspv_cg_solve(None, None, None, 1e-10, 10, None, None, None) == _lib.EINVAL
    info = _lib.MatrixInfo()
    assert lib.mspv_info(None, ctypes.byref(info)) == _lib.EINVAL
    lib.mspv_destroy(None)   # no-op


def test_product_path_has_no_oracle_or_fallback():
    """The package never imports the oracle and has no CPU compute path."""
    pkg = os.path.join(ROOT, "paper_2304_09511_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text, f


def test_selector_entry_points_reject_bad_host_input(lib):
    """Validation happens on the host, before any device work."""
    import numpy as np
    from paper_2304_09511_gb300 import _lib
    X = np.zeros((4, _lib.NUM_FEATURES), dtype=np.float32)
    params = np.zeros(_lib.SELECTOR_PARAMS, dtype=np.float32)
    bad = np.array([0, 1, 3, 2], dtype=np.int32)
    assert lib.mspv_selector_train(X.ctypes.data, bad.ctypes.data, 4, 1, 1e-3, 0, params.ctypes.data,
                                   None) == _lib.EINVAL
    assert b"label 3" in lib.mspv_last_error()
    ok = np.array([0, 1, 2, 2], dtype=np.int32)
    assert lib.mspv_selector_train(X.ctypes.data, ok.ctypes.data, 0, 1, 1e-3, 0, params.ctypes.data,
                                   None) == _lib.EINVAL
    assert lib.mspv_selector_train(X.ctypes.data, ok.ctypes.data, 4, 1, 0.0, 0, params.ctypes.data,
                                   None) == _lib.EINVAL
    assert lib.mspv_selector_train(None, ok.ctypes.data, 4, 1, 1e-3, 0, params.ctypes.data,
                                   None) == _lib.EINVAL
    out = np.zeros(4, dtype=np.int32)
    assert lib.mspv_selector_predict(params.ctypes.data, X.ctypes.data, -1, out.ctypes.data,
                                     None) == _lib.EINVAL
    assert lib.mspv_selector_predict(None, X.ctypes.data, 4, out.ctypes.data, None) == _lib.EINVAL
    fmt = ctypes.c_int(0)
    ms = np.zeros(3)
    assert lib.mspv_features(None, X.ctypes.data, None) == _lib.EINVAL
    assert lib.mspv_tune_format(None, 10, None, ms.ctypes.data, ctypes.byref(fmt)) == _lib.EINVAL
    assert lib.mspv_select_format(None, None, None, ctypes.byref(fmt)) == _lib.EINVAL
