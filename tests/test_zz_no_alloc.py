"""The allocation-free COO SpMV entry point (mspv_spmv_coo_noalloc), called through the
C ABI, against the regular entry point (create_coo + spmv) on the same matrix and against
the CPU oracle's Algorithm 1.

It serves callers that cannot allocate device memory (their memory is reserved or
budgeted by their own allocator); its scratch is a fixed array inside the library, so
two calls in a row must both be right -- the second one sees the first one's leftovers.
This file is collected last on purpose."""
import numpy as np
import pytest

import synth
from _parity import assert_spmv_parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

U = 2.0 ** -53


@pytest.fixture(scope="module")
def mspv():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2304_09511_gb300 as m
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return m


def _matrix(seed):
    """Unsorted triplets with duplicates, empty rows and a 9000-entry row crossing
    several 3072-entry windows."""
    n = 30000
    rng = np.random.default_rng(seed)
    r, c, v = synth.random_coo(n, n, 400_000, seed, dup_frac=0.05, empty_rows=3000)
    r = np.concatenate([r, np.full(9000, 12345, np.int32)])
    c = np.concatenate([c, rng.integers(0, n, 9000).astype(np.int32)])
    v = np.concatenate([v, rng.uniform(-1, 1, 9000)])
    return n, r, c, v


def _bound(mspv, n, e, x):
    """Per-row tolerance of the parity tests: max(1e-13, 2 (k + 2) u) * sum_j |a_ij x_j|,
    doubled because both results carry it."""
    dev = torch.device("cuda")
    Aabs = mspv.Matrix.from_coo(n, n, torch.from_numpy(e["rows"]).to(dev), torch.from_numpy(e["cols"]).to(dev),
                                torch.from_numpy(np.abs(e["vals"])).to(dev))
    scale = Aabs.spmv(x.abs()).cpu().numpy()
    k = np.bincount(e["rows"], minlength=n)[:n]
    return 2.0 * np.maximum(1e-13, 2.0 * (k + 2) * U) * scale


def test_noalloc_matches_regular_entry_point_twice(mspv):
    n, r, c, v = _matrix(17)
    dev = torch.device("cuda")
    A = mspv.Matrix.from_coo(n, n, r, c, v)      # regular entry point: canonical COO
    e = A.export()
    rows = torch.from_numpy(e["rows"]).to(dev)
    cols = torch.from_numpy(e["cols"]).to(dev)
    vals = torch.from_numpy(e["vals"]).to(dev)
    for call, seed in enumerate((1, 2)):
        x = torch.from_numpy(synth.uniform_x(n, seed) * 2 - 1).to(dev)
        want = A.spmv(x).cpu().numpy()
        y = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)   # every row must be written
        mspv.spmv_coo_noalloc(n, n, rows, cols, vals, x, y)
        got = y.cpu().numpy()
        bound = _bound(mspv, n, e, x)
        err = np.abs(got - want)
        assert np.all(err <= bound), f"call {call}: max excess {np.max(err - bound):.3e}"


def _oracle_check(orc, n, rows, cols, vals, x, got):
    """The oracle's Algorithm 1 on the same triplets, at the single-result parity bound
    max(1e-13, 2 (k + 2) u) * sum_j |a_ij x_j| of the other SpMV tests."""
    O = orc.Matrix(orc.COO, n, n, rows.size, ai=rows.astype(np.int32), aj=cols.astype(np.int32),
                   av=vals.astype(np.float64))
    assert_spmv_parity(got, O, x, orc)


def test_noalloc_matches_oracle_twice(mspv, orc):
    """Row-sorted triplets with duplicates and empty rows, checked against the CPU oracle
    directly on two calls in a row (the second sees the first call's scratch)."""
    n, r, c, v = _matrix(23)
    order = np.argsort(r, kind="stable")            # rows non-decreasing, columns in input order
    r, c, v = r[order], c[order], v[order]
    dev = torch.device("cuda")
    rows, cols, vals = (torch.from_numpy(a).to(dev) for a in (r, c, v))
    for seed in (3, 4):
        xh = synth.uniform_x(n, seed) * 2 - 1
        y = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
        mspv.spmv_coo_noalloc(n, n, rows, cols, vals, torch.from_numpy(xh).to(dev), y)
        _oracle_check(orc, n, r, c, v, xh, y.cpu().numpy())


def test_noalloc_row_spanning_whole_windows(mspv, orc):
    """One row of 4 x 3072 + 100 entries starting exactly on a window boundary (entry 3072):
    its sum runs through the fix-up chain over three whole middle windows."""
    w = 3072
    rng = np.random.default_rng(31)
    n = 5000
    head_rows = np.sort(rng.integers(0, 1000, w)).astype(np.int32)      # exactly one window
    long_rows = np.full(4 * w + 100, 1500, np.int32)
    tail_rows = np.sort(rng.integers(1501, n, 7000)).astype(np.int32)
    r = np.concatenate([head_rows, long_rows, tail_rows])
    c = rng.integers(0, n, r.size).astype(np.int32)
    v = rng.uniform(-1, 1, r.size)
    assert np.all(np.diff(r) >= 0) and r[w] == 1500 and r[w - 1] < 1500
    dev = torch.device("cuda")
    rows, cols, vals = (torch.from_numpy(a).to(dev) for a in (r, c, v))
    for seed in (5, 6):
        xh = synth.uniform_x(n, seed) * 2 - 1
        y = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
        mspv.spmv_coo_noalloc(n, n, rows, cols, vals, torch.from_numpy(xh).to(dev), y)
        _oracle_check(orc, n, r, c, v, xh, y.cpu().numpy())


def test_noalloc_no_entries_zeroes_y(mspv):
    """nnz = 0 with rows: y = 0 on every row (y starts as NaN)."""
    dev = torch.device("cuda")
    n = 777
    empty_i = torch.zeros(0, dtype=torch.int32, device=dev)
    empty_v = torch.zeros(0, dtype=torch.float64, device=dev)
    x = torch.ones(n, dtype=torch.float64, device=dev)
    for _ in range(2):
        y = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
        mspv.spmv_coo_noalloc(n, n, empty_i, empty_i, empty_v, x, y)
        assert torch.all(y == 0).item()


def test_noalloc_rejects_bad_input(mspv):
    dev = torch.device("cuda")
    n = 100
    x = torch.ones(n, dtype=torch.float64, device=dev)
    y = torch.zeros(n, dtype=torch.float64, device=dev)
    rows = torch.tensor([0, 5, 3], dtype=torch.int32, device=dev)       # decreasing
    cols = torch.tensor([1, 2, 3], dtype=torch.int32, device=dev)
    vals = torch.tensor([1.0, 2.0, 3.0], dtype=torch.float64, device=dev)
    with pytest.raises(mspv.MspvError, match="EINVAL"):
        mspv.spmv_coo_noalloc(n, n, rows, cols, vals, x, y)
    bad_cols = torch.tensor([1, 2, 100], dtype=torch.int32, device=dev)  # outside the shape
    with pytest.raises(mspv.MspvError, match="EINVAL"):
        mspv.spmv_coo_noalloc(n, n, torch.tensor([0, 1, 2], dtype=torch.int32, device=dev), bad_cols, vals, x, y)
    # beyond the fixed scratch: rejected before any device work
    lib = mspv.load()
    st = lib.mspv_spmv_coo_noalloc(n, n, 201_326_593, rows.data_ptr(), cols.data_ptr(), vals.data_ptr(),
                                   x.data_ptr(), y.data_ptr(), mspv.stream_handle())
    assert st == 3   # MSPV_ETOOBIG
    # the context is still usable and a valid call still works
    ok_rows = torch.tensor([0, 3, 3], dtype=torch.int32, device=dev)
    mspv.spmv_coo_noalloc(n, n, ok_rows, cols, vals, x, y)
    out = y.cpu().numpy()
    assert out[0] == 1.0 and out[3] == 5.0 and np.count_nonzero(out) == 2
