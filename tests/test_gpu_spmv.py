"""GPU parity: format converters (bit-exact) and SpMV (per-row FP64 bound) through the
C ABI, against the CPU oracle on the same seeded inputs."""
import os

import numpy as np
import pytest

import synth
from _parity import assert_spmv_parity, assert_structure_equal, spmv_tolerance

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mspv():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2304_09511_gb300 as m
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = [
    # (nrows, ncols, nnz, seed, dup_frac, empty_rows)
    (1, 1, 1, 0, 0.0, 0),
    (1, 1, 5, 1, 0.8, 0),
    (5, 5, 11, 2, 0.0, 0),
    (7, 13, 30, 3, 0.2, 2),
    (13, 7, 30, 4, 0.2, 3),
    (64, 64, 700, 6, 0.3, 9),
    (64, 64, 4096, 7, 0.0, 0),
    (300, 300, 257, 8, 0.0, 100),        # just over one COO chunk, many empty rows
    (1000, 1000, 4097, 9, 0.1, 50),      # one radix tile + 1, ragged
    (20000, 20000, 333_333, 10, 0.05, 2000),   # many tiles, ragged tails
    (5000, 37000, 100_001, 11, 0.0, 7),  # rectangular, wide
    (37000, 5000, 100_001, 12, 0.02, 7),  # rectangular, tall
]


def build_pair(mspv, orc, case, on_device):
    nrows, ncols, nnz, seed, dup, empty = case
    r, c, v = synth.random_coo(nrows, ncols, nnz, seed, dup_frac=dup, empty_rows=empty)
    if on_device:
        A = mspv.Matrix.from_coo(nrows, ncols, dev(r), dev(c), dev(v))
    else:
        A = mspv.Matrix.from_coo(nrows, ncols, r, c, v)
    O = orc.canonicalize(nrows, ncols, r, c, v)
    return A, O


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}nnz{c[2]}")
@pytest.mark.parametrize("on_device", [False, True], ids=["host_in", "dev_in"])
def test_canonical_coo_bit_exact(mspv, orc, case, on_device):
    A, O = build_pair(mspv, orc, case, on_device)
    assert A.info["nnz"] == O.nnz
    assert_structure_equal(A, O, orc)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}nnz{c[2]}")
def test_csr_and_dia_bit_exact(mspv, orc, case):
    A, O = build_pair(mspv, orc, case, True)
    C = A.convert("csr")
    assert_structure_equal(C, orc.coo_to_csr(O), orc)
    inf = C.info
    lens = np.bincount(O.ai, minlength=case[0])[:case[0]]
    assert inf["row_max"] == (lens.max() if lens.size else 0)
    assert inf["empty_rows"] == int(np.sum(lens == 0))
    assert inf["row_mean"] == pytest.approx(O.nnz / case[0])
    if case[0] == case[1]:
        G = orc.coo_to_dia(O)
        if G.ndiags * G.npad > max(32 * O.nnz, 1 << 20):
            with pytest.raises(mspv.MspvError, match="ETOOBIG"):
                A.convert("dia")
        else:
            assert_structure_equal(A.convert("dia"), G, orc)
            # CSR-sourced DIA is the same structure
            assert_structure_equal(C.convert("dia"), G, orc)
    else:
        with pytest.raises(mspv.MspvError, match="EFORMAT"):
            A.convert("dia")


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}nnz{c[2]}")
@pytest.mark.parametrize("fmt", ["coo", "csr"])
def test_spmv_parity(mspv, orc, case, fmt):
    A, O = build_pair(mspv, orc, case, True)
    M = A if fmt == "coo" else A.convert(fmt)
    Of = orc.convert(O, fmt)
    x = synth.uniform_x(case[1], case[3]) * 2 - 1
    y = M.spmv(dev(x)).cpu().numpy()
    assert_spmv_parity(y, Of, x, orc)


BANDED = [
    # (n, k diagonals, seed, fill, spread)
    (1, 1, 0, 1.0, None),
    (5, 3, 1, 1.0, None),
    (33, 9, 2, 0.7, None),
    (64, 127, 3, 1.0, None),        # dense: every diagonal
    (1000, 27, 4, 0.9, 60),
    (20001, 27, 5, 1.0, 300),       # ragged against the 32-row padding and the tiles
    (50000, 40, 6, 0.5, 49000),     # far offsets: long out-of-range stretches
]


@pytest.mark.parametrize("case", BANDED, ids=lambda c: f"n{c[0]}k{c[1]}")
@pytest.mark.parametrize("fmt", ["coo", "csr", "dia"])
def test_banded_structure_and_spmv(mspv, orc, case, fmt):
    n, k, seed, fill, spread = case
    r, c, v = synth.banded(n, k, seed, fill, spread)
    A = mspv.Matrix.from_coo(n, n, dev(r), dev(c), dev(v))
    O = orc.convert(orc.canonicalize(n, n, r, c, v), fmt)
    M = A if fmt == "coo" else A.convert(fmt)
    assert_structure_equal(M, O, orc)
    x = synth.uniform_x(n, seed) * 2 - 1
    assert_spmv_parity(M.spmv(dev(x)).cpu().numpy(), O, x, orc)


@pytest.mark.parametrize("kernel", ["rb", "vec", "seg"])
@pytest.mark.parametrize("acc", [False, True])
def test_coo_long_empty_gaps(mspv, orc, kernel, acc, monkeypatch):
    """Ten million rows, five entries (first rows, the middle, the last row): the rows between
    them are zeroed in parallel (y = A x) or left as they are (y += A x) by every COO kernel."""
    monkeypatch.setenv("MSPV_COO_KERNEL", kernel)
    n = 10_000_000
    r = np.array([0, 0, 3, n // 2, n - 1], np.int32)
    c = np.array([1, 5, 3, n - 7, 0], np.int32)
    v = np.array([0.5, -2.0, 3.0, 1.25, -0.75])
    A = mspv.Matrix.from_coo(n, n, dev(r), dev(c), dev(v))
    x = torch.linspace(-1.0, 1.0, n, dtype=torch.float64, device="cuda")
    y0 = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
    y = y0.clone()
    if acc:
        A.spmv_add(x, y)
    else:
        A.spmv(x, y)
    xh = x.cpu().numpy()
    want = np.full(n, 7.0) if acc else np.zeros(n)
    np.add.at(want, r, v * xh[c])
    got = y.cpu().numpy()
    assert np.allclose(got, want, rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("arith", ["f64", "f32", "bf16"])
def test_dia_more_diagonals_than_shared_tables(mspv, orc, arith):
    """600 scattered diagonals (about 550 runs of consecutive offsets): past the 256 offsets and
    runs the DIA kernels cache in shared memory they read the tables from global memory; FP64
    SpMV and FP32-arithmetic SpMV (FP32 / BF16 values) against the oracle."""
    n, k = 4003, 600
    r, c, v = synth.banded(n, k, 17, 0.8, 1900)
    A = mspv.Matrix.from_coo(n, n, dev(r), dev(c), dev(v))
    vt = "f64" if arith == "f64" else arith
    D = A.convert("dia", vt)
    O = orc.with_values(orc.coo_to_dia(orc.canonicalize(n, n, r, c, v)), vt)
    assert O.ndiags == k and D.info["ndiags"] == k
    if arith == "f64":
        x = synth.uniform_x(n, 18) * 2 - 1
        assert_spmv_parity(D.spmv(dev(x)).cpu().numpy(), O, x, orc)
        return
    x32 = (synth.uniform_x(n, 18) * 2 - 1).astype(np.float32)
    y = D.spmv_f32(dev(x32)).cpu().numpy().astype(np.float64)
    x64 = x32.astype(np.float64)
    want = orc.spmv(O, x64)
    absO = orc.Matrix(O.fmt, O.nrows, O.ncols, O.nnz, ai=O.ai, aj=O.aj, irp=O.irp, av=np.abs(O.av),
                      doff=O.doff, npad=O.npad)
    bound = 2.0 * (k + 2) * 2.0 ** -24 * orc.spmv(absO, np.abs(x64)) + 1e-30
    assert np.all(np.abs(y - want) <= bound)


@pytest.mark.parametrize("vec", ["0w", "0b", 1, 2, 4, 8, 16, 32])
def test_csr_every_kernel_choice(mspv, orc, vec, monkeypatch):
    if isinstance(vec, str):   # staged kernels: warp-private slices or CTA row blocks
        monkeypatch.setenv("MSPV_CSR_KERNEL", "block" if vec == "0b" else "warp")
        vec = 0
    monkeypatch.setenv("MSPV_CSR_VEC", str(vec))
    case = (3000, 3000, 60_000, 21, 0.0, 30)
    A, O = build_pair(mspv, orc, case, True)
    C = A.convert("csr")
    assert C.info["csr_vector"] == vec
    x = synth.uniform_x(case[1], 5)
    assert_spmv_parity(C.spmv(dev(x)).cpu().numpy(), orc.coo_to_csr(O), x, orc)
    # long rows: a block too large to stage takes the whole-CTA path
    r = np.concatenate([np.full(9000, 7), np.full(5000, 2999), np.arange(3000)]).astype(np.int32)
    c = np.random.default_rng(2).integers(0, 3000, r.size).astype(np.int32)
    v = np.random.default_rng(3).uniform(-1, 1, r.size)
    L = mspv.Matrix.from_coo(3000, 3000, dev(r), dev(c), dev(v)).convert("csr")
    OL = orc.coo_to_csr(orc.canonicalize(3000, 3000, r, c, v))
    assert_spmv_parity(L.spmv(dev(x)).cpu().numpy(), OL, x, orc)


@pytest.mark.parametrize("kernel", ["seg", "vec", "vec512", "rb"])
def test_coo_every_kernel_choice(mspv, orc, kernel, monkeypatch):
    """Every COO kernel (lane-sequential 512-entry segments; run-vector 256-entry chunks; 32-row
    blocks, here also with rows far above the 128 entries it is chosen for) on shapes that hit
    their edges: rows spanning lanes and chunks, a row covering many
    chunks, empty rows before, between and after entries (whole empty row blocks), partial
    last lanes and chunks, one entry."""
    monkeypatch.setenv("MSPV_COO_KERNEL", kernel[:3])
    monkeypatch.setenv("MSPV_COO_CHUNK", "512" if kernel == "vec512" else "256")
    rng = np.random.default_rng(31)
    shapes = []
    n = 6000
    lens = rng.choice([0, 1, 2, 15, 16, 17, 27, 31, 33, 511, 513, 1500], size=n,
                      p=[.2, .1, .1, .1, .1, .1, .1, .05, .05, .04, .04, .02])
    shapes.append((n, np.repeat(np.arange(n), lens)))
    shapes.append((50, np.full(7000, 49)))                  # one row covering 14 chunks
    shapes.append((3000, np.sort(rng.integers(1000, 1010, 1025))))   # empty rows both ends
    shapes.append((100, np.array([37])))                     # a single entry
    shapes.append((9000, np.repeat(np.arange(9000), 27)[: 512 * 7 + 5]))
    for nr, r in shapes:
        r = r.astype(np.int32)
        c = rng.integers(0, nr, r.size).astype(np.int32)
        v = rng.uniform(-1, 1, r.size)
        for vt in ("f64", "f32"):
            A = mspv.Matrix.from_coo(nr, nr, dev(r), dev(c), dev(v))
            M = A if vt == "f64" else A.convert("coo", vt)
            O = orc.canonicalize(nr, nr, r, c, v)
            if vt != "f64":
                O = orc.with_values(O, vt)
            x = synth.uniform_x(nr, 4) * 2 - 1
            y = torch.full((nr,), float("nan"), dtype=torch.float64, device="cuda")
            M.spmv(dev(x), y)
            assert_spmv_parity(y.cpu().numpy(), O, x, orc)


def test_window_edges_of_staged_kernels(mspv, orc):
    """Rows cut by COO window edges (every 3072 entries) and CSR row blocks of every size
    agree with the oracle: long rows span several windows, short rows straddle edges."""
    n = 9000
    rng = np.random.default_rng(12)
    lens = rng.choice([1, 2, 27, 130, 3071, 3072, 3073, 7000], size=60)
    rows = np.repeat(rng.choice(n, 60, replace=False), lens)
    cols = rng.integers(0, n, rows.size)
    vals = rng.uniform(-1, 1, rows.size)
    A = mspv.Matrix.from_coo(n, n, dev(rows.astype(np.int32)), dev(cols.astype(np.int32)), dev(vals))
    O = orc.canonicalize(n, n, rows, cols, vals)
    x = synth.uniform_x(n, 8) * 2 - 1
    for fmt in ("coo", "csr"):
        M = A if fmt == "coo" else A.convert(fmt)
        assert_spmv_parity(M.spmv(dev(x)).cpu().numpy(), orc.convert(O, fmt), x, orc)


def test_csr_long_rows_split_off(mspv, orc):
    """Power-law-like rows: most short, some far above 32 V entries; the long ones are
    listed at conversion and reduced by a CTA each (also inside CG's fused dot)."""
    rng = np.random.default_rng(21)
    n = 20000
    lens = np.minimum((rng.pareto(1.1, n) * 4 + 1).astype(np.int64), 5000)
    r = np.repeat(np.arange(n), lens).astype(np.int32)
    c = rng.integers(0, n, r.size).astype(np.int32)
    v = rng.uniform(-1, 1, r.size)
    A = mspv.Matrix.from_coo(n, n, dev(r), dev(c), dev(v))
    C = A.convert("csr")
    assert C.info["csr_vector"] == 4 and C.info["row_max"] > 128
    O = orc.coo_to_csr(orc.canonicalize(n, n, r, c, v))
    x = synth.uniform_x(n, 3) * 2 - 1
    assert_spmv_parity(C.spmv(dev(x)).cpu().numpy(), O, x, orc)


def test_long_rows_and_chunk_spanning(mspv, orc):
    """A 20,000-entry row spans ~80 COO chunks; short rows around it; empty rows at both ends."""
    rng = np.random.default_rng(3)
    n = 30000
    r = np.concatenate([np.full(20000, 17000), rng.integers(100, 29000, 50000), [5, 5, 29990]])
    c = np.concatenate([rng.permutation(n)[:20000], rng.integers(0, n, 50003)])
    v = rng.uniform(-1, 1, r.size)
    A = mspv.Matrix.from_coo(n, n, dev(r.astype(np.int32)), dev(c.astype(np.int32)), dev(v))
    O = orc.canonicalize(n, n, r, c, v)
    x = synth.uniform_x(n, 9)
    for fmt in ("coo", "csr"):
        M = A if fmt == "coo" else A.convert(fmt)
        assert_spmv_parity(M.spmv(dev(x)).cpu().numpy(), orc.convert(O, fmt), x, orc)


def test_all_entries_in_one_row(mspv, orc):
    n = 4000
    rng = np.random.default_rng(4)
    r = np.full(3000, 1234, np.int32)
    c = rng.integers(0, n, 3000).astype(np.int32)
    v = rng.uniform(-1, 1, 3000)
    A = mspv.Matrix.from_coo(n, n, r, c, v)
    O = orc.canonicalize(n, n, r, c, v)
    x = synth.uniform_x(n, 1)
    for fmt in ("coo", "csr"):
        M = A if fmt == "coo" else A.convert(fmt)
        y = M.spmv(dev(x)).cpu().numpy()
        assert_spmv_parity(y, orc.convert(O, fmt), x, orc)
        assert np.count_nonzero(y) == 1


def test_empty_matrix_gives_zero(mspv):
    A = mspv.Matrix.from_coo(10, 7, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    for M in (A, A.convert("csr")):
        y = torch.full((10,), 5.0, dtype=torch.float64, device="cuda")
        M.spmv(torch.ones(7, dtype=torch.float64, device="cuda"), y)
        assert torch.all(y == 0)


@pytest.mark.parametrize("vt", ["f32", "bf16"])
@pytest.mark.parametrize("fmt", ["coo", "csr", "dia"])
def test_low_precision_values(mspv, orc, vt, fmt):
    n = 20001
    r, c, v = synth.banded(n, 27, 7, 0.95, 500)
    v = v * 37.0   # values over several binades so rounding is exercised
    A = mspv.Matrix.from_coo(n, n, dev(r), dev(c), dev(v))
    O = orc.canonicalize(n, n, r, c, v)
    M = A.convert(fmt, vt)
    assert M.info["value_type"] == vt
    Of = orc.with_values(orc.convert(O, fmt), vt)
    assert_structure_equal(M, Of, orc)   # rounding is bit-exact with the oracle's
    x = synth.uniform_x(n, 2)
    assert_spmv_parity(M.spmv(dev(x)).cpu().numpy(), Of, x, orc)


def test_spmv_is_deterministic(mspv):
    r, c, v = synth.random_coo(50000, 50000, 800_000, 41, dup_frac=0.05)
    A = mspv.Matrix.from_coo(50000, 50000, dev(r), dev(c), dev(v))
    x = dev(synth.uniform_x(50000, 3))
    for M in (A, A.convert("csr")):
        y1 = M.spmv(x).clone()
        y2 = M.spmv(x)
        assert torch.equal(y1, y2)


def test_device_triplets_out_of_range_rejected(mspv):
    r = dev(np.array([0, 1, 7], np.int32))
    c = dev(np.array([0, 1, 1], np.int32))
    v = dev(np.array([1.0, 2.0, 3.0]))
    with pytest.raises(mspv.MspvError, match="EINVAL"):
        mspv.Matrix.from_coo(3, 3, r, c, v)
    # the context stays usable
    A = mspv.Matrix.from_coo(3, 3, dev(np.array([0, 2], np.int32)), dev(np.array([1, 2], np.int32)),
                             dev(np.array([1.0, 2.0])))
    y = A.spmv(dev(np.ones(3))).cpu().numpy()
    assert y.tolist() == [1.0, 0.0, 2.0]


def test_dia_too_big(mspv):
    r, c, v = synth.random_coo(200_000, 200_000, 400_000, 5)
    A = mspv.Matrix.from_coo(200_000, 200_000, dev(r), dev(c), dev(v))
    with pytest.raises(mspv.MspvError, match="ETOOBIG"):
        A.convert("dia")


def test_memory_cap_injects_enomem(mspv, monkeypatch):
    r, c, v = synth.random_coo(1000, 1000, 5000, 6)
    A = mspv.Matrix.from_coo(1000, 1000, r, c, v)
    monkeypatch.setenv("MSPV_MAX_BYTES", "1000")
    with pytest.raises(mspv.MspvError, match="ENOMEM"):
        A.convert("csr")
    with pytest.raises(mspv.MspvError, match="ENOMEM"):
        mspv.Matrix.from_coo(1000, 1000, r, c, v)
    monkeypatch.delenv("MSPV_MAX_BYTES")
    A.convert("csr")   # works again


def _fp32_cases():
    # (name, n, triplet generator): consecutive offsets (runs of 3), isolated offsets (runs of
    # 1), mixed runs, and a size that is not a multiple of 4 (ragged windows at the ends)
    return [
        ("stencil20", 20 ** 3, lambda: synth.stencil27_perturbed(20, 5)),
        ("banded_isolated", 20001, lambda: synth.banded(20001, 9, 11, 1.0, 3000)),
        ("banded_mixed", 30003, lambda: synth.banded(30003, 27, 12, 0.9, 40)),
    ]


@pytest.mark.parametrize("case", _fp32_cases(), ids=lambda c: c[0])
@pytest.mark.parametrize("vt", ["f32", "bf16"])
@pytest.mark.parametrize("fmt", ["coo", "csr", "dia"])
def test_fp32_arithmetic_spmv(mspv, orc, case, vt, fmt):
    """The FP32-arithmetic SpMV (the inner SpMV of the FP32 refinement solver) against the
    oracle on the same rounded values and FP32 x: per row within 2(k+2) u32 sum |a x|, the
    FP32 counterpart of the FP64 bound (u32 = 2^-24; the products of FP32/BF16 values and FP32
    x are exact in FP64, only the FP32 sum rounds)."""
    name, n, gen = case
    r, c, v = gen()
    A = mspv.Matrix.from_coo(n, n, dev(r), dev(c), dev(v))
    M = A.convert(fmt, vt)
    O = orc.with_values(orc.convert(orc.canonicalize(n, n, r, c, v), fmt), vt)
    x32 = (synth.uniform_x(n, 21) * 2 - 1).astype(np.float32)
    y = M.spmv_f32(dev(x32)).cpu().numpy().astype(np.float64)
    x64 = x32.astype(np.float64)
    want = orc.spmv(O, x64)
    absO = orc.Matrix(O.fmt, O.nrows, O.ncols, O.nnz, ai=O.ai, aj=O.aj, irp=O.irp, av=np.abs(O.av),
                      doff=O.doff, npad=O.npad)
    scale = orc.spmv(absO, np.abs(x64))
    if fmt == "dia":
        k = np.full(n, O.ndiags)
    elif fmt == "csr":
        k = np.diff(O.irp)
    else:
        k = np.bincount(O.ai, minlength=n)
    bound = 2.0 * (k + 2) * 2.0 ** -24 * scale + 1e-30
    bad = np.nonzero(np.abs(y - want) > bound)[0]
    assert bad.size == 0, f"{bad.size} rows out of tolerance, first {bad[:5]}"


def test_fp32_arithmetic_spmv_rejects_bad_input(mspv):
    r, c, v = synth.stencil27(6)
    A = mspv.Matrix.from_coo(216, 216, r, c, v)
    x = torch.ones(217, dtype=torch.float32, device="cuda")
    with pytest.raises(mspv.MspvError, match="EFORMAT"):
        A.convert("dia").spmv_f32(x[:216])
    D = A.convert("dia", "f32")
    with pytest.raises(mspv.MspvError, match="EINVAL"):
        D.spmv_f32(x[1:])   # 4-byte aligned only


# ---------------------------------------------------------------------------
# DIA with distant and ragged diagonals: a banded matrix whose offsets reach past several
# 512-row strips, ending in a partial strip
# ---------------------------------------------------------------------------
BAND_OFFSETS = [-700, -699, -13, -5, -4, -3, -2, 0, 1, 2, 9, 10, 11, 12, 600, 1201]


def _banded_coo(n, offsets, seed):
    """Every in-range slot of the given diagonals, values U(-1, 1) (diagonal 4 + |.|)."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for o in offsets:
        i = np.arange(max(0, -o), min(n, n - o), dtype=np.int64)
        rows.append(i)
        cols.append(i + o)
    r = np.concatenate(rows).astype(np.int32)
    c = np.concatenate(cols).astype(np.int32)
    v = rng.uniform(-1.0, 1.0, r.size)
    v[r == c] = 4.0 + np.abs(v[r == c])
    return r, c, v


def test_dia_banded_ragged_fp64(mspv, orc):
    """FP64 DIA on 16 diagonals between -700 and +1201 over 155,685 rows (the last strip
    partial), y = A x and y += A x, against the oracle's Algorithm 3."""
    n = 152 * 4 * 256 + 37
    r, c, v = _banded_coo(n, BAND_OFFSETS, 5)
    A = mspv.Matrix.from_coo(n, n, dev(r), dev(c), dev(v))
    D = A.convert("dia")
    O = orc.coo_to_dia(orc.canonicalize(n, n, r, c, v))
    x = synth.uniform_x(n, 9) * 2 - 1
    xd = dev(x)
    y0 = synth.uniform_x(n, 10)
    ya = dev(y0)
    D.spmv_add(xd, ya)
    assert_spmv_parity(D.spmv(xd).cpu().numpy(), O, x, orc)
    # y += A x: one more rounding of the sum
    want = y0 + orc.spmv(O, x)
    bound = spmv_tolerance(O, x, orc) + 2.0 ** -52 * np.abs(want)
    assert np.all(np.abs(ya.cpu().numpy() - want) <= bound)


@pytest.mark.parametrize("vt", ["f32", "bf16"])
def test_dia_banded_ragged_fp32_arithmetic(mspv, orc, vt):
    """FP32-arithmetic DIA (FP32 / BF16 values) on the banded matrix: within the FP32 bound
    2 (k + 2) 2^-24 sum |a x| of the oracle's product on the rounded values."""
    n = 152 * 4 * 512 + 3
    r, c, v = _banded_coo(n, BAND_OFFSETS, 5)
    A = mspv.Matrix.from_coo(n, n, dev(r), dev(c), dev(v))
    D = A.convert("dia", vt)
    O = orc.with_values(orc.coo_to_dia(orc.canonicalize(n, n, r, c, v)), vt)
    x32 = (synth.uniform_x(n, 11) * 2 - 1).astype(np.float32)
    got = D.spmv_f32(dev(x32)).cpu().numpy()
    x64 = x32.astype(np.float64)
    want = orc.spmv(O, x64)
    absO = orc.Matrix(O.fmt, O.nrows, O.ncols, O.nnz, ai=O.ai, aj=O.aj, irp=O.irp, av=np.abs(O.av),
                      doff=O.doff, npad=O.npad)
    scale = orc.spmv(absO, np.abs(x64))
    bound = 2.0 * (O.ndiags + 2) * 2.0 ** -24 * scale + 1e-30
    assert np.all(np.abs(got.astype(np.float64) - want) <= bound)
