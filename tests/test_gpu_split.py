"""GPU parity of the local/remote split (the per-process matrix split of the paper's
distributed HPCG, Sec. VI) and of the accumulating SpMV y += A x, against the oracle."""
import numpy as np
import pytest

import synth
from _parity import assert_structure_equal, spmv_tolerance

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def assert_acc_parity(y_gpu, y0, O, x, orc):
    """y_gpu = y0 + A x: the SpMV bound of each row plus the rounding of the final add."""
    want = y0 + orc.spmv(O, x)
    bound = spmv_tolerance(O, x, orc) + 2 * U * (np.abs(y0) + np.abs(want))
    assert not np.any(np.isnan(y_gpu))
    bad = np.nonzero(np.abs(y_gpu - want) > bound)[0]
    assert bad.size == 0, f"{bad.size} rows out of tolerance, first {bad[0]}"


@pytest.mark.parametrize("src", ["coo", "csr"])
def test_split_of_a_process_matrix_is_bit_exact(mspv, orc, src):
    nx, ny, nz = 20, 16, 12
    r, c, v, n, ng = synth.hpcg_rank_matrix(nx, ny, nz)
    A = mspv.Matrix.from_coo(n, n + ng, dev(r), dev(c), dev(v))
    if src == "csr":
        A = A.convert("csr")
    L, R = A.split_columns(n)
    O = orc.canonicalize(n, n + ng, r, c, v)
    OL, OR = orc.split_columns(O, n)
    assert L.shape == (n, n) and R.shape == (n, ng)
    assert_structure_equal(L, OL, orc)
    assert_structure_equal(R, OR, orc)
    assert L.info["nnz"] == (3 * nx - 2) * (3 * ny - 2) * (3 * nz - 2)


@pytest.mark.parametrize("local_fmt,remote_fmt", [("dia", "coo"), ("dia", "csr"), ("csr", "coo"), ("coo", "coo")])
def test_split_spmv_equals_whole(mspv, orc, local_fmt, remote_fmt):
    """y = local x_local, then y += remote x_ghost, equals the whole matrix's SpMV."""
    nx, ny, nz = 24, 20, 16
    r, c, v, n, ng = synth.hpcg_rank_matrix(nx, ny, nz)
    A = mspv.Matrix.from_coo(n, n + ng, dev(r), dev(c), dev(v))
    L0, R0 = A.split_columns(n)
    L = L0 if local_fmt == "coo" else L0.convert(local_fmt)
    R = R0 if remote_fmt == "coo" else R0.convert(remote_fmt)
    x = synth.uniform_x(n + ng, 3) * 2 - 1
    xd = dev(x)
    y = L.spmv(xd[:n].contiguous())
    R.spmv_add(xd[n:].contiguous(), y)
    O = orc.canonicalize(n, n + ng, r, c, v)
    OL, OR = orc.split_columns(O, n)
    y_local = orc.spmv(OL, x[:n])
    want = y_local + orc.spmv(OR, x[n:])
    # each part's SpMV bound (the GPU sums in another order than the oracle) plus the add
    bound = (spmv_tolerance(OL, x[:n], orc) + spmv_tolerance(OR, x[n:], orc)
             + 2 * U * (np.abs(y_local) + np.abs(want)))
    yg = y.cpu().numpy()
    assert not np.any(np.isnan(yg))
    assert np.all(np.abs(yg - want) <= bound)
    # and the unsplit matrix's SpMV, within its own bound on top
    whole = orc.spmv(O, x)
    assert np.all(np.abs(yg - whole) <= bound + spmv_tolerance(O, x, orc))


CASES = [
    ("coo_rb", "coo", "rb"), ("coo_vec", "coo", "vec"), ("coo_seg", "coo", "seg"), ("csr", "csr", None),
    ("dia", "dia", None),
]


@pytest.mark.parametrize("name,fmt,coo_kernel", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("vt", ["f64", "f32"])
def test_spmv_add_every_kernel(mspv, orc, monkeypatch, name, fmt, coo_kernel, vt):
    """y += A x for each kernel, with empty rows (left untouched), rows spanning chunks and
    rows too long for the CSR V-lane kernel."""
    if coo_kernel:
        monkeypatch.setenv("MSPV_COO_KERNEL", coo_kernel)
    n = 9000
    rng = np.random.default_rng(7)
    lens = rng.choice([0, 1, 3, 27, 40, 300, 1500], size=n, p=[.25, .1, .1, .35, .1, .08, .02])
    r = np.repeat(np.arange(n), lens)
    if fmt == "dia":   # a banded pattern DIA can hold, every seventh row emptied
        r, c, v = synth.banded(n, 15, 4, 0.9, 60)
        keep = r % 7 != 3
        r, c, v = r[keep], c[keep], v[keep]
    else:
        c = rng.integers(0, n, r.size)
        v = rng.uniform(-1, 1, r.size)
    A = mspv.Matrix.from_coo(n, n, dev(np.asarray(r, np.int32)), dev(np.asarray(c, np.int32)), dev(v))
    M = A.convert(fmt, vt) if (fmt != "coo" or vt != "f64") else A
    O = orc.canonicalize(n, n, r, c, v)
    Of = orc.convert(O, fmt)
    if vt != "f64":
        Of = orc.with_values(Of, vt)
    x = synth.uniform_x(n, 11) * 2 - 1
    y0 = rng.uniform(-5, 5, n)
    y = dev(y0.copy())
    M.spmv_add(dev(x), y)
    yg = y.cpu().numpy()
    assert_acc_parity(yg, y0, Of, x, orc)
    empty = np.bincount(O.ai, minlength=n) == 0
    assert empty.any() and np.array_equal(yg[empty], y0[empty])


def test_split_rejects_bad_arguments(mspv):
    A = mspv.Matrix.from_coo(4, 6, np.array([0, 1], np.int32), np.array([5, 2], np.int32), np.ones(2))
    with pytest.raises(mspv.MspvError, match="EINVAL"):
        A.split_columns(7)
    D = mspv.Matrix.from_coo(4, 4, np.array([0, 1], np.int32), np.array([0, 1], np.int32),
                             np.ones(2)).convert("dia")
    with pytest.raises(mspv.MspvError, match="EFORMAT"):
        D.split_columns(2)
    L, R = A.split_columns(0)
    assert L.info["nnz"] == 0 and R.info["nnz"] == 2 and R.shape == (4, 6)


@pytest.mark.parametrize("local_fmt,remote_fmt", [("dia", "coo"), ("csr", "csr")])
def test_zslab_partition_on_one_gpu(mspv, orc, local_fmt, remote_fmt):
    """The row-block partition of the distributed HPCG run through the library on one GPU: the
    40^3 stencil cut into 4 z-slabs, each slab's matrix (own columns, then ghost columns by
    first appearance) split by the library, y_s = A_local x_s then y_s += A_remote x_ghost;
    the slabs together equal the whole matrix's SpMV bit for bit (integer data and x, so every
    partial sum is exact)."""
    from test_partition_cpu import slab_matrix
    g, P = 40, 4
    n = g ** 3
    rows, cols, vals = synth.stencil27(g)
    x = np.random.default_rng(7).integers(-4, 5, n).astype(np.float64)
    W = mspv.Matrix.from_coo(n, n, dev(rows), dev(cols), dev(vals)).convert("dia")
    want = W.spmv(dev(x)).cpu().numpy()
    assert np.array_equal(want, orc.spmv(orc.Matrix(orc.COO, n, n, rows.size, ai=rows, aj=cols, av=vals), x))
    cuts = np.linspace(0, g, P + 1).round().astype(int)
    got = []
    for s in range(P):
        z0, z1 = cuts[s], cuts[s + 1]
        r, c, v, n_s, ghosts = slab_matrix(g, z0, z1, rows, cols, vals)
        S = mspv.Matrix.from_coo(n_s, n_s + ghosts.size, dev(r), dev(c), dev(v))
        L, R = S.split_columns(n_s)
        L = L if local_fmt == "coo" else L.convert(local_fmt)
        R = R if remote_fmt == "coo" else R.convert(remote_fmt)
        y = L.spmv(dev(x[z0 * g * g:z1 * g * g]))
        R.spmv_add(dev(x[ghosts]), y)
        got.append(y.cpu().numpy())
    assert np.array_equal(np.concatenate(got), want)
