"""The largest matrices the int32-index formats hold (nnz < 2^31; ETOOBIG from 2^31 on, a host
check covered on the CPU).

* The 27-point stencil on a 430^3 grid (n = 79,507,000, nnz = 1288^3 = 2,136,719,872; at 431^3
  it would pass 2^31): SpMV in COO, CSR and DIA, every output row against the separable closed
  form and sampled rows against the oracle's Algorithm 1; FP64 CG and reliable updates with
  BF16 values reaching a 1e-10 FP64 residual of the closed form.
* A 16,384 x 131,072 matrix stored densely less its last entry: nnz = 2^31 - 1 exactly, the
  last row ending at the last index int32 holds, so every entry loop of the COO segment kernel,
  the CSR long-row kernel and both staged CSR kernels runs up to the limit. Small-integer
  values and x make every row sum exact in FP64: the output equals the closed form and the
  oracle's sampled rows bit for bit.

Each case holds about 110 GB of device memory at its peak (triplets, the canonical COO and the
sort keys while the handle is built)."""
import numpy as np
import pytest

import synth
from _parity import assert_spmv_parity

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mspv():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2304_09511_gb300 as m
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return m


def sep_apply(x, g):
    """(A x, sum_j |a_ij x_j|) of the g^3 stencil by three separable 3-point passes."""
    x3 = x.reshape(g, g, g)
    out = x3
    for ax in range(3):
        s = out.copy()
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax], hi[ax] = slice(0, -1), slice(1, None)
        s[tuple(lo)] += out[tuple(hi)]
        s[tuple(hi)] += out[tuple(lo)]
        out = s
    return (27.0 * x3 - out).ravel(), (25.0 * np.abs(x3) + out).ravel()


def stencil_rows(g, rows):
    """The entries of the given rows of the g^3 stencil (26 on the diagonal, -1 to each
    neighbour inside the grid), renumbered 0..k-1, columns ascending."""
    ri, cj, v = [], [], []
    for k, i in enumerate(rows):
        ix, iy, iz = i % g, (i // g) % g, i // (g * g)
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    jx, jy, jz = ix + dx, iy + dy, iz + dz
                    if 0 <= jx < g and 0 <= jy < g and 0 <= jz < g:
                        ri.append(k)
                        cj.append(jz * g * g + jy * g + jx)
                        v.append(26.0 if dx == dy == dz == 0 else -1.0)
    return np.array(ri, np.int32), np.array(cj, np.int32), np.array(v, np.float64)


G_MAX = 430


def test_largest_stencil_spmv_and_solvers(mspv, orc):
    g = G_MAX
    n = g ** 3
    assert (3 * g - 2) ** 3 < 2 ** 31 <= (3 * g + 1) ** 3   # the largest grid int32 holds
    r, c, v = synth.stencil27_torch(g, "cuda")
    A = mspv.Matrix.from_coo(n, n, r, c, v)
    del r, c, v
    torch.cuda.empty_cache()
    assert A.info["nnz"] == (3 * g - 2) ** 3

    x = synth.uniform_x(n, 5)
    want, scale = sep_apply(x, g)
    xd = torch.from_numpy(x).cuda()
    rng = np.random.default_rng(430)
    sample = np.unique(np.concatenate([[0, 1, g - 1, g * g, n // 2, n - g * g - 1, n - 1],
                                       rng.integers(0, n, 9)]))
    sr, sc, sv = stencil_rows(g, sample)
    O = orc.canonicalize(sample.size, n, sr, sc, sv)
    for fmt in ("coo", "csr", "dia"):
        M = A if fmt == "coo" else A.convert(fmt)
        y = M.spmv(xd).cpu().numpy()
        assert np.all(np.abs(y - want) <= 1e-13 * scale), fmt
        assert_spmv_parity(y[sample], O, x, orc)
        if fmt == "dia":
            assert M.info["ndiags"] == 27
            D = M
        elif M is not A:
            M.close()
    del xd, y

    b_host, _ = sep_apply(np.ones(n), g)
    b = torch.from_numpy(b_host).cuda()
    bn = np.linalg.norm(b_host)
    # kappa <= 36 / lambda_min with lambda_min = 27 - (1 + 2 cos(pi / (g + 1)))^3: ~25,100
    kappa = 36.0 / (27.0 - (1.0 + 2.0 * np.cos(np.pi / (g + 1))) ** 3)

    def check(res):
        assert res.converged
        xs = res.x.cpu().numpy()
        ax, _ = sep_apply(xs, g)
        assert np.linalg.norm(b_host - ax) / bn <= 1.2e-10
        assert np.linalg.norm(xs - 1.0) / np.sqrt(n) <= kappa * 1.2e-10

    ref = D.cg(b, tol=1e-10, maxit=10000)
    check(ref)
    assert ref.iters <= int(np.sqrt(kappa) / 2 * np.log(2 / 1e-10)) + 1
    L = A.convert("dia", "bf16")
    A.close()
    check(D.cg_ru(L, b, tol=1e-10, maxit=10000))
    L.close()
    D.close()


M_ROWS, M_COLS = 1 << 14, 1 << 17
NNZ_LIMIT = (1 << 31) - 1


def dense_value(i, j):
    return ((i + j) % 7) - 3


def dense_x(j):
    return ((j % 5) - 2).astype(np.float64)


@pytest.fixture(scope="module")
def dense_limit(mspv):
    """The 2^14 x 2^17 matrix with every entry stored except the last: nnz = 2^31 - 1."""
    e = torch.arange(NNZ_LIMIT, dtype=torch.int64, device="cuda")
    rows = (e >> 17).to(torch.int32)
    cols = (e & (M_COLS - 1)).to(torch.int32)
    del e
    t = rows + cols
    t.remainder_(7).sub_(3)
    vals = t.to(torch.float64)
    del t
    A = mspv.Matrix.from_coo(M_ROWS, M_COLS, rows, cols, vals)
    del rows, cols, vals
    torch.cuda.empty_cache()
    yield A
    A.close()
    torch.cuda.empty_cache()


def dense_expected():
    j = np.arange(M_COLS, dtype=np.int64)
    xj = (j % 5) - 2
    per = [int(np.dot(dense_value(rho, j), xj)) for rho in range(7)]
    want = np.array([per[i % 7] for i in range(M_ROWS)], np.float64)
    last = M_ROWS - 1
    want[last] -= dense_value(last, M_COLS - 1) * xj[-1]   # the entry left out
    return want


def dense_oracle_rows(orc, rows, x):
    ri, cj, v = [], [], []
    for k, i in enumerate(rows):
        m = M_COLS - 1 if i == M_ROWS - 1 else M_COLS
        j = np.arange(m, dtype=np.int64)
        ri.append(np.full(m, k, np.int32))
        cj.append(j.astype(np.int32))
        v.append(dense_value(i, j).astype(np.float64))
    O = orc.canonicalize(len(rows), M_COLS, np.concatenate(ri), np.concatenate(cj), np.concatenate(v))
    return orc.spmv(O, x)


@pytest.mark.parametrize("kernel", ["coo", "csr", "csr_warp_staged", "csr_block_staged"])
def test_entry_loops_at_the_int32_limit(mspv, orc, dense_limit, monkeypatch, kernel):
    A = dense_limit
    info = A.info
    assert info["nnz"] == NNZ_LIMIT and info["row_max"] == M_COLS
    x = dense_x(np.arange(M_COLS))
    want = dense_expected()
    sample = [0, 1, 6, 8191, M_ROWS - 2, M_ROWS - 1]
    if kernel == "csr_warp_staged":
        monkeypatch.setenv("MSPV_CSR_VEC", "0")
    elif kernel == "csr_block_staged":
        monkeypatch.setenv("MSPV_CSR_VEC", "0")
        monkeypatch.setenv("MSPV_CSR_KERNEL", "block")
    M = A if kernel == "coo" else A.convert("csr")
    if kernel != "coo":
        assert M.info["csr_vector"] == (32 if kernel == "csr" else 0)
    y = M.spmv(torch.from_numpy(x).cuda()).cpu().numpy()
    if M is not A:
        M.close()
        torch.cuda.empty_cache()
    assert np.array_equal(y, want)
    assert np.array_equal(y[sample], dense_oracle_rows(orc, sample, x))
