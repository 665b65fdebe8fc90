"""Full-size parity on the benchmark workload: the 27-point stencil on a 128^3 grid
(n = 2,097,152, nnz = 382^3 = 55,742,968) in COO, CSR and DIA, in the launch
configuration the benchmark times, against the oracle on the whole output; plus the
separable closed form A x = 27 x - (T (x) T (x) T) x as a size-independent property,
and 50 FP64 CG iterations against the oracle's."""
import numpy as np
import pytest

import synth
from _parity import assert_spmv_parity, assert_structure_equal

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

G = 128


@pytest.fixture(scope="module")
def mspv():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2304_09511_gb300 as m
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return m


@pytest.fixture(scope="module")
def big(mspv, orc):
    n = G ** 3
    r, c, v = synth.stencil27(G)
    A = mspv.Matrix.from_coo(n, n, torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda(),
                             torch.from_numpy(v).cuda())
    O = orc.canonicalize(n, n, r, c, v)
    del r, c, v
    mats = {"coo": (A, O), "csr": (A.convert("csr"), orc.coo_to_csr(O)),
            "dia": (A.convert("dia"), orc.coo_to_dia(O))}
    return n, mats


def sep_apply(x):
    x3 = x.reshape(G, G, G)
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


@pytest.mark.parametrize("fmt", ["coo", "csr", "dia"])
def test_fullsize_structure_and_spmv(mspv, orc, big, fmt):
    n, mats = big
    M, O = mats[fmt]
    assert M.info["nnz"] == (3 * G - 2) ** 3
    assert_structure_equal(M, O, orc)
    x = synth.uniform_x(n, 0)
    y = M.spmv(torch.from_numpy(x).cuda()).cpu().numpy()
    assert_spmv_parity(y, O, x, orc)
    want, scale = sep_apply(x)   # x >= 0, so the scale is sum |a x|
    assert np.all(np.abs(y - want) <= 1e-13 * scale)


def test_fullsize_cg_50_iterations(mspv, orc, big):
    n, mats = big
    D, Od = mats["dia"]
    b = orc.spmv(Od, np.ones(n))
    res = D.cg(torch.from_numpy(b).cuda(), tol=0.0, maxit=50)
    xo, st, k, rel, _, _ = orc.cg(Od, b, tol=0.0, maxit=50)
    assert res.converged and res.iters == 50 == k
    x = res.x.cpu().numpy()
    assert np.max(np.abs(x - xo)) <= 1e-10 * np.max(np.abs(xo))
    assert res.relres == pytest.approx(rel, rel=1e-8)
    # the other formats take the same path to the same iterate
    for fmt in ("csr", "coo"):
        M, _ = mats[fmt]
        r2 = M.cg(torch.from_numpy(b).cuda(), tol=0.0, maxit=50)
        assert np.max(np.abs(r2.x.cpu().numpy() - xo)) <= 1e-10 * np.max(np.abs(xo))
