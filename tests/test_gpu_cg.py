"""GPU parity for CG (and iterative refinement) through the C ABI against the CPU
oracle: the 27-point stencil of the HPCG experiments, plus the special cases."""
import numpy as np
import pytest

import synth
from _parity import assert_spmv_parity, assert_structure_equal

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


@pytest.fixture(scope="module")
def stencil16(mspv, orc):
    g = 16
    n = g ** 3
    r, c, v = synth.stencil27(g)
    A = mspv.Matrix.from_coo(n, n, dev(r), dev(c), dev(v))
    O = orc.canonicalize(n, n, r, c, v)
    return g, n, A, O


@pytest.mark.parametrize("fmt", ["coo", "csr", "dia"])
def test_stencil16_structure_spmv(mspv, orc, stencil16, fmt):
    """The small HPCG case: 16^3 grid, n = 4096, nnz = 46^3 = 97,336, 27 diagonals."""
    g, n, A, O = stencil16
    assert O.nnz == (3 * g - 2) ** 3
    M = A if fmt == "coo" else A.convert(fmt)
    Of = orc.convert(O, fmt)
    assert_structure_equal(M, Of, orc)
    if fmt == "dia":
        assert M.info["ndiags"] == 27
    x = synth.uniform_x(n, 0)
    assert_spmv_parity(M.spmv(dev(x)).cpu().numpy(), Of, x, orc)


@pytest.mark.parametrize("fmt", ["coo", "csr", "dia"])
def test_stencil16_cg_matches_oracle(mspv, orc, stencil16, fmt):
    g, n, A, O = stencil16
    M = A if fmt == "coo" else A.convert(fmt)
    Of = orc.convert(O, fmt)
    b = orc.spmv(Of, np.ones(n))
    res = M.cg(dev(b), tol=1e-10, maxit=1000)
    xo, st, k, rel, _, _ = orc.cg(Of, b, tol=1e-10, maxit=1000)
    assert res.converged and st == orc.OK
    assert abs(res.iters - k) <= 1
    assert res.relres <= 1e-10
    x = res.x.cpu().numpy()
    true = np.linalg.norm(b - orc.spmv(Of, x)) / np.linalg.norm(b)
    assert true <= 1.5e-10
    # both iterates approximate x = 1 to within kappa * 1e-10 (kappa ~ 39 at g = 16)
    assert np.max(np.abs(x - xo)) <= 1e-8
    assert np.max(np.abs(x - 1.0)) <= 40 * 1e-10 * np.sqrt(n)


@pytest.mark.parametrize("fmt", ["csr", "dia"])
def test_fixed_iterations_track_oracle(mspv, orc, stencil16, fmt):
    """tol = 0 runs exactly maxit iterations; iterates agree with the oracle's."""
    g, n, A, O = stencil16
    M = A.convert(fmt)
    Of = orc.convert(O, fmt)
    b = synth.uniform_x(n, 7)
    for k in (1, 2, 5, 20):
        res = M.cg(dev(b), tol=0.0, maxit=k)
        xo, st, ko, rel, _, _ = orc.cg(Of, b, tol=0.0, maxit=k)
        assert res.converged and res.iters == k == ko
        assert np.max(np.abs(res.x.cpu().numpy() - xo)) <= 1e-12 * np.max(np.abs(xo)) * k
        assert res.relres == pytest.approx(rel, rel=1e-9)


@pytest.mark.parametrize("vec", [1, 2, 4, 8, 16])
def test_csr_cg_every_lane_width(mspv, orc, vec, monkeypatch):
    """FP64 CG in CSR with every lane width V of the CSR kernels inside the iteration, whose
    grid is capped at 12 CTAs per SM (each CTA writes one p.q partial): on the 89^3 stencil
    (n = 704,969 rows, not a multiple of 32) the capped grid covers fewer rows than that in one
    pass, so the warps stride over the rows; fixed iterations track the oracle's iterates."""
    monkeypatch.setenv("MSPV_CSR_VEC", str(vec))
    g = 89
    n = g ** 3
    r, c, v = synth.stencil27(g)
    A = mspv.Matrix.from_coo(n, n, dev(r), dev(c), dev(v))
    C = A.convert("csr")
    assert C.info["csr_vector"] == vec
    # the generator emits canonical COO (sorted by (row, col), no duplicates)
    O = orc.coo_to_csr(orc.Matrix(orc.COO, n, n, r.size, ai=r, aj=c, av=v))
    assert n > 12 * torch.cuda.get_device_properties(0).multi_processor_count * 256
    b = synth.uniform_x(n, 8)
    for k in (1, 6):
        res = C.cg(dev(b), tol=0.0, maxit=k)
        xo, st, ko, rel, _, _ = orc.cg(O, b, tol=0.0, maxit=k)
        assert res.converged and res.iters == k == ko
        assert np.max(np.abs(res.x.cpu().numpy() - xo)) <= 1e-12 * np.max(np.abs(xo)) * k


def test_cg_nonzero_start_and_restart(mspv, orc, stencil16):
    """x0 is honoured; resuming from a saved iterate is the same as one longer run
    up to rounding (checkpoint/resume is calling again with the saved x)."""
    g, n, A, O = stencil16
    D = A.convert("dia")
    b = orc.spmv(orc.convert(O, "dia"), np.ones(n))
    x0 = synth.uniform_x(n, 3)
    res = D.cg(dev(b), x=dev(x0.copy()), tol=1e-10, maxit=1000)
    xo, st, k, rel, _, _ = orc.cg(orc.convert(O, "dia"), b, x0=x0, tol=1e-10, maxit=1000)
    assert res.converged and abs(res.iters - k) <= 1
    part = D.cg(dev(b), tol=0.0, maxit=10)
    resumed = D.cg(dev(b), x=part.x, tol=1e-10, maxit=1000)
    assert resumed.converged
    assert np.max(np.abs(resumed.x.cpu().numpy() - 1.0)) <= 1e-7


def test_cg_special_cases(mspv):
    n = 1000
    d = np.arange(1.0, n + 1)
    idx = np.arange(n, dtype=np.int32)
    A = mspv.Matrix.from_coo(n, n, idx, idx, d).convert("csr")
    # b = 0 -> x = 0, zero iterations
    res = A.cg(torch.zeros(n, dtype=torch.float64, device="cuda"),
               x=torch.ones(n, dtype=torch.float64, device="cuda"), tol=1e-10, maxit=10)
    assert res.converged and res.iters == 0 and torch.all(res.x == 0)
    # the same with a fixed iteration count (tol = 0): the b = 0 decision is the device's, and
    # the iterations launched behind it do nothing
    res = A.cg(torch.zeros(n, dtype=torch.float64, device="cuda"),
               x=torch.ones(n, dtype=torch.float64, device="cuda"), tol=0.0, maxit=300)
    assert res.converged and res.iters == 0 and torch.all(res.x == 0)
    # iteration limit -> ENOTCONV with the last iterate
    b = torch.ones(n, dtype=torch.float64, device="cuda")
    res = A.cg(b, tol=1e-14, maxit=3)
    assert res.status == 6 and res.iters == 3
    # indefinite -> EBREAKDOWN before any update
    ind = mspv.Matrix.from_coo(2, 2, np.array([0, 1], np.int32), np.array([0, 1], np.int32),
                               np.array([1.0, -1.0])).convert("dia")
    res = ind.cg(torch.ones(2, dtype=torch.float64, device="cuda"), tol=1e-10, maxit=10)
    assert res.status == 7 and res.iters == 0
    assert torch.all(res.x == 0)
    # diagonal with m distinct eigenvalues: at most m iterations
    m = 5
    dd = np.linspace(1.0, 10.0, m)[np.arange(n) % m]
    Dm = mspv.Matrix.from_coo(n, n, idx, idx, dd).convert("dia")
    res = Dm.cg(b, tol=1e-12, maxit=50)
    assert res.converged and res.iters <= m
    # rectangular -> EFORMAT
    R = mspv.Matrix.from_coo(3, 4, np.array([0], np.int32), np.array([3], np.int32), np.array([1.0]))
    with pytest.raises(mspv.MspvError, match="EFORMAT"):
        R.cg(torch.ones(3, dtype=torch.float64, device="cuda"), x=torch.zeros(3, dtype=torch.float64, device="cuda"))


def test_check_interval_does_not_change_result(mspv, stencil16, monkeypatch):
    g, n, A, O = stencil16
    D = A.convert("dia")
    b = dev(synth.uniform_x(n, 1))
    outs = []
    for every in ("1", "7", "1000"):
        monkeypatch.setenv("MSPV_CG_CHECK_EVERY", every)
        res = D.cg(b, tol=1e-10, maxit=500)
        outs.append((res.iters, res.x.cpu().numpy().copy()))
    assert outs[0][0] == outs[1][0] == outs[2][0]
    assert np.array_equal(outs[0][1], outs[1][1]) and np.array_equal(outs[0][1], outs[2][1])


@pytest.mark.parametrize("inner_fp32", [False, True], ids=["fp64_inner", "fp32_inner"])
@pytest.mark.parametrize("vt", ["f32", "bf16"])
@pytest.mark.parametrize("fmt", ["coo", "csr", "dia"])
def test_iterative_refinement(mspv, orc, vt, fmt, inner_fp32):
    """Perturbed SPD stencil whose values are not exact in FP32/BF16: the FP64 outer loop
    still reaches 1e-10 relative residual, with the inner CG in FP64 or in FP32
    arithmetic; the answer matches the oracle's refinement (FP64 inner)."""
    g = 20
    n = g ** 3
    r, c, v = synth.stencil27_perturbed(g, 3)
    A = mspv.Matrix.from_coo(n, n, dev(r), dev(c), dev(v))
    A64 = A.convert(fmt)
    Alo = A.convert(fmt, vt)
    O = orc.convert(orc.canonicalize(n, n, r, c, v), fmt)
    Olo = orc.with_values(O, vt)
    assert not np.array_equal(Olo.av, O.av)
    b = orc.spmv(O, np.ones(n))
    res = A64.cg_ir(Alo, dev(b), tol=1e-10, inner_tol=1e-4, inner_fp32=inner_fp32)
    xo, st, outer, inner, rel = orc.cg_ir(O, Olo, b, tol=1e-10, inner_tol=1e-4)
    assert res.converged and st == orc.OK
    assert res.relres <= 1e-10
    x = res.x.cpu().numpy()
    assert np.linalg.norm(b - orc.spmv(O, x)) / np.linalg.norm(b) <= 1.5e-10
    if not inner_fp32:
        assert abs(res.outer_iters - outer) <= 1
    else:
        assert res.outer_iters <= 6
    assert np.max(np.abs(x - xo)) <= 1e-8


@pytest.mark.parametrize("vt", ["f32", "bf16"])
@pytest.mark.parametrize("fmt", ["coo", "csr", "dia"])
def test_fp64_cg_on_low_precision_values_matches_oracle(mspv, orc, vt, fmt):
    """FP64 CG on FP32 / BF16 stored values (the restarted refinement's FP64 inner solver):
    same iteration count and iterate as the oracle's CG on the rounded matrix. The BF16 DIA
    kernel runs 8 rows per thread in FP64 and 4 in FP32, so its p.q partial count differs
    from the FP32 launch's: summing the wrong count corrupts alpha."""
    g = 24
    n = g ** 3
    r, c, v = synth.stencil27_perturbed(g, 5)
    A = mspv.Matrix.from_coo(n, n, dev(r), dev(c), dev(v))
    L = A.convert(fmt, vt)
    Olo = orc.with_values(orc.convert(orc.canonicalize(n, n, r, c, v), fmt), vt)
    b = synth.uniform_x(n, 8) - 0.5
    res = L.cg(dev(b), tol=1e-10, maxit=1000)
    xo, st, k, rel, _, _ = orc.cg(Olo, b, tol=1e-10, maxit=1000)
    assert res.converged and st == orc.OK
    assert abs(res.iters - k) <= 1
    assert np.max(np.abs(res.x.cpu().numpy() - xo)) <= 1e-8 * np.max(np.abs(xo))
    # and 25 fixed iterations track the oracle's iterate
    res = L.cg(dev(b), tol=0.0, maxit=25)
    xo, _, _, _, _, _ = orc.cg(Olo, b, tol=0.0, maxit=25)
    assert np.max(np.abs(res.x.cpu().numpy() - xo)) <= 1e-10 * np.max(np.abs(xo))


@pytest.mark.parametrize("vt", ["f32", "bf16"])
@pytest.mark.parametrize("fmt", ["coo", "csr", "dia"])
def test_reliable_updates_match_oracle(mspv, orc, vt, fmt):
    """One FP32 CG with reliable FP64 residual updates on the perturbed stencil: reaches
    1e-10 in the FP64 residual, agrees with the oracle's reliable-update CG (FP64
    arithmetic) to the accuracy the tolerance fixes, and with FP32 values takes FP64 CG's
    iteration count up to FP32 rounding."""
    g = 20
    n = g ** 3
    r, c, v = synth.stencil27_perturbed(g, 3)
    A = mspv.Matrix.from_coo(n, n, dev(r), dev(c), dev(v))
    A64 = A.convert(fmt)
    Alo = A.convert(fmt, vt)
    O = orc.convert(orc.canonicalize(n, n, r, c, v), fmt)
    Olo = orc.with_values(O, vt)
    b = orc.spmv(O, synth.uniform_x(n, 6) + 0.5)
    delta = 1e-2 if vt == "f32" else 1e-1
    res = A64.cg_ru(Alo, dev(b), tol=1e-10)          # library default delta for the value type
    xo, st, nu, it, rel = orc.cg_ru(O, Olo, b, tol=1e-10, delta=delta)
    assert res.converged and st == orc.OK
    assert res.relres <= 1e-10
    x = res.x.cpu().numpy()
    assert np.linalg.norm(b - orc.spmv(O, x)) / np.linalg.norm(b) <= 1.5e-10
    assert np.max(np.abs(x - xo)) <= 1e-8 * np.max(np.abs(xo))
    _, _, k64, _, _, _ = orc.cg(O, b, tol=1e-10, maxit=2000)
    if vt == "f32":
        assert abs(res.iters - k64) <= 3 and abs(res.iters - it) <= 3
    else:
        assert res.iters <= 1.5 * it
    assert 1 <= res.outer_iters <= nu + 3


@pytest.mark.parametrize("vt", ["f32", "bf16"])
def test_reliable_updates_ragged_size(mspv, orc, vt):
    """21^3 = 9,261 rows (not a multiple of the 4 or 8 rows a thread of the FP32 DIA kernel
    owns, nor of the 32-row padding): reliable updates on DIA still reach the FP64 answer."""
    g = 21
    n = g ** 3
    r, c, v = synth.stencil27_perturbed(g, 9)
    A = mspv.Matrix.from_coo(n, n, dev(r), dev(c), dev(v))
    D = A.convert("dia")
    O = orc.coo_to_dia(orc.canonicalize(n, n, r, c, v))
    b = orc.spmv(O, synth.uniform_x(n, 13) - 0.5)
    res = D.cg_ru(A.convert("dia", vt), dev(b), tol=1e-10, maxit=2000)
    assert res.converged and res.relres <= 1e-10
    x = res.x.cpu().numpy()
    assert np.linalg.norm(b - orc.spmv(O, x)) / np.linalg.norm(b) <= 1.5e-10
    xo, st, _, _, _, _ = orc.cg(O, b, tol=1e-12, maxit=2000)
    assert st == orc.OK and np.max(np.abs(x - xo)) <= 1e-8 * np.max(np.abs(xo))


def test_reliable_updates_large_dia(mspv):
    """64^3 perturbed stencil (262,144 rows) in DIA: FP32 values take at most 5% more
    iterations than FP64 CG, BF16 values at most 40% more; both reach 1e-10."""
    g = 64
    n = g ** 3
    r, c, v = synth.stencil27_perturbed(g, 3)
    A = mspv.Matrix.from_coo(n, n, dev(r), dev(c), dev(v))
    D = A.convert("dia")
    b = D.spmv(dev(synth.uniform_x(n, 7) + 0.5))
    ref = D.cg(b, tol=1e-10, maxit=5000)
    assert ref.converged
    for vt, factor in (("f32", 1.05), ("bf16", 1.4)):
        res = D.cg_ru(A.convert("dia", vt), b, tol=1e-10, maxit=5000)
        assert res.converged and res.relres <= 1e-10
        assert res.iters <= factor * ref.iters + 2, (vt, res.iters, ref.iters)
        true = torch.linalg.norm(b - D.spmv(res.x)) / torch.linalg.norm(b)
        assert float(true) <= 1.5e-10


def test_reliable_updates_special_cases(mspv, stencil16):
    g, n, A, O = stencil16
    D = A.convert("csr")
    L = A.convert("csr", "f32")
    # b = 0: x = 0 without iterating
    res = D.cg_ru(L, torch.zeros(n, dtype=torch.float64, device="cuda"),
                  x=torch.ones(n, dtype=torch.float64, device="cuda"))
    assert res.converged and res.iters == 0 and res.outer_iters == 0 and not torch.any(res.x)
    # start at the solution (the stencil maps ones to its row sums)
    b = D.spmv(torch.ones(n, dtype=torch.float64, device="cuda"))
    res = D.cg_ru(L, b, x=torch.ones(n, dtype=torch.float64, device="cuda"))
    assert res.converged and res.iters == 0 and res.outer_iters == 0
    # iteration limit: not converged after exactly maxit FP32 iterations
    res = D.cg_ru(L, b, tol=1e-14, maxit=7)
    assert res.status == 6 and res.iters == 7 and res.outer_iters >= 1
    # update limit
    res = D.cg_ru(L, b, tol=1e-14, delta=0.9, max_updates=2)
    assert res.status == 6 and res.outer_iters == 2
    with pytest.raises(mspv.MspvError, match="EINVAL"):
        D.cg_ir(L, b, inner_fp32=3)
    with pytest.raises(mspv.MspvError, match="EFORMAT"):
        D.cg_ru(D, b)


def test_fp32_inner_needs_low_precision_values(mspv, stencil16):
    g, n, A, O = stencil16
    D = A.convert("dia")
    with pytest.raises(mspv.MspvError, match="EFORMAT"):
        D.cg_ir(D, dev(np.ones(n)), inner_fp32=True)


def test_cg_with_an_unaligned_solution_vector(mspv, stencil16):
    """x may be any 8-byte-aligned view (here offset by one element); the iterate is the
    same as with an aligned x."""
    g, n, A, O = stencil16
    D = A.convert("dia")
    b = dev(synth.uniform_x(n, 4))
    buf = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    xu = buf[1:]
    assert xu.data_ptr() % 16 == 8
    r1 = D.cg(b, x=xu, tol=0.0, maxit=15)
    r2 = D.cg(b, tol=0.0, maxit=15)
    assert r1.iters == r2.iters == 15
    assert torch.equal(r1.x, r2.x)


@pytest.mark.parametrize("fmt", ["csr", "coo"])
@pytest.mark.parametrize("mean_len", [6, 60])
def test_cg_with_long_rows_matches_oracle(mspv, orc, fmt, mean_len):
    """SPD matrices whose CSR form lists long rows (a few dense rows and columns) and whose
    mean row length selects V = 4 or V = 8: inside CG the V-lane kernel runs on a capped grid
    and the long-row kernel writes its p.q partials after it; COO takes the segment kernel.
    Fixed iterations track the oracle's iterates."""
    rng = np.random.default_rng(mean_len)
    n = 200_000
    m = n * mean_len // 2
    r = rng.integers(0, n, m)
    c = rng.integers(0, n, m)
    hubs = rng.choice(n, 6, replace=False)
    hr = np.repeat(hubs, 3000)
    hc = rng.integers(0, n, hr.size)
    r = np.concatenate([r, hr])
    c = np.concatenate([c, hc])
    keep = r != c
    r, c = r[keep], c[keep]
    v = -rng.uniform(0.1, 1.0, r.size)
    rows = np.concatenate([r, c, np.arange(n)])          # symmetric off-diagonal part
    cols = np.concatenate([c, r, np.arange(n)])
    absrow = np.bincount(np.concatenate([r, c]), weights=np.abs(np.concatenate([v, v])), minlength=n)
    vals = np.concatenate([v, v, absrow + 1.0])           # strictly diagonally dominant
    A = mspv.Matrix.from_coo(n, n, dev(rows.astype(np.int32)), dev(cols.astype(np.int32)), dev(vals))
    M = A if fmt == "coo" else A.convert(fmt)
    if fmt == "csr":
        info = M.info
        assert info["csr_vector"] == (4 if mean_len < 48 else 8) and info["row_max"] > 32 * info["csr_vector"]
    O = orc.convert(orc.canonicalize(n, n, rows, cols, vals), fmt)
    b = synth.uniform_x(n, 3)
    for k in (3, 12):
        res = M.cg(dev(b), tol=0.0, maxit=k)
        xo, st, ko, rel, _, _ = orc.cg(O, b, tol=0.0, maxit=k)
        assert res.iters == k == ko
        assert np.max(np.abs(res.x.cpu().numpy() - xo)) <= 1e-11 * np.max(np.abs(xo))
        assert res.relres == pytest.approx(rel, rel=1e-8)
