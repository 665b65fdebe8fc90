"""Pins for the FP64 oracle: each test checks it against something other than
itself -- the dense definition of A*x, brute force on tiny inputs, closed forms of
the 27-point stencil, exact rational CG, and textbook CG properties. CPU only."""
from fractions import Fraction

import numpy as np
import pytest

import synth

U = 2.0 ** -53  # unit roundoff, FP64


def dense_of(nrows, ncols, rows, cols, vals):
    """Dense matrix with duplicates summed (the definition, via numpy scatter-add)."""
    D = np.zeros((nrows, ncols))
    np.add.at(D, (rows, cols), vals)
    return D


def assert_spmv_close(y, D, x, k_max):
    """|y - D x| <= tol * (|D| |x|), tol = max(1e-13, 2 (k+2) u) for rows of <= k terms:
    any two summation orders of k products each lie within gamma_k |D||x| of the exact sum."""
    ref = D @ x
    scale = np.abs(D) @ np.abs(x)
    tol = max(1e-13, 2 * (k_max + 2) * U)
    assert np.all(np.abs(y - ref) <= tol * scale + 1e-300), np.max(np.abs(y - ref) - tol * scale)


SMALL_CASES = [
    # (nrows, ncols, nnz, seed, dup_frac, empty_rows)
    (1, 1, 1, 0, 0.0, 0),
    (1, 1, 3, 1, 0.6, 0),
    (5, 5, 11, 2, 0.0, 0),
    (7, 13, 30, 3, 0.2, 2),
    (13, 7, 30, 4, 0.2, 3),
    (33, 33, 200, 5, 0.1, 4),
    (64, 64, 700, 6, 0.3, 9),
    (64, 64, 4096, 7, 0.0, 0),
    (40, 64, 0, 8, 0.0, 0),
    (64, 17, 64 * 17, 9, 0.5, 0),
]


@pytest.mark.parametrize("case", SMALL_CASES)
def test_spmv_matches_dense_brute_force(orc, case):
    nrows, ncols, nnz, seed, dup, empty = case
    r, c, v = synth.random_coo(nrows, ncols, nnz, seed, dup_frac=dup, empty_rows=empty)
    D = dense_of(nrows, ncols, r, c, v)
    x = synth.uniform_x(ncols, seed) * 2 - 1
    A = orc.canonicalize(nrows, ncols, r, c, v)
    kmax = max(int(np.bincount(r, minlength=1).max()) if nnz else 0, 1)
    assert_spmv_close(orc.spmv(A, x), D, x, kmax)
    C = orc.coo_to_csr(A)
    assert_spmv_close(orc.spmv(C, x), D, x, kmax)
    if nrows == ncols:
        Dg = orc.coo_to_dia(A)
        assert_spmv_close(orc.spmv(Dg, x), D, x, kmax)


@pytest.mark.parametrize("case", SMALL_CASES)
def test_canonical_coo_brute_force(orc, case):
    """Sorted unique (row, col); each value is the input-order left-to-right sum of its
    duplicates (Python floats are IEEE FP64, so this is exact)."""
    nrows, ncols, nnz, seed, dup, empty = case
    r, c, v = synth.random_coo(nrows, ncols, nnz, seed, dup_frac=dup, empty_rows=empty)
    acc = {}
    for ri, ci, vi in zip(r.tolist(), c.tolist(), v.tolist()):
        acc[(ri, ci)] = acc[(ri, ci)] + vi if (ri, ci) in acc else vi
    keys = sorted(acc)
    A = orc.canonicalize(nrows, ncols, r, c, v)
    assert A.nnz == len(keys)
    assert [(int(a), int(b)) for a, b in zip(A.ai, A.aj)] == keys
    assert A.av.tolist() == [acc[k] for k in keys]


def test_canonicalize_rejects_out_of_range(orc):
    with pytest.raises(ValueError):
        orc.canonicalize(3, 3, np.array([0, 3]), np.array([0, 0]), np.array([1.0, 2.0]))
    with pytest.raises(ValueError):
        orc.canonicalize(3, 3, np.array([0, 1]), np.array([-1, 0]), np.array([1.0, 2.0]))


@pytest.mark.parametrize("case", SMALL_CASES)
def test_csr_structure_and_round_trip(orc, case):
    nrows, ncols, nnz, seed, dup, empty = case
    r, c, v = synth.random_coo(nrows, ncols, nnz, seed, dup_frac=dup, empty_rows=empty)
    A = orc.canonicalize(nrows, ncols, r, c, v)
    C = orc.coo_to_csr(A)
    assert C.irp[0] == 0 and C.irp[-1] == A.nnz
    assert np.all(np.diff(C.irp) >= 0)
    assert np.array_equal(np.diff(C.irp), np.bincount(A.ai, minlength=nrows)[:nrows])
    B = orc.csr_to_coo(C)
    assert np.array_equal(B.ai, A.ai) and np.array_equal(B.aj, A.aj)
    assert np.array_equal(B.av, A.av)


@pytest.mark.parametrize("case", [c for c in SMALL_CASES if c[0] == c[1]])
def test_dia_structure_and_round_trip(orc, case):
    nrows, ncols, nnz, seed, dup, empty = case
    r, c, v = synth.random_coo(nrows, ncols, nnz, seed, dup_frac=dup, empty_rows=empty)
    A = orc.canonicalize(nrows, ncols, r, c, v)
    D = dense_of(nrows, ncols, A.ai, A.aj, A.av)
    G = orc.coo_to_dia(A)
    n = nrows
    assert G.npad % 32 == 0 and n <= G.npad < n + 32
    assert np.array_equal(G.doff, np.unique(A.aj.astype(np.int64) - A.ai))
    AV = G.av.reshape(G.ndiags, G.npad)
    for j, off in enumerate(G.doff.tolist()):
        for i in range(G.npad):
            k = i + off
            want = D[i, k] if (i < n and 0 <= k < n) else 0.0
            assert AV[j, i] == want
    # round trip on entries without explicit zeros (DIA cannot tell a zero from padding)
    keep = A.av != 0.0
    B = orc.dia_to_coo(G)
    assert np.array_equal(B.ai, A.ai[keep]) and np.array_equal(B.aj, A.aj[keep])
    assert np.array_equal(B.av, A.av[keep])


def test_dia_drops_explicit_zeros(orc):
    r = np.array([0, 1, 1, 2])
    c = np.array([0, 1, 2, 0])
    v = np.array([1.0, 0.0, 2.0, 3.0])
    A = orc.canonicalize(3, 3, r, c, v)
    assert A.nnz == 4  # COO keeps the explicit zero
    B = orc.dia_to_coo(orc.coo_to_dia(A))
    assert B.nnz == 3 and list(zip(B.ai.tolist(), B.aj.tolist())) == [(0, 0), (1, 2), (2, 0)]


# ---------------------------------------------------------------------------
# 27-point stencil closed forms
# ---------------------------------------------------------------------------

def sep3(x3):
    """(T x T x T) x with T = tridiag(1, 1, 1): three independent 3-point passes."""
    out = x3
    for ax in range(3):
        s = out.copy()
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax], hi[ax] = slice(0, -1), slice(1, None)
        s[tuple(lo)] += out[tuple(hi)]
        s[tuple(hi)] += out[tuple(lo)]
        out = s
    return out


def stencil_apply_closed_form(g, x):
    """A x with A = 27 I - T(x)T(x)T: diagonal 27 - 1 = 26, each neighbour -1."""
    x3 = x.reshape(g, g, g)
    return (27.0 * x3 - sep3(x3)).ravel(), (25.0 * np.abs(x3) + sep3(np.abs(x3))).ravel()


@pytest.mark.parametrize("g", [2, 3, 5, 16, 24])
def test_stencil_structure(orc, g):
    r, c, v = synth.stencil27(g)
    n = g ** 3
    assert r.size == (3 * g - 2) ** 3
    A = orc.canonicalize(n, n, r, c, v)
    assert A.nnz == (3 * g - 2) ** 3
    C = orc.coo_to_csr(A)
    lens = np.diff(C.irp)
    # a row's length is prod over the 3 axes of (2 at a face, 3 inside)
    want = {}
    for kb in range(4):  # number of axes on which the point sits on a face
        from math import comb
        length = 3 ** (3 - kb) * 2 ** kb
        count = comb(3, kb) * (2 ** kb) * max(g - 2, 0) ** (3 - kb) if g > 1 else 0
        want[length] = want.get(length, 0) + count
    got = {int(k): int(cnt) for k, cnt in zip(*np.unique(lens, return_counts=True))}
    assert got == {k: c for k, c in want.items() if c}
    # b = A 1 has b_i = 27 - len_i exactly: interior rows sum to zero
    b = orc.spmv(C, np.ones(n))
    assert np.array_equal(b, 27.0 - lens)
    G = orc.coo_to_dia(A)
    offs = sorted({dz * g * g + dy * g + dx for dz in (-1, 0, 1) for dy in (-1, 0, 1)
                   for dx in (-1, 0, 1)})
    if g >= 3:
        assert G.doff.tolist() == offs
    assert np.count_nonzero(G.av) == A.nnz


@pytest.mark.parametrize("g", [4, 16, 24])
@pytest.mark.parametrize("fmt", ["coo", "csr", "dia"])
def test_stencil_spmv_matches_separable_closed_form(orc, g, fmt):
    n = g ** 3
    r, c, v = synth.stencil27(g)
    A = orc.convert(orc.canonicalize(n, n, r, c, v), fmt)
    x = synth.uniform_x(n, 0)
    ref, scale = stencil_apply_closed_form(g, x)
    y = orc.spmv(A, x)
    assert np.all(np.abs(y - ref) <= 1e-13 * scale)


def stencil_eigs(g):
    """Eigenvalues of A = 27 I - T(x)T(x)T: T has eigenvalues 1 + 2 cos(k pi/(g+1))."""
    t = 1.0 + 2.0 * np.cos(np.arange(1, g + 1) * np.pi / (g + 1))
    return 27.0 - np.einsum("i,j,k->ijk", t, t, t).ravel()


@pytest.mark.parametrize("g", [3, 5, 7])
def test_stencil_eigenvalue_closed_form(orc, g):
    n = g ** 3
    r, c, v = synth.stencil27(g)
    D = dense_of(n, n, r, c, v)
    assert np.allclose(np.sort(stencil_eigs(g)), np.linalg.eigvalsh(D), atol=1e-10)


# ---------------------------------------------------------------------------
# CG
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("g", [8, 16])
@pytest.mark.parametrize("fmt", ["csr", "dia", "coo"])
def test_cg_recovers_ones(orc, g, fmt):
    n = g ** 3
    r, c, v = synth.stencil27(g)
    A = orc.convert(orc.canonicalize(n, n, r, c, v), fmt)
    lam = stencil_eigs(g)
    kappa = lam.max() / lam.min()
    b = orc.spmv(A, np.ones(n))
    x, st, k, rel, hist, aerr = orc.cg(A, b, tol=1e-10, maxit=2000, xstar=np.ones(n))
    assert st == orc.OK
    assert rel <= 1e-10 and hist[-1] == pytest.approx(rel)
    # the textbook bound on iterations: sqrt(kappa)/2 * ln(2/eps) with eps the A-norm
    # error reduction; eps <= tol / sqrt(kappa) suffices for the residual test
    bound = int(np.ceil(np.sqrt(kappa) / 2 * np.log(2 * np.sqrt(kappa) / 1e-10)))
    assert k <= bound
    # forward error bounded by kappa times the relative residual
    assert np.linalg.norm(x - 1) / np.sqrt(n) <= kappa * rel * 1.01
    # A-norm error is monotonically non-increasing (rounding slack 1e-12 of its start)
    assert np.all(np.diff(aerr) <= 1e-12 * aerr[0])
    # true residual agrees with the recursive one
    true = np.linalg.norm(b - orc.spmv(A, x)) / np.linalg.norm(b)
    assert true <= 2e-10


def test_cg_diagonal_distinct_eigenvalues(orc):
    """CG on an SPD matrix with m distinct eigenvalues ends in at most m iterations."""
    for m in (1, 2, 3, 5, 8):
        n = 200
        eig = np.linspace(1.0, 10.0, m)
        d = eig[np.arange(n) % m]
        A = orc.canonicalize(n, n, np.arange(n), np.arange(n), d)
        b = synth.uniform_x(n, m) + 0.5
        x, st, k, rel, _, _ = orc.cg(A, b, tol=1e-12, maxit=50)
        assert st == orc.OK and k <= m
        assert np.allclose(x, b / d, rtol=1e-11)


def _exact_cg(M, b, iters):
    """CG in exact rational arithmetic (fractions), from x0 = 0."""
    n = len(b)
    x = [Fraction(0)] * n
    r = list(b)
    p = list(r)
    rho = sum(ri * ri for ri in r)
    out = []
    for _ in range(iters):
        q = [sum(M[i][j] * p[j] for j in range(n)) for i in range(n)]
        alpha = rho / sum(p[i] * q[i] for i in range(n))
        x = [x[i] + alpha * p[i] for i in range(n)]
        r = [r[i] - alpha * q[i] for i in range(n)]
        rho_new = sum(ri * ri for ri in r)
        beta = rho_new / rho
        rho = rho_new
        p = [r[i] + beta * p[i] for i in range(n)]
        out.append([float(t) for t in x])
    return out


def test_cg_iterates_match_exact_rational_cg(orc):
    rng = np.random.default_rng(11)
    n = 7
    B = rng.integers(-3, 4, size=(n, n))
    M = B @ B.T + n * np.eye(n, dtype=np.int64)  # SPD, integer
    b = rng.integers(-5, 6, size=n)
    exact = _exact_cg([[Fraction(int(t)) for t in row] for row in M],
                      [Fraction(int(t)) for t in b], n - 1)
    rows, cols = np.nonzero(M)
    A = orc.canonicalize(n, n, rows, cols, M[rows, cols].astype(float))
    for k in range(1, n):
        x, st, it, _, _, _ = orc.cg(A, b.astype(float), tol=0.0, maxit=k)
        assert st == orc.OK and it == k
        assert np.allclose(x, exact[k - 1], rtol=1e-12, atol=1e-12)


def test_cg_special_cases(orc):
    n = 10
    A = orc.canonicalize(n, n, np.arange(n), np.arange(n), np.arange(1.0, n + 1))
    # b = 0 -> x = 0, zero iterations
    x, st, k, rel, _, _ = orc.cg(A, np.zeros(n), x0=np.ones(n), tol=1e-10, maxit=5)
    assert st == orc.OK and k == 0 and np.all(x == 0)
    # too few iterations -> not converged, last iterate kept
    x, st, k, rel, _, _ = orc.cg(A, np.ones(n), tol=1e-14, maxit=3)
    assert st == orc.NOTCONV and k == 3 and rel > 1e-14
    # tol <= 0 runs exactly maxit iterations and reports success
    x, st, k, rel, _, _ = orc.cg(A, np.ones(n), tol=0.0, maxit=4)
    assert st == orc.OK and k == 4
    # indefinite matrix: p.Ap <= 0 is a breakdown
    Aind = orc.canonicalize(2, 2, np.array([0, 1]), np.array([0, 1]), np.array([1.0, -1.0]))
    x, st, k, rel, _, _ = orc.cg(Aind, np.array([1.0, 1.0]), tol=1e-10, maxit=10)
    assert st == orc.BREAKDOWN and k == 0 and np.all(x == 0)
    # already converged start
    x, st, k, rel, _, _ = orc.cg(A, np.arange(1.0, n + 1), x0=np.ones(n), tol=1e-10, maxit=10)
    assert st == orc.OK and k == 0


# ---------------------------------------------------------------------------
# storage rounding
# ---------------------------------------------------------------------------

def _bf16_by_bits(v):
    """BF16 round-to-nearest-even from FP64 by integer arithmetic on the FP64 bits:
    keep 7 explicit mantissa bits (45 bits dropped) and round the dropped part."""
    out = []
    for t in np.asarray(v, np.float64).tolist():
        bits = np.array([t], np.float64).view(np.uint64)[0].item()
        sign, rest = bits >> 63, bits & ((1 << 63) - 1)
        drop = 52 - 7
        low = rest & ((1 << drop) - 1)
        kept = rest >> drop
        half = 1 << (drop - 1)
        if low > half or (low == half and (kept & 1)):
            kept += 1
        res = np.array([(sign << 63) | (kept << drop)], np.uint64).view(np.float64)[0]
        out.append(float(res))
    return np.array(out)


def test_round_values(orc):
    rng = np.random.default_rng(5)
    v = np.concatenate([rng.uniform(-4, 4, 5000), rng.normal(0, 1e3, 1000),
                        [1.0, -1.0, 26.0, -26.0, 0.0, 1 + 2**-8, 1 + 3 * 2**-8,
                         1 + 2**-8 + 2**-30, 3.0e38]])
    assert np.array_equal(orc.round_values(v, "f32"), v.astype(np.float32).astype(np.float64))
    bf = orc.round_values(v, "bf16")
    assert np.array_equal(bf[:-1], _bf16_by_bits(v[:-1]))
    # ties to even, and no double rounding through FP32
    assert orc.round_values([1 + 2**-8], "bf16")[0] == 1.0
    assert orc.round_values([1 + 3 * 2**-8], "bf16")[0] == 1 + 2**-6
    assert orc.round_values([1 + 2**-8 + 2**-30], "bf16")[0] == 1 + 2**-7
    assert np.isinf(orc.round_values([3.5e38], "bf16")[0])
    # stencil values are exact in both
    assert np.array_equal(orc.round_values([26.0, -1.0], "bf16"), [26.0, -1.0])


def test_cg_ir_reaches_fp64_tolerance_with_bf16_values(orc):
    g = 12
    n = g ** 3
    r, c, v = synth.stencil27_perturbed(g, 3)
    A = orc.canonicalize(n, n, r, c, v)
    C = orc.coo_to_csr(A)
    Clo = orc.with_values(C, "bf16")
    assert not np.array_equal(Clo.av, C.av)  # the rounding is exercised
    b = orc.spmv(C, np.ones(n))
    x, st, outer, inner, rel = orc.cg_ir(C, Clo, b, tol=1e-10, inner_tol=1e-3)
    assert st == orc.OK and rel <= 1e-10 and outer >= 2
    true = np.linalg.norm(b - orc.spmv(C, x)) / np.linalg.norm(b)
    assert true <= 1e-10 and np.max(np.abs(x - 1)) < 1e-8


def check_refinement_outer_steps(orc, vt="bf16"):
    """Iterative refinement with exact inner solves is the stationary iteration
    x_{k+1} = x_k + Alo^{-1} (b - A64 x_k). On a perturbed stencil small enough for dense
    elimination, with the inner CG run to 1e-14, the oracle's k-th outer iterate must be
    that recursion's (to cond * 1e-13), its reported residual the recursion's FP64 residual,
    and each outer step must contract the residual by at most ||I - A64 Alo^{-1}||_2. The
    first iterate is Alo^{-1} b, which differs from A64^{-1} b by the storage rounding, so an
    inner solve on the FP64 matrix, a residual taken from the rounded matrix or a wrong sign
    in the update each fail here."""
    g = 5
    n = g ** 3
    r, c, v = synth.stencil27_perturbed(g, 3)
    C = orc.coo_to_csr(orc.canonicalize(n, n, r, c, v))
    Clo = orc.with_values(C, vt)
    D = dense_of(n, n, orc.csr_to_coo(C).ai, C.aj, C.av)
    Dlo = dense_of(n, n, orc.csr_to_coo(C).ai, C.aj, Clo.av)
    assert not np.array_equal(D, Dlo)
    cond = np.linalg.cond(Dlo)
    contraction = np.linalg.norm(np.eye(n) - D @ np.linalg.inv(Dlo), 2)
    assert contraction < 1.0
    b = synth.uniform_x(n, 4) - 0.5
    bnorm = np.linalg.norm(b)
    xd = np.zeros(n)
    prev = 1.0
    for k in (1, 2, 3):
        xd = xd + np.linalg.solve(Dlo, b - D @ xd)
        want_rel = np.linalg.norm(b - D @ xd) / bnorm
        x, st, outer, inner, rel = orc.cg_ir(C, Clo, b, tol=1e-300, inner_tol=1e-14,
                                             max_outer=k, maxit_inner=5000)
        assert st == orc.NOTCONV and outer == k and inner > 0
        assert np.linalg.norm(x - xd) <= cond * 1e-13 * np.linalg.norm(xd)
        assert abs(rel - want_rel) <= 1e-12
        assert rel <= contraction * prev + 1e-12
        prev = rel
        if k == 1:
            # the storage rounding is visible far above the tolerance
            x64 = np.linalg.solve(D, b)
            assert np.linalg.norm(x - x64) > 1e3 * cond * 1e-13 * np.linalg.norm(x64)


@pytest.mark.parametrize("vt", ["bf16", "f32"])
def test_cg_ir_outer_steps_follow_dense_refinement(orc, vt):
    check_refinement_outer_steps(orc, vt)


def test_cg_ru_iterates_match_exact_rational_cg(orc):
    """With both matrices equal, the replaced residual is the recursive one up to rounding,
    so reliable updates after every iteration (delta = 2) reproduce the textbook iterates
    of exact rational CG: this pins the direction p = r + beta p formed after each update."""
    rng = np.random.default_rng(12)
    n = 7
    B = rng.integers(-3, 4, size=(n, n))
    M = B @ B.T + n * np.eye(n, dtype=np.int64)
    b = rng.integers(-5, 6, size=n)
    exact = _exact_cg([[Fraction(int(t)) for t in row] for row in M],
                      [Fraction(int(t)) for t in b], n - 1)
    rows, cols = np.nonzero(M)
    A = orc.canonicalize(n, n, rows, cols, M[rows, cols].astype(float))
    for k in range(1, n):
        for delta in (2.0, 1e-30):   # update after every iteration / only at maxit
            x, st, nu, it, _ = orc.cg_ru(A, A, b.astype(float), tol=1e-300, delta=delta, maxit=k)
            assert it == k and nu == (k if delta > 1 else 1)
            assert np.allclose(x, exact[k - 1], rtol=1e-12, atol=1e-12)


def test_cg_ru_finite_termination(orc):
    """SPD diagonal with m distinct eigenvalues: at most m iterations, as for CG."""
    for m in (1, 2, 3, 5):
        n = 120
        eig = np.linspace(1.0, 10.0, m)
        d = eig[np.arange(n) % m]
        A = orc.canonicalize(n, n, np.arange(n), np.arange(n), d)
        b = synth.uniform_x(n, m) + 0.5
        x, st, nu, it, rel = orc.cg_ru(A, A, b, tol=1e-12, delta=1e-2, maxit=50)
        assert st == orc.OK and it <= m and rel <= 1e-12
        assert np.allclose(x, b / d, rtol=1e-11)


@pytest.mark.parametrize("vt", ["f32", "bf16"])
def test_cg_ru_solves_the_fp64_system(orc, vt):
    """Perturbed SPD stencil whose values round in FP32 / BF16: the answer is the solution
    of the FP64 system by dense elimination (not that of the rounded matrix), with the
    error bound cond(A) * tol; equal matrices take exactly textbook CG's iteration count."""
    g = 6
    n = g ** 3
    r, c, v = synth.stencil27_perturbed(g, 3)
    A = orc.canonicalize(n, n, r, c, v)
    Alo = orc.with_values(A, vt)
    assert not np.array_equal(Alo.av, A.av)
    D = dense_of(n, n, A.ai, A.aj, A.av)
    Dlo = dense_of(n, n, Alo.ai, Alo.aj, Alo.av)
    b = synth.uniform_x(n, 2) - 0.5
    xs = np.linalg.solve(D, b)
    x_lo = np.linalg.solve(Dlo, b)
    cond = np.linalg.cond(D)
    tol = 1e-11
    x, st, nu, it, rel = orc.cg_ru(A, Alo, b, tol=tol, delta=0.1, maxit=2000)
    assert st == orc.OK and rel <= tol and nu >= 2
    assert np.linalg.norm(b - D @ x) / np.linalg.norm(b) <= tol * 1.01
    err = np.linalg.norm(x - xs) / np.linalg.norm(xs)
    assert err <= 2 * cond * tol
    # the rounded matrix's own solution is far off: the pin sees which system was solved
    assert np.linalg.norm(x_lo - xs) / np.linalg.norm(xs) > 1e3 * err
    xc, stc, kc, _, _, _ = orc.cg(A, b, tol=tol, maxit=2000)
    x2, st2, nu2, it2, _ = orc.cg_ru(A, A, b, tol=tol, delta=0.1, maxit=2000)
    assert st2 == orc.OK and abs(it2 - kc) <= 1


def test_cg_ru_special_cases(orc):
    n = 10
    A = orc.canonicalize(n, n, np.arange(n), np.arange(n), np.arange(1.0, n + 1))
    x, st, nu, it, rel = orc.cg_ru(A, A, np.zeros(n), x0=np.ones(n))
    assert st == orc.OK and nu == 0 and it == 0 and np.all(x == 0)
    x, st, nu, it, rel = orc.cg_ru(A, A, np.arange(1.0, n + 1), x0=np.ones(n))
    assert st == orc.OK and nu == 0 and it == 0
    x, st, nu, it, rel = orc.cg_ru(A, A, np.ones(n), tol=1e-14, maxit=3)
    assert st == orc.NOTCONV and it == 3 and nu >= 1 and rel > 1e-14
    x, st, nu, it, rel = orc.cg_ru(A, A, np.ones(n), tol=1e-14, delta=0.999, max_updates=2)
    assert st == orc.NOTCONV and nu == 2
    Aind = orc.canonicalize(2, 2, np.array([0, 1]), np.array([0, 1]), np.array([1.0, -1.0]))
    x, st, nu, it, rel = orc.cg_ru(Aind, Aind, np.array([1.0, 1.0]))
    assert st == orc.BREAKDOWN and it == 0 and np.all(x == 0)


@pytest.mark.parametrize("dims", [(3, 4, 5), (6, 6, 6), (9, 5, 7)])
def test_hpcg_rank_split_closed_forms(orc, dims):
    """An interior process's matrix: 27 entries per row; the local part is the block's own
    27-point stencil ((3nx-2)(3ny-2)(3nz-2) entries, bit-identical to the stencil generator for
    cubes); ghosts are the (nx+2)(ny+2)(nz+2) - n cells around the block."""
    nx, ny, nz = dims
    r, c, v, n, ng = synth.hpcg_rank_matrix(nx, ny, nz)
    assert ng == (nx + 2) * (ny + 2) * (nz + 2) - n
    O = orc.canonicalize(n, n + ng, r, c, v)
    assert O.nnz == 27 * n
    loc, rem = orc.split_columns(O, n)
    assert loc.nnz == (3 * nx - 2) * (3 * ny - 2) * (3 * nz - 2)
    assert rem.nnz == 27 * n - loc.nnz and rem.ncols == ng
    assert np.all(np.diff(loc.ai) >= 0) and np.all(np.diff(rem.ai) >= 0)
    if nx == ny == nz:
        sr, sc, sv = synth.stencil27(nx)
        assert np.array_equal(loc.ai, sr) and np.array_equal(loc.aj, sc) and np.array_equal(loc.av, sv)
    # b = A 1 is 26 - 26 = 0 on every row (all 27 neighbours exist)
    assert np.all(orc.spmv(O, np.ones(n + ng)) == 0.0)
    # every ghost column is used, and only by rows on the block's surface
    assert np.array_equal(np.unique(rem.aj), np.arange(ng))
    ix, iy, iz = rem.ai % nx, (rem.ai // nx) % ny, rem.ai // (nx * ny)
    assert np.all((ix == 0) | (ix == nx - 1) | (iy == 0) | (iy == ny - 1) | (iz == 0) | (iz == nz - 1))


def test_split_spmv_adds_up(orc):
    """A x = local x[:c] + remote x[c:] exactly for integer data (every partial sum exact)."""
    rng = np.random.default_rng(5)
    nr, nc, c = 40, 70, 33
    r = rng.integers(0, nr, 600)
    col = rng.integers(0, nc, 600)
    v = rng.integers(-4, 5, 600).astype(np.float64)
    O = orc.canonicalize(nr, nc, r, col, v)
    x = rng.integers(-3, 4, nc).astype(np.float64)
    loc, rem = orc.split_columns(O, c)
    assert loc.nnz + rem.nnz == O.nnz and loc.ncols == c and rem.ncols == nc - c
    assert np.array_equal(orc.spmv(O, x), orc.spmv(loc, x[:c]) + orc.spmv(rem, x[c:]))
    for cut in (0, nc):
        a, b = orc.split_columns(O, cut)
        assert (a.nnz, b.nnz) == ((0, O.nnz) if cut == 0 else (O.nnz, 0))
