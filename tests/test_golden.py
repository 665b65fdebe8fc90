"""Stored expected values (tests/golden/, written by tests/golden/make_golden.py from the oracle
alone): each fixture is checked against closed forms on the CPU, reproduced by the oracle, and
(-m gpu) matched by the CUDA path."""
import itertools
import math
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if not ln.startswith("#")]


def load_dia():
    ls = _lines("stencil4_dia.txt")
    n, nd, npad = map(int, ls[0])
    doff = np.array(ls[1], dtype=np.int64)
    av = np.array([[float(t) for t in row] for row in ls[2:2 + nd]])
    return n, nd, npad, doff, av


def load_cg():
    ls = _lines("cg_stencil8.txt")
    st, k = int(ls[0][0]), int(ls[0][1])
    return st, k, float(ls[0][2]), np.array([float(r[0]) for r in ls[1:]])


def load_split():
    ls = _lines("rank_split_3x4x5.txt")
    n, ng, nl, nr = map(int, ls[0])
    trip = np.array([[float(t) for t in row] for row in ls[1:]])
    return n, ng, nl, nr, trip


# ---------------------------------------------------------------- closed forms (CPU)
def test_stencil4_dia_closed_form():
    """Offsets dz*16 + dy*4 + dx in ascending order; slot (d, i) holds 26 on the main
    diagonal, -1 where the neighbour is inside the grid, 0 elsewhere (and in padding)."""
    g = 4
    n, nd, npad, doff, av = load_dia()
    assert (n, nd, npad) == (64, 27, 64)
    offs = sorted(dz * g * g + dy * g + dx for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3))
    assert list(doff) == offs
    for d, (dz, dy, dx) in enumerate(sorted(itertools.product((-1, 0, 1), repeat=3),
                                            key=lambda t: t[0] * 16 + t[1] * 4 + t[2])):
        for i in range(npad):
            ix, iy, iz = i % g, (i // g) % g, i // (g * g)
            inside = i < n and 0 <= ix + dx < g and 0 <= iy + dy < g and 0 <= iz + dz < g
            want = 0.0 if not inside else (26.0 if (dx, dy, dz) == (0, 0, 0) else -1.0)
            assert av[d, i] == want


def test_cg_stencil8_within_the_excited_spectrum():
    """b = A 1 on the 8^3 stencil only excites modes with odd wave numbers in every axis
    (the eigenvectors of T = tridiag(1, 1, 1) are sines; 1 is orthogonal to the even ones), so
    exact CG ends within the number of distinct eigenvalues 27 - prod(1 + 2 cos(k pi / 9))
    over odd k: the stored run converges no later, with a residual history that ends at the
    reported relative residual."""
    st, k, rel, hist = load_cg()
    c = [1 + 2 * math.cos(kk * math.pi / 9) for kk in (1, 3, 5, 7)]
    distinct = {round(27 - a * b * d, 9) for a, b, d in itertools.product(c, repeat=3)}
    assert st == 0 and 1 <= k <= len(distinct)
    assert hist[0] == 1.0 and len(hist) == k + 1
    assert rel <= 1e-10 and hist[-1] == pytest.approx(rel, rel=1e-12)
    assert np.all(hist[:-1] > 1e-10)


def test_rank_split_closed_form():
    n, ng, nl, nr, trip = load_split()
    assert n == 60 and ng == 5 * 6 * 7 - 60
    assert nl == 7 * 10 * 13 and nl + nr == 27 * n and len(trip) == nr
    rows = trip[:, 0].astype(int)
    ix, iy, iz = rows % 3, (rows // 3) % 4, rows // 12
    assert np.all((ix == 0) | (ix == 2) | (iy == 0) | (iy == 3) | (iz == 0) | (iz == 4))
    assert np.all(trip[:, 2] == -1.0) and np.all(np.diff(rows) >= 0)
    assert set(trip[:, 1].astype(int)) == set(range(ng))


# ---------------------------------------------------------------- oracle reproduces (CPU)
def test_oracle_reproduces_the_fixtures(orc):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    D = mg.stencil4_dia()
    n, nd, npad, doff, av = load_dia()
    assert np.array_equal(D.doff, doff) and np.array_equal(D.av.reshape(nd, npad), av)
    st, k, rel, hist = mg.cg_stencil8()
    assert (st, k, rel) == load_cg()[:3] and np.array_equal(hist, load_cg()[3])
    n2, ng, (L, R) = mg.rank_split()
    _, _, nl, nr, trip = load_split()
    assert (L.nnz, R.nnz) == (nl, nr)
    assert np.array_equal(np.stack([R.ai, R.aj, R.av], 1), trip)


# ---------------------------------------------------------------- GPU path
@pytest.fixture(scope="module")
def mspv():
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2304_09511_gb300 as m
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return m


@pytest.mark.gpu
def test_gpu_dia_of_stencil4_is_the_fixture(mspv):
    r, c, v = synth.stencil27(4)
    D = mspv.Matrix.from_coo(64, 64, r, c, v).convert("dia")
    e = D.export()
    n, nd, npad, doff, av = load_dia()
    assert np.array_equal(e["doff"], doff) and e["npad"] == npad
    assert np.array_equal(np.asarray(e["vals"]).reshape(nd, npad), av)


@pytest.mark.gpu
def test_gpu_cg_on_stencil8_matches_the_fixture(mspv):
    import torch
    st, k, rel, hist = load_cg()
    r, c, v = synth.stencil27(8)
    for fmt in ("coo", "csr", "dia"):
        A = mspv.Matrix.from_coo(512, 512, r, c, v)
        M = A if fmt == "coo" else A.convert(fmt)
        b = M.spmv(torch.ones(512, dtype=torch.float64, device="cuda"))
        res = M.cg(b, tol=1e-10, maxit=200)
        assert res.converged and abs(res.iters - k) <= 1 and res.relres <= 1e-10


@pytest.mark.gpu
def test_gpu_rank_split_is_the_fixture(mspv):
    r, c, v, n, ng = synth.hpcg_rank_matrix(3, 4, 5)
    A = mspv.Matrix.from_coo(n, n + ng, r, c, v)
    L, R = A.split_columns(n)
    _, _, nl, nr, trip = load_split()
    e = R.export()
    assert L.info["nnz"] == nl and R.info["nnz"] == nr
    assert np.array_equal(np.stack([e["rows"], e["cols"], e["vals"]], 1), trip)
