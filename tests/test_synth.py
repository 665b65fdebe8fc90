"""The seeded input generators: the torch stencil equals the numpy one, and the selector
families have the shapes their recipe states."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("g", [2, 3, 7, 12])
def test_torch_stencil_equals_numpy_stencil(g):
    r, c, v = synth.stencil27(g)
    rt, ct, vt = synth.stencil27_torch(g, "cpu", planes_per_chunk=5)
    assert np.array_equal(r, rt.numpy()) and np.array_equal(c, ct.numpy())
    assert np.array_equal(v, vt.numpy())


@pytest.mark.parametrize("g,seed", [(2, 1), (5, 3), (12, 7)])
def test_torch_perturbed_stencil_equals_numpy(g, seed):
    """The perturbed stencil built by torch (int64 hash arithmetic) is bit for bit the numpy
    one: same hash of each unordered pair, same left-to-right diagonal sum."""
    r, c, v = synth.stencil27_perturbed(g, seed)
    rt, ct, vt = synth.stencil27_torch(g, "cpu", planes_per_chunk=3, perturb_seed=seed)
    assert np.array_equal(r, rt.numpy()) and np.array_equal(c, ct.numpy())
    assert np.array_equal(v.view(np.uint64), vt.numpy().view(np.uint64))
    # symmetric, strictly diagonally dominant
    n = g ** 3
    D = np.zeros((n, n))
    D[r, c] = v
    assert np.array_equal(D, D.T)
    assert np.all(np.diag(D) > np.abs(D - np.diag(np.diag(D))).sum(axis=1))


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("backend", ["numpy", "torch"])
def test_family_recipe(seed, backend):
    if backend == "numpy":
        fam, n, r, c, v = synth.family_matrix(seed, n_min=1_000, n_max=20_000)
    else:
        fam, n, r, c, v = synth.family_matrix_torch(seed, "cpu", n_min=1_000, n_max=20_000)
        r, c, v = r.numpy(), c.numpy(), v.numpy()
    spec = synth.family_spec(seed, n_min=1_000, n_max=20_000)
    assert fam == synth.FAMILIES[seed % 4] == spec["family"] and n == spec["n"]
    assert 1_000 <= n <= 20_000 or fam == "blockdiag"
    assert r.dtype == np.int32 and c.dtype == np.int32 and v.dtype == np.float64
    assert np.all(np.diff(r) >= 0) and r.min() >= 0 and r.max() < n and c.min() >= 0 and c.max() < n
    lens = np.bincount(r, minlength=n)
    off = v[r != c]
    assert np.all(np.abs(off) <= 1.0)
    # diagonal entries dominate their rows (SPD-friendly values)
    d = r == c
    absrow = np.bincount(r, weights=np.abs(np.where(d, 0.0, v)), minlength=n)
    assert np.all(v[d] > absrow[r[d]])
    if fam == "banded":
        offs = np.unique(c.astype(np.int64) - r)
        assert 5 <= offs.size <= 27 and 0 in offs
        assert np.array_equal(offs, spec["offsets"])
    elif fam == "uniform":
        assert lens.min() >= 8 and lens.max() <= 64
    elif fam == "powerlaw":
        assert lens.min() >= 1 and lens.max() <= 20_000
        assert 10 <= lens.mean() <= 20
    else:
        assert np.all(lens == 32) and np.all(c // 32 == r // 32)


@pytest.mark.parametrize("g,seed", [(5, 1), (8, 3)])
def test_perturbed_stencil_recipe(g, seed):
    """The perturbed SPD stencil as stated: the 27-point pattern, off-diagonals -(1 + 0.1 u)
    with u in [0, 1) and the same value for (i, j) and (j, i), the diagonal the left-to-right
    sum of |off| plus 1 (so every row sums to exactly 1 up to that sum's rounding), values that
    FP32 does round, and a symmetric positive definite matrix (Gershgorin)."""
    n = g ** 3
    r0, c0, _ = synth.stencil27(g)
    r, c, v = synth.stencil27_perturbed(g, seed)
    assert np.array_equal(r, r0) and np.array_equal(c, c0)
    D = np.zeros((n, n))
    D[r, c] = v
    off = r != c
    assert np.all((v[off] <= -1.0) & (v[off] > -1.1))
    assert np.array_equal(D, D.T)
    for i in range(n):
        row = np.nonzero(r == i)[0]
        s = 0.0
        for e in row:   # left to right in column order, off-diagonals only
            if c[e] != i:
                s += abs(v[e])
        assert D[i, i] == s + 1.0
    assert np.allclose(D.sum(axis=1), 1.0, rtol=0, atol=1e-12)
    assert np.any(v.astype(np.float32).astype(np.float64) != v)
    assert np.linalg.eigvalsh(D).min() >= 1.0 - 1e-9
