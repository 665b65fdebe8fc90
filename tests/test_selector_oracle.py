"""Pins of the selector oracle (oracle/selector.py) against things outside itself:
a published generator test vector, dense brute force, closed forms of the 27-point
stencil, scalar-loop forward passes, finite differences and Adam's closed form."""
import math

import numpy as np
import pytest

import synth
from oracle import selector as sel


def test_splitmix64_published_vector():
    # SplitMix64 seeded with 1234567: the first five outputs of the reference
    # implementation (Steele, Lea & Flood 2014; Vigna's splitmix64.c)
    assert sel.splitmix64(1234567, 5) == [6457827717110365317, 3203168211198807973,
                                          9817491932198370423, 4593380528125082431,
                                          16408922859458223821]


def test_glorot_init_bounds_and_spread():
    p = sel.unpack(sel.init_params(7))
    assert np.all(p["mu"] == 0) and np.all(p["sd"] == 1)
    for name, (fo, fi) in (("W1", (64, 10)), ("W2", (64, 64)), ("W3", (3, 64))):
        lim = math.sqrt(6.0 / (fi + fo))
        w = p[name]
        assert np.all(np.abs(w) <= lim)
        # uniform on [-lim, lim]: variance lim^2 / 3, mean 0 (loose statistical bounds)
        assert abs(w.mean()) < 0.2 * lim
        assert abs(w.var() / (lim * lim / 3.0) - 1.0) < 0.35
    for name in ("b1", "b2", "b3"):
        assert np.all(p[name] == 0)
    assert not np.array_equal(sel.init_params(7), sel.init_params(8))


def _dense_features(A: np.ndarray) -> np.ndarray:
    """Brute force over a dense pattern with scalar loops."""
    n, m = A.shape
    lens = [sum(1 for j in range(m) if A[i, j]) for i in range(n)]
    nnz = sum(lens)
    diags = set()
    band = 0
    for i in range(n):
        for j in range(m):
            if A[i, j]:
                diags.add(j - i)
                band = max(band, abs(j - i))
    mean = nnz / n
    var = sum((L - mean) ** 2 for L in lens) / n
    nd = len(diags)
    return np.array([math.log2(max(n, 1)), math.log2(max(nnz, 1)), mean, math.sqrt(var), max(lens),
                     min(lens), math.log2(max(nd, 1)), nnz / (nd * n) if nd else 0.0,
                     sum(1 for L in lens if L == 0) / n, band / n])


@pytest.mark.parametrize("seed", range(6))
def test_features_match_dense_brute_force(seed):
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(1, 40)), int(rng.integers(1, 40))
    A = rng.random((n, m)) < rng.uniform(0.02, 0.4)
    if seed == 0:
        A[:] = False            # no entries at all
    if seed == 1:
        A[::3] = False          # empty rows
    r, c = np.nonzero(A)
    # duplicates and shuffled order must not matter
    r2 = np.concatenate([r, r[: len(r) // 3]])
    c2 = np.concatenate([c, c[: len(c) // 3]])
    perm = rng.permutation(len(r2))
    got = sel.features(n, m, r2[perm], c2[perm])
    np.testing.assert_allclose(got, _dense_features(A), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("g", [3, 5, 8])
def test_features_stencil_closed_form(g):
    r, c, _ = synth.stencil27(g)
    n = g ** 3
    nnz = (3 * g - 2) ** 3
    f = sel.features(n, n, r, c)
    assert f[0] == pytest.approx(3 * math.log2(g))
    assert f[1] == pytest.approx(math.log2(nnz))
    assert f[2] == pytest.approx(nnz / n)
    assert f[4] == 27 and f[5] == 8          # interior rows, corner rows
    assert f[6] == pytest.approx(math.log2(27))
    assert f[7] == pytest.approx(nnz / (27 * n))
    assert f[8] == 0.0
    assert f[9] == pytest.approx((g * g + g + 1) / n)
    # row lengths are products of per-axis counts (2 at a face, 3 inside): std in closed form
    per_axis = np.array([2.0] * 2 + [3.0] * (g - 2))
    lens = np.einsum("i,j,k->ijk", per_axis, per_axis, per_axis).ravel()
    assert f[3] == pytest.approx(lens.std(), rel=1e-12)


def _scalar_forward(p, x):
    d = sel.unpack(p)
    xs = [(x[f] - d["mu"][f]) / d["sd"][f] for f in range(sel.NF)]
    h1 = []
    for j in range(sel.NH):
        a = d["b1"][j]
        for f in range(sel.NF):
            a += d["W1"][j, f] * xs[f]
        h1.append(max(a, 0.0))
    h2 = []
    for k in range(sel.NH):
        a = d["b2"][k]
        for j in range(sel.NH):
            a += d["W2"][k, j] * h1[j]
        h2.append(max(a, 0.0))
    out = []
    for cl in range(sel.NC):
        a = d["b3"][cl]
        for k in range(sel.NH):
            a += d["W3"][cl, k] * h2[k]
        out.append(a)
    return np.array(out)


def test_forward_matches_scalar_loops():
    rng = np.random.default_rng(3)
    p = sel.init_params(11)
    d = sel.unpack(p)
    d["mu"][:] = rng.normal(size=sel.NF)
    d["sd"][:] = rng.uniform(0.5, 2.0, sel.NF)
    d["b1"][:] = rng.normal(scale=0.1, size=sel.NH)
    d["b2"][:] = rng.normal(scale=0.1, size=sel.NH)
    d["b3"][:] = rng.normal(scale=0.1, size=sel.NC)
    X = rng.normal(size=(5, sel.NF))
    Z = sel.logits(p, X)
    for i in range(5):
        np.testing.assert_allclose(Z[i], _scalar_forward(p, X[i]), rtol=1e-12, atol=1e-12)


def test_zero_network_loss_is_ln3_and_ties_pick_class0():
    p = np.zeros(sel.NPARAM)
    sel.unpack(p)["sd"][:] = 1.0
    X = np.random.default_rng(0).normal(size=(9, sel.NF))
    y = np.array([0, 1, 2] * 3)
    assert sel.loss(p, X, y) == pytest.approx(math.log(3.0), rel=1e-15)
    assert np.all(sel.predict(p, X) == 0)
    # b3 alone decides the class
    sel.unpack(p)["b3"][:] = [0.0, 0.5, -1.0]
    assert np.all(sel.predict(p, X) == 1)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(5)
    p = sel.init_params(2)
    d = sel.unpack(p)
    d["b1"][:] = rng.uniform(0.05, 0.2, sel.NH)     # keep units active, away from kinks
    d["b2"][:] = rng.uniform(0.05, 0.2, sel.NH)
    d["b3"][:] = rng.normal(size=sel.NC)
    X = rng.normal(size=(7, sel.NF))
    y = rng.integers(0, 3, 7)
    g = sel.gradient(p, X, y)
    assert np.all(g[: sel.FIRST_TRAINED] == 0)
    idx = np.concatenate([rng.choice(np.arange(sel.FIRST_TRAINED, sel.NPARAM), 150, replace=False),
                          [sel.NPARAM - 1, sel.NPARAM - 4, sel.FIRST_TRAINED]])
    h = 1e-6
    for k in idx:
        e = np.zeros(sel.NPARAM)
        e[k] = h
        fd = (sel.loss(p + e, X, y) - sel.loss(p - e, X, y)) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-8), k


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g the bias-corrected moments are exactly g and g^2, so every
    step moves theta by lr * g / (|g| + eps)."""
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    theta = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    lr = 0.01
    for t in range(1, 51):
        theta, m, v = sel.adam_step(theta, g, m, v, t, lr)
    np.testing.assert_allclose(theta, -50 * lr * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=1e-15)


def test_training_separates_a_separable_problem():
    """Labels are the arg max of three linear scores of the features: a 64-unit ReLU
    network fits them; the loss falls and training accuracy reaches 97%."""
    rng = np.random.default_rng(9)
    X = rng.normal(size=(640, sel.NF)) * rng.uniform(0.1, 10.0, sel.NF) + rng.normal(size=sel.NF) * 5
    Wt = rng.normal(size=(3, sel.NF))
    y = np.argmax(((X - X.mean(0)) / X.std(0)) @ Wt.T, axis=1)
    p0 = sel.train(X, y, epochs=0, lr=1e-2, seed=1)
    p = sel.train(X, y, epochs=40, lr=1e-2, seed=1)
    Xs = sel.standardise(p, X)
    assert sel.loss(p, Xs, y) < 0.5 * sel.loss(p0, sel.standardise(p0, X), y)
    assert np.mean(sel.predict(p, X) == y) >= 0.97
    np.testing.assert_allclose(sel.unpack(p)["mu"], X.mean(0))


def test_features_are_clamped_to_the_training_range():
    """Prediction clamps each feature to [lo, hi] of the training set before standardising;
    inside the range nothing changes."""
    rng = np.random.default_rng(12)
    X = rng.normal(size=(200, sel.NF)) * 3
    y = rng.integers(0, 3, 200)
    p = sel.train(X, y, epochs=2, lr=1e-2, seed=4)
    d = sel.unpack(p)
    assert np.array_equal(d["lo"], X.min(0)) and np.array_equal(d["hi"], X.max(0))
    np.testing.assert_array_equal(sel.standardise(p, X), (X - d["mu"]) / d["sd"])
    far = X * 40.0 + 100.0
    np.testing.assert_array_equal(sel.logits(p, far), sel.logits(p, np.clip(far, d["lo"], d["hi"])))
    assert np.all(np.abs(sel.standardise(p, far)) <= np.abs((np.stack([d["lo"], d["hi"]]) - d["mu"]) / d["sd"]).max(0))


def test_regret_definition():
    ms = np.array([[1.0, 2.0, np.inf], [3.0, 1.0, 0.5], [2.0, 2.0, 4.0]])
    r = sel.regret(ms, np.array([0, 1, 1]))
    assert r["regret"] == pytest.approx((1.0 + 1.0 + 2.0) / (1.0 + 0.5 + 2.0) - 1.0)
    assert r["max_slowdown"] == pytest.approx(2.0)
    assert r["exact"] == pytest.approx(2 / 3)
    assert r["geomean_slowdown"] == pytest.approx(2.0 ** (1 / 3))
    assert r["within_10pct"] == pytest.approx(2 / 3)
