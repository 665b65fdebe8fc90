"""GPU parity of format selection through the C ABI against oracle/selector.py: the
feature kernels, the run-first tuner's contract, and the MLP's training and inference
kernels."""
import numpy as np
import pytest

import synth
from oracle import selector as sel

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


def _matrices():
    out = []
    for seed in range(8):   # two of each family, small sizes
        fam, n, r, c, v = synth.family_matrix(seed, n_min=2_000, n_max=30_000)
        out.append((f"{fam}{seed}", n, n, r, c))
    r, c, _ = synth.stencil27(12)
    out.append(("stencil12", 12 ** 3, 12 ** 3, r, c))
    rng = np.random.default_rng(4)
    r = np.sort(rng.integers(0, 300, 2000)).astype(np.int32)
    out.append(("rect300x700", 300, 700, r, rng.integers(0, 700, 2000).astype(np.int32)))
    r = rng.integers(0, 500, 3000).astype(np.int32) * 2          # odd rows empty, duplicates
    out.append(("emptyrows", 1000, 1000, r, rng.integers(0, 1000, 3000).astype(np.int32)))
    out.append(("noentries", 50, 50, np.zeros(0, np.int32), np.zeros(0, np.int32)))
    return out


MATRICES = _matrices()


@pytest.mark.parametrize("case", MATRICES, ids=[m[0] for m in MATRICES])
def test_features_match_oracle_in_every_format(mspv, case):
    name, nr, nc, r, c = case
    v = np.ones(len(r))
    A = mspv.Matrix.from_coo(nr, nc, dev(r), dev(c), dev(v)) if len(r) else \
        mspv.Matrix.from_coo(nr, nc, r, c, v)
    want = sel.features(nr, nc, r, c).astype(np.float32)
    got = A.features()
    np.testing.assert_allclose(got, want, rtol=2e-7, atol=1e-7)
    np.testing.assert_array_equal(A.convert("csr").features(), got)
    if nr == nc and len(r):
        try:
            D = A.convert("dia")
        except mspv.MspvError as e:
            assert "ETOOBIG" in str(e)
        else:
            np.testing.assert_array_equal(D.features(), got)


def test_tuner_contract(mspv):
    # uniform random columns: DIA is over its fill cap -> +inf, never chosen
    fam, n, r, c, v = synth.family_matrix(1, n_min=20_000, n_max=20_001)
    assert fam == "uniform"
    A = mspv.Matrix.from_coo(n, n, dev(r), dev(c), dev(v))
    best, ms = A.tune_format(reps=5)
    assert np.isinf(ms["dia"]) and ms["coo"] > 0 and ms["csr"] > 0
    assert np.isfinite(ms["coo"]) and np.isfinite(ms["csr"])
    assert best in ("coo", "csr")
    # the tie rule: start at CSR, then DIA, then COO; replace only when more than 1% faster
    pick = "csr"
    for f in ("dia", "coo"):
        if ms[f] < ms[pick] * 0.99:
            pick = f
    assert best == pick
    # a stencil builds in all three formats
    r, c, v = synth.stencil27(24)
    S = mspv.Matrix.from_coo(24 ** 3, 24 ** 3, dev(r), dev(c), dev(v)).convert("csr")
    best, ms = S.tune_format(reps=5)
    assert all(np.isfinite(t) and t > 0 for t in ms.values())
    assert S.select_format() in ("coo", "csr", "dia")
    with pytest.raises(mspv.MspvError, match="EFORMAT"):
        S.convert("dia").tune_format()


def _gpu_params_b3(mspv, b3):
    p = np.zeros(sel.NPARAM)
    sel.unpack(p)["sd"][:] = 1.0
    sel.unpack(p)["b3"][:] = b3
    return p.astype(np.float32)


def test_select_format_with_params_and_dia_fallback(mspv):
    rng = np.random.default_rng(0)
    r = np.sort(rng.integers(0, 300, 2000)).astype(np.int32)
    R = mspv.Matrix.from_coo(300, 700, dev(r), dev(rng.integers(0, 700, 2000).astype(np.int32)),
                             dev(np.ones(2000)))
    assert R.select_format(_gpu_params_b3(mspv, [10.0, 0.0, 0.0])) == "coo"
    assert R.select_format(_gpu_params_b3(mspv, [0.0, 0.0, 10.0])) == "csr"   # not square
    fam, n, r, c, v = synth.family_matrix(1, n_min=20_000, n_max=20_001)
    U = mspv.Matrix.from_coo(n, n, dev(r), dev(c), dev(v))
    assert U.select_format(_gpu_params_b3(mspv, [0.0, 0.0, 10.0])) == "csr"   # over the DIA cap
    r, c, v = synth.stencil27(10)
    S = mspv.Matrix.from_coo(1000, 1000, dev(r), dev(c), dev(v))
    assert S.select_format(_gpu_params_b3(mspv, [0.0, 0.0, 10.0])) == "dia"


def _separable(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, sel.NF)) * rng.uniform(0.1, 10.0, sel.NF) + rng.normal(size=sel.NF) * 5
    Wt = rng.normal(size=(3, sel.NF))
    y = np.argmax(((X - X.mean(0)) / X.std(0)) @ Wt.T, axis=1)
    return X.astype(np.float32), y.astype(np.int32)


def test_initial_parameters_match_oracle(mspv):
    """epochs = 0 returns the standardisation and the SplitMix64 Glorot initialisation."""
    X, y = _separable(100, 4)
    p = mspv.selector_train(X, y, epochs=0, lr=1e-3, seed=17).astype(np.float64)
    want = sel.init_params(17)
    k = slice(sel.FIRST_TRAINED, sel.NPARAM)
    np.testing.assert_allclose(p[k], want[k], rtol=1e-6, atol=1e-7)
    d = sel.unpack(p)
    np.testing.assert_allclose(d["mu"], X.astype(np.float64).mean(0), rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(d["sd"], X.astype(np.float64).std(0), rtol=1e-6)
    assert np.array_equal(d["lo"], X.min(0).astype(np.float64))
    assert np.array_equal(d["hi"], X.max(0).astype(np.float64))
    assert np.all(d["b1"] == 0) and np.all(d["b2"] == 0) and np.all(d["b3"] == 0)


def test_one_adam_step_matches_oracle(mspv):
    """After one minibatch step every parameter moves by lr * g / (|g| + eps) on both sides.
    Where |g| is within FP32 rounding of zero its sign is not unique: there only the step's
    bound (|change| <= lr) is checked."""
    X, y = _separable(64, 1)
    lr = 1e-2
    p = mspv.selector_train(X, y, epochs=1, lr=lr, seed=3)
    want = sel.train(X.astype(np.float64), y, epochs=1, lr=lr, seed=3)
    dp, dw = sel.unpack(p.astype(np.float64)), sel.unpack(want)
    np.testing.assert_allclose(dp["mu"], dw["mu"], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(dp["sd"], dw["sd"], rtol=1e-6)
    # gradient at the start, for the sign-ambiguity test
    p0 = sel.init_params(3)
    sel.unpack(p0)["mu"][:] = dw["mu"]
    sel.unpack(p0)["sd"][:] = dw["sd"]
    g = sel.gradient(p0, sel.standardise(p0, X.astype(np.float64)), y)
    init = sel.init_params(3)
    k = slice(sel.FIRST_TRAINED, sel.NPARAM)
    diff = np.abs(p[k].astype(np.float64) - want[k])
    tight = diff <= 1e-6 + 1e-5 * np.abs(want[k])
    ambiguous = np.abs(g[k]) <= 1e-3 * np.max(np.abs(g[k]))
    assert np.all(tight | ambiguous)
    assert np.mean(tight) >= 0.99
    assert np.all(np.abs(p[k] - init[k]) <= lr * 1.0001 + 1e-7)


def test_training_tracks_oracle_and_is_deterministic(mspv):
    X, y = _separable(512, 2)
    p1 = mspv.selector_train(X, y, epochs=15, lr=1e-2, seed=5)
    p2 = mspv.selector_train(X, y, epochs=15, lr=1e-2, seed=5)
    assert np.array_equal(p1, p2)
    want = sel.train(X.astype(np.float64), y, epochs=15, lr=1e-2, seed=5)
    pg = mspv.selector_predict(p1, X)
    po = sel.predict(want, X)
    assert np.mean(pg == y) >= 0.95 and np.mean(po == y) >= 0.95
    assert np.mean(pg == po) >= 0.93
    lg = sel.loss(p1.astype(np.float64), sel.standardise(p1.astype(np.float64), X), y)
    lo = sel.loss(want, sel.standardise(want, X), y)
    assert lg == pytest.approx(lo, rel=0.25, abs=0.05)


def test_predict_matches_oracle_where_the_margin_is_unique(mspv):
    X, y = _separable(256, 3)
    p = mspv.selector_train(X, y, epochs=5, lr=1e-2, seed=9)
    rng = np.random.default_rng(8)
    Xq = (rng.normal(size=(3000, sel.NF)) * X.std(0) + X.mean(0)).astype(np.float32)
    got = mspv.selector_predict(p, Xq)
    Z = sel.logits(p.astype(np.float64), Xq.astype(np.float64))
    top2 = np.sort(Z, axis=1)[:, -2:]
    clear = (top2[:, 1] - top2[:, 0]) > 1e-4 * (1.0 + np.abs(top2[:, 1]))
    assert np.mean(clear) > 0.99
    np.testing.assert_array_equal(got[clear], np.argmax(Z, axis=1)[clear])
    assert np.all((got >= 0) & (got <= 2))
    assert len(mspv.selector_predict(p, np.zeros((0, sel.NF), np.float32))) == 0
    # features beyond the training range predict as their clamped values
    d = sel.unpack(p.astype(np.float64))
    far = Xq * 50.0
    clamped = np.clip(far, d["lo"], d["hi"]).astype(np.float32)
    np.testing.assert_array_equal(mspv.selector_predict(p, far), mspv.selector_predict(p, clamped))
