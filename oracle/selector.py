"""Oracle for format selection: sparsity features, and the FP32 MLP selector written out
as plain FP64 numpy.

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline and
reference arm may import this module; the library never does.

What it follows:
  * The run-first auto-tuner of the paper's distributed HPCG (Sec. VI): time every format,
    keep the fastest. Its labels train the selector; the tuner itself is timing, so it has
    no oracle beyond `regret` below.
  * The learned selector is not specified by the paper (Sec. VII only cites learned
    auto-tuners). Its definition is textbook: a 10 -> 64 -> 64 -> 3 ReLU network with a
    softmax cross-entropy loss (Goodfellow, Bengio, Courville, "Deep Learning", Sec. 6.2 and
    6.5), weights initialised uniformly in +-sqrt(6 / (fan_in + fan_out)) (Glorot & Bengio,
    AISTATS 2010), trained by Adam (Kingma & Ba, ICLR 2015, Algorithm 1). The initial
    weights are drawn from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), the one
    counter-based generator both sides implement from its published definition.

Pins (tests/test_selector_oracle.py): the published SplitMix64 test vector; features against
dense brute force and the stencil's closed forms; the forward pass against scalar loops and
the ln 3 loss of a zero network; gradients against central finite differences; the Adam step
against its closed form under a constant gradient; training on a separable problem.
"""
from __future__ import annotations

import numpy as np

NF, NH, NC = 10, 64, 3
BATCH = 64
# parameter layout: mu[10] sd[10] lo[10] hi[10] W1[64][10] b1[64] W2[64][64] b2[64] W3[3][64] b3[3]
_SHAPES = [("mu", (NF,)), ("sd", (NF,)), ("lo", (NF,)), ("hi", (NF,)), ("W1", (NH, NF)), ("b1", (NH,)),
           ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NC, NH)), ("b3", (NC,))]
NPARAM = sum(int(np.prod(s)) for _, s in _SHAPES)
FIRST_TRAINED = 4 * NF   # mu, sd, lo, hi come from the training data, the rest from Adam
TRAINED = ("W1", "b1", "W2", "b2", "W3", "b3")
FORMATS = ("coo", "csr", "dia")

_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def splitmix64(seed: int, count: int) -> list[int]:
    """The first `count` outputs of SplitMix64 seeded with `seed` (Steele et al. 2014):
    the state advances by the golden gamma, then is mixed by two xor-shift-multiply rounds
    and a final xor-shift."""
    out = []
    state = seed & _M64
    for _ in range(count):
        state = (state + _GAMMA) & _M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        out.append(z ^ (z >> 31))
    return out


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------
def unpack(p: np.ndarray) -> dict:
    """Views of the flat parameter vector by name."""
    p = np.asarray(p)
    assert p.shape == (NPARAM,)
    out, k = {}, 0
    for name, shape in _SHAPES:
        m = int(np.prod(shape))
        out[name] = p[k:k + m].reshape(shape)
        k += m
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in _SHAPES])


def init_params(seed: int) -> np.ndarray:
    """mu = 0, sd = 1, lo = -inf, hi = +inf; trained parameter k (in layout order, counted from W1) is, for a
    weight, (2u - 1) * sqrt(6 / (fan_in + fan_out)) with u = (top 24 bits of SplitMix64
    output k) / 2^24; biases are 0."""
    d = {name: np.zeros(shape) for name, shape in _SHAPES}
    d["sd"][:] = 1.0
    d["lo"][:] = -np.inf
    d["hi"][:] = np.inf
    ntrain = NPARAM - FIRST_TRAINED
    u = np.array([(z >> 40) / float(1 << 24) for z in splitmix64(seed, ntrain)])
    k = 0
    for name in TRAINED:
        shape = d[name].shape
        m = int(np.prod(shape))
        if name.startswith("W"):
            fan_out, fan_in = shape
            lim = np.sqrt(6.0 / (fan_in + fan_out))
            d[name][...] = ((2.0 * u[k:k + m] - 1.0) * lim).reshape(shape)
        k += m
    return pack(d)


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------
def standardise(p: np.ndarray, X) -> np.ndarray:
    """Clamp each feature to the training range [lo, hi], then standardise."""
    d = unpack(p)
    return (np.clip(np.asarray(X, dtype=np.float64), d["lo"], d["hi"]) - d["mu"]) / d["sd"]


def forward(p: np.ndarray, Xs: np.ndarray):
    """Logits of standardised inputs Xs (B x 10), with the hidden activations."""
    d = unpack(p)
    H1 = np.maximum(Xs @ d["W1"].T + d["b1"], 0.0)
    H2 = np.maximum(H1 @ d["W2"].T + d["b2"], 0.0)
    Z = H2 @ d["W3"].T + d["b3"]
    return Z, H1, H2


def softmax(Z: np.ndarray) -> np.ndarray:
    E = np.exp(Z - Z.max(axis=1, keepdims=True))
    return E / E.sum(axis=1, keepdims=True)


def loss(p: np.ndarray, Xs: np.ndarray, y: np.ndarray) -> float:
    """Mean cross-entropy of the softmax of the logits against labels y."""
    Z, _, _ = forward(p, Xs)
    P = softmax(Z)
    return float(-np.mean(np.log(P[np.arange(len(y)), y])))


def gradient(p: np.ndarray, Xs: np.ndarray, y: np.ndarray) -> np.ndarray:
    """d loss / d p by back-propagation (zero for mu, sd, lo and hi, which are not trained)."""
    d = unpack(p)
    Z, H1, H2 = forward(p, Xs)
    B = len(y)
    dZ = softmax(Z)
    dZ[np.arange(B), y] -= 1.0
    dZ /= B
    g = {name: np.zeros(shape) for name, shape in _SHAPES}
    g["W3"] = dZ.T @ H2
    g["b3"] = dZ.sum(axis=0)
    dH2 = (dZ @ d["W3"]) * (H2 > 0)
    g["W2"] = dH2.T @ H1
    g["b2"] = dH2.sum(axis=0)
    dH1 = (dH2 @ d["W2"]) * (H1 > 0)
    g["W1"] = dH1.T @ Xs
    g["b1"] = dH1.sum(axis=0)
    return pack(g)


def adam_step(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Step t (1-based) of Adam: returns the new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def train(X, y, epochs: int, lr: float, seed: int) -> np.ndarray:
    """Standardise by the training set's mean and population standard deviation (1 where it
    is below 1e-6), keep its per-feature minimum and maximum (the clamping range used at
    prediction), initialise from `seed`, then for each epoch take Adam steps over minibatches
    of 64 consecutive samples in index order."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.int64)
    p = init_params(seed)
    d = unpack(p)
    d["mu"][:] = X.mean(axis=0)
    sd = X.std(axis=0)
    d["sd"][:] = np.where(sd > 1e-6, sd, 1.0)
    d["lo"][:] = X.min(axis=0)
    d["hi"][:] = X.max(axis=0)
    Xs = standardise(p, X)
    trained = np.zeros(NPARAM, dtype=bool)
    trained[FIRST_TRAINED:] = True
    m = np.zeros(NPARAM)
    v = np.zeros(NPARAM)
    t = 0
    for _ in range(epochs):
        for i0 in range(0, len(y), BATCH):
            t += 1
            g = gradient(p, Xs[i0:i0 + BATCH], y[i0:i0 + BATCH])
            new, m, v = adam_step(p, g, m, v, t, lr)
            p = np.where(trained, new, p)
    return p


def logits(p, X) -> np.ndarray:
    return forward(np.asarray(p, dtype=np.float64), standardise(p, X))[0]


def predict(p, X) -> np.ndarray:
    """Arg max of the logits (lowest class on ties)."""
    return np.argmax(logits(p, X), axis=1)


# ---------------------------------------------------------------------------
# features and regret
# ---------------------------------------------------------------------------
def features(nrows: int, ncols: int, rows, cols) -> np.ndarray:
    """The ten features of the set of stored positions {(rows[e], cols[e])} (duplicates
    count once), in FP64:
    log2 max(n,1), log2 max(nnz,1), mean, population std, max and min of the row lengths,
    log2 max(ndiags,1), nnz / (ndiags n), empty rows / n, max |col - row| / n, where n = nrows
    and ndiags = number of distinct col - row. Row-based entries are 0 when n = 0."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    pos = np.unique(rows * max(ncols, 1) + cols) if rows.size else np.zeros(0, np.int64)
    r = pos // max(ncols, 1)
    c = pos % max(ncols, 1)
    nnz = pos.size
    n = nrows
    f = np.zeros(NF)
    f[0] = np.log2(max(n, 1))
    f[1] = np.log2(max(nnz, 1))
    if n > 0:
        lens = np.bincount(r, minlength=n)
        f[2] = nnz / n
        f[3] = lens.std()
        f[4] = lens.max()
        f[5] = lens.min()
        offs = np.unique(c - r)
        nd = offs.size
        f[6] = np.log2(max(nd, 1))
        f[7] = nnz / (nd * n) if nd > 0 else 0.0
        f[8] = np.count_nonzero(lens == 0) / n
        f[9] = (np.abs(c - r).max() / n) if nnz > 0 else 0.0
    return f


def regret(ms: np.ndarray, picks: np.ndarray) -> dict:
    """ms: (N, 3) per-format times (inf where a format was not built); picks: chosen format
    per matrix. Aggregate regret = sum of chosen times / sum of best times - 1; also the
    geometric mean, mean and maximum per-matrix slowdown, the share within 10% of the best
    and the fraction of picks as fast as the best."""
    ms = np.asarray(ms, dtype=np.float64)
    picks = np.asarray(picks)
    best = ms.min(axis=1)
    chosen = ms[np.arange(len(picks)), picks]
    slow = chosen / best
    return {"regret": float(chosen.sum() / best.sum() - 1.0),
            "geomean_slowdown": float(np.exp(np.mean(np.log(slow)))),
            "mean_slowdown": float(np.mean(slow)),
            "max_slowdown": float(np.max(slow)),
            "within_10pct": float(np.mean(slow <= 1.10)),
            "exact": float(np.mean(chosen == best))}
