"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and
the benchmark. This module only produces inputs (triplets and vectors); it holds
none of the SpMV / CG arithmetic.

* ``stencil27(g)``: the HPCG problem matrix, a 27-point finite-difference stencil on a
  g x g x g grid (Sec. VI, HPCG experiments): row i = ix + g*iy + g^2*iz couples to
  every neighbour (dx, dy, dz) in {-1, 0, 1}^3 inside the grid, diagonal 26.0,
  off-diagonals -1.0. Triplets are emitted in ascending (row, col) order, and nnz is
  exactly (3g - 2)^3.
* ``stencil27_perturbed(g, seed)``: the same pattern with symmetric off-diagonals
  -(1 + 0.1 u), u in [0, 1) from a counter-based hash of the unordered pair (so the
  matrix is symmetric), and diagonal = sum |off-diagonals| + 1 (strictly diagonally
  dominant, hence SPD). Used where FP32/BF16 rounding of the values must matter.
* ``uniform_x(n, seed)``: x ~ U[0, 1) from numpy's PCG64 stream (``default_rng(seed)``).
* ``random_coo(...)``: small unstructured COO triplets with controllable duplicates,
  empty rows and input order, for edge-case and brute-force tests.
"""
from __future__ import annotations

import numpy as np

_OFFSETS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def stencil_nnz(g: int) -> int:
    return (3 * g - 2) ** 3


def stencil_offsets(g: int) -> np.ndarray:
    """The 27 column offsets dz*g^2 + dy*g + dx, ascending."""
    return np.array(sorted(dz * g * g + dy * g + dx for dz, dy, dx in _OFFSETS), np.int64)


def _splitmix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014) on uint64 counters."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z += np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def _unit(z: np.ndarray) -> np.ndarray:
    """uint64 -> [0, 1) with 53 random bits."""
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def stencil27(g: int, perturb_seed: int | None = None, planes_per_chunk: int = 16):
    """27-point stencil triplets (rows int32, cols int32, vals float64), sorted by (row, col)."""
    n = g * g * g
    nnz = stencil_nnz(g)
    rows = np.empty(nnz, np.int32)
    cols = np.empty(nnz, np.int32)
    vals = np.empty(nnz, np.float64)
    pos = 0
    for z0 in range(0, g, planes_per_chunk):
        z1 = min(g, z0 + planes_per_chunk)
        iz, iy, ix = np.meshgrid(np.arange(z0, z1), np.arange(g), np.arange(g), indexing="ij")
        iz, iy, ix = iz.ravel(), iy.ravel(), ix.ravel()
        r = (ix + g * iy + g * g * iz).astype(np.int64)
        m = r.size
        C = np.empty((m, 27), np.int64)
        valid = np.empty((m, 27), bool)
        for k, (dz, dy, dx) in enumerate(_OFFSETS):  # lexicographic (dz,dy,dx) = ascending col
            jx, jy, jz = ix + dx, iy + dy, iz + dz
            valid[:, k] = (jx >= 0) & (jx < g) & (jy >= 0) & (jy < g) & (jz >= 0) & (jz < g)
            C[:, k] = r + dz * g * g + dy * g + dx
        R = np.broadcast_to(r[:, None], (m, 27))
        rr, cc = R[valid], C[valid]
        cnt = rr.size
        rows[pos:pos + cnt] = rr
        cols[pos:pos + cnt] = cc
        if perturb_seed is None:
            vals[pos:pos + cnt] = np.where(rr == cc, 26.0, -1.0)
        else:
            lo, hi = np.minimum(rr, cc), np.maximum(rr, cc)
            key = (lo.astype(np.uint64) * np.uint64(n) + hi.astype(np.uint64)) ^ \
                  _splitmix64(np.array([perturb_seed], np.uint64))[0]
            u = _unit(_splitmix64(key))
            off = -(1.0 + 0.1 * u)
            v = np.where(rr == cc, 0.0, off)
            # diagonal = sum |off| + 1, accumulated per row in column order
            Vm = np.zeros((m, 27))
            Vm[valid] = v
            diag = np.abs(Vm).sum(axis=1) + 1.0
            diag_rep = np.broadcast_to(diag[:, None], (m, 27))[valid]
            vals[pos:pos + cnt] = np.where(rr == cc, diag_rep, v)
        pos += cnt
    assert pos == nnz and n < 2**31
    return rows, cols, vals


def stencil27_perturbed(g: int, seed: int = 1):
    return stencil27(g, perturb_seed=seed)


def uniform_x(n: int, seed: int = 0) -> np.ndarray:
    return np.random.default_rng(seed).random(n)


def random_coo(nrows: int, ncols: int, nnz: int, seed: int, dup_frac: float = 0.0,
               empty_rows: int = 0, shuffle: bool = True, value_range=(-1.0, 1.0)):
    """Unstructured triplets. ``dup_frac`` of them repeat an earlier (row, col);
    ``empty_rows`` rows are kept free of entries; order is random when ``shuffle``."""
    rng = np.random.default_rng(seed)
    allowed = np.arange(nrows)
    if empty_rows and nrows > empty_rows:
        allowed = np.sort(rng.choice(nrows, nrows - empty_rows, replace=False))
    ndup = int(nnz * dup_frac) if nnz else 0
    base = nnz - ndup
    r = allowed[rng.integers(0, allowed.size, base)] if allowed.size else np.zeros(0, np.int64)
    c = rng.integers(0, ncols, base) if ncols else np.zeros(0, np.int64)
    if ndup and base:
        pick = rng.integers(0, base, ndup)
        r = np.concatenate([r, r[pick]])
        c = np.concatenate([c, c[pick]])
    v = rng.uniform(value_range[0], value_range[1], r.size)
    if shuffle:
        p = rng.permutation(r.size)
        r, c, v = r[p], c[p], v[p]
    return r.astype(np.int32), c.astype(np.int32), v.astype(np.float64)


def banded(n: int, k: int, seed: int, fill: float = 1.0, spread: int | None = None):
    """Square matrix with k distinct diagonals (offsets drawn from [-spread, spread],
    always including 0), each in-range slot kept with probability ``fill``; values
    U(-1, 1). Triplets in random order."""
    rng = np.random.default_rng(seed)
    spread = max(1, n - 1) if spread is None else min(spread, max(n - 1, 0))
    pool = np.arange(-spread, spread + 1)
    pool = pool[pool != 0]
    k = max(1, min(k, pool.size + 1))
    offs = np.sort(np.concatenate([[0], rng.choice(pool, k - 1, replace=False)])) if n > 1 else np.array([0])
    rows, cols = [], []
    for off in offs.tolist():
        i = np.arange(max(0, -off), min(n, n - off))
        keep = rng.random(i.size) < fill
        rows.append(i[keep])
        cols.append(i[keep] + off)
    r = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    c = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    v = rng.uniform(-1.0, 1.0, r.size)
    p = rng.permutation(r.size)
    return r[p].astype(np.int32), c[p].astype(np.int32), v[p]
