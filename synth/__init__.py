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
            # diagonal = sum |off| + 1, accumulated per row left to right in column order
            Vm = np.zeros((m, 27))
            Vm[valid] = v
            diag = np.zeros(m)
            for k in range(27):
                diag = diag + np.abs(Vm[:, k])
            diag = diag + 1.0
            diag_rep = np.broadcast_to(diag[:, None], (m, 27))[valid]
            vals[pos:pos + cnt] = np.where(rr == cc, diag_rep, v)
        pos += cnt
    assert pos == nnz and n < 2**31
    return rows, cols, vals


def _as_i64(c: int) -> int:
    """The int64 with the bit pattern of the uint64 c."""
    return c - (1 << 64) if c >= (1 << 63) else c


def _splitmix64_torch(z):
    """_splitmix64 on int64 tensors holding uint64 bit patterns (products wrap mod 2^64;
    right shifts are made logical by masking the sign extension)."""
    def lsr(t, k):
        return (t >> k) & ((1 << (64 - k)) - 1)
    z = z + _as_i64(0x9E3779B97F4A7C15)
    z = (z ^ lsr(z, 30)) * _as_i64(0xBF58476D1CE4E5B9)
    z = (z ^ lsr(z, 27)) * _as_i64(0x94D049BB133111EB)
    return z ^ lsr(z, 31)


def stencil27_torch(g: int, device, planes_per_chunk: int = 32, perturb_seed: int | None = None):
    """The 27-point stencil of stencil27 (plain or perturbed), built by torch on `device`:
    the same triplets bit for bit, in the same (row, col) order, for grids whose host
    generation would be slow."""
    import torch
    n = g * g * g
    nnz = stencil_nnz(g)
    kw = {"device": device}
    rows = torch.empty(nnz, dtype=torch.int32, **kw)
    cols = torch.empty(nnz, dtype=torch.int32, **kw)
    vals = torch.empty(nnz, dtype=torch.float64, **kw)
    off = torch.tensor([dz * g * g + dy * g + dx for dz, dy, dx in _OFFSETS], dtype=torch.int64, **kw)
    d = torch.tensor(_OFFSETS, dtype=torch.int64, **kw)          # (27, 3): dz, dy, dx
    pos = 0
    for z0 in range(0, g, planes_per_chunk):
        z1 = min(g, z0 + planes_per_chunk)
        r = torch.arange(z0 * g * g, z1 * g * g, dtype=torch.int64, **kw)
        ix, iy, iz = r % g, (r // g) % g, r // (g * g)
        jz = iz[:, None] + d[None, :, 0]
        jy = iy[:, None] + d[None, :, 1]
        jx = ix[:, None] + d[None, :, 2]
        valid = (jx >= 0) & (jx < g) & (jy >= 0) & (jy < g) & (jz >= 0) & (jz < g)
        C = r[:, None] + off[None, :]
        rr = r[:, None].expand_as(C)[valid]
        cc = C[valid]
        cnt = rr.numel()
        rows[pos:pos + cnt] = rr.to(torch.int32)
        cols[pos:pos + cnt] = cc.to(torch.int32)
        if perturb_seed is None:
            vals[pos:pos + cnt] = torch.where(rr == cc, 26.0, -1.0).to(torch.float64)
        else:
            lo, hi = torch.minimum(rr, cc), torch.maximum(rr, cc)
            salt = _as_i64(int(_splitmix64(np.array([perturb_seed], np.uint64))[0]))
            u = (_splitmix64_torch((lo * n + hi) ^ salt) >> 11) & ((1 << 53) - 1)
            offv = -(1.0 + 0.1 * (u.to(torch.float64) * (1.0 / 9007199254740992.0)))
            v = torch.where(rr == cc, torch.zeros_like(offv), offv)
            Vm = torch.zeros(C.shape, dtype=torch.float64, **kw)
            Vm[valid] = v
            diag = torch.zeros(C.shape[0], dtype=torch.float64, **kw)
            for k in range(27):
                diag = diag + Vm[:, k].abs()
            diag = diag + 1.0
            diag_rep = diag[:, None].expand_as(C)[valid]
            vals[pos:pos + cnt] = torch.where(rr == cc, diag_rep, v)
        pos += cnt
    assert pos == nnz
    return rows, cols, vals


def hpcg_rank_matrix(nx: int, ny: int, nz: int):
    """The matrix one interior process holds in a distributed 27-point HPCG problem (the
    paper's Sec. VI set-up): the process owns an nx x ny x nz block of a 3 x 3 x 3 block
    decomposition (all 26 neighbours present). Rows are its cells, row i = ix + nx*iy +
    nx*ny*iz; a neighbour inside the block is local column j < n = nx*ny*nz, a neighbour in
    another block is a ghost column n + g, ghosts numbered in order of first appearance
    scanning rows in order and, within a row, neighbours in ascending global index (the
    external-column numbering of HPCG's halo set-up). Diagonal 26, off-diagonals -1; every row
    has 27 entries. Returns (rows, cols, vals, n, n_ghost), triplets sorted by row."""
    n = nx * ny * nz
    r = np.arange(n, dtype=np.int64)
    ix, iy, iz = r % nx, (r // nx) % ny, r // (nx * ny)
    gx, gy = 3 * nx, 3 * ny
    rows = np.repeat(r, 27)
    cols = np.empty(27 * n, np.int64)
    ghost_key = np.full(27 * n, -1, np.int64)
    for k, (dz, dy, dx) in enumerate(_OFFSETS):   # ascending global index within a row
        jx, jy, jz = ix + dx, iy + dy, iz + dz
        inside = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny) & (jz >= 0) & (jz < nz)
        cols[k::27] = np.where(inside, jx + nx * jy + nx * ny * jz, -1)
        # global index of the neighbour in the 3nx x 3ny x 3nz grid (this block in the middle)
        key = (jx + nx) + gx * (jy + ny) + gx * gy * (jz + nz)
        ghost_key[k::27] = np.where(inside, -1, key)
    is_ghost = ghost_key >= 0
    keys = ghost_key[is_ghost]
    uniq, first = np.unique(keys, return_index=True)
    order = np.argsort(first, kind="stable")          # ghosts by first appearance
    gid = np.empty(uniq.size, np.int64)
    gid[order] = np.arange(uniq.size)
    cols[is_ghost] = n + gid[np.searchsorted(uniq, keys)]
    vals = np.where(cols == rows, 26.0, -1.0)
    return rows.astype(np.int32), cols.astype(np.int32), vals, n, int(uniq.size)


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


# ---------------------------------------------------------------------------
# Format-selector families: seeded matrices of four kinds, n log-uniform in
# [n_min, n_max]. The family is seed % 4:
#   0 banded: k in [5, 27] diagonals, symmetric offsets around 0 (DIA-friendly)
#   1 uniform random rows: 8..64 entries per row, uniform columns (CSR-friendly)
#   2 power-law rows: Pareto exponent in [1.8, 2.5], mean 16, at most 20,000 (COO-friendly)
#   3 block diagonal: dense 32 x 32 blocks
# Off-diagonal values U(-1, 1); the diagonal (where present) is sum |row| + 1.
# ---------------------------------------------------------------------------
FAMILIES = ("banded", "uniform", "powerlaw", "blockdiag")


def family_spec(seed: int, n_min: int = 10_000, n_max: int = 2_000_000) -> dict:
    """The scalar choices of selector sample `seed`: family, n (log-uniform in
    [n_min, n_max]), and the family's parameter (banded: the diagonal offsets; power law:
    the exponent), plus the numpy generator that continues the sample's stream."""
    rng = np.random.default_rng(1_000_003 + seed)
    fam = FAMILIES[seed % 4]
    n = int(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
    spec = {"family": fam, "n": n, "rng": rng}
    if fam == "blockdiag":
        spec["n"] = max(32, (n // 32) * 32)
    elif fam == "banded":
        k = int(rng.integers(5, 28))
        half = (k - 1) // 2
        span = int(rng.integers(half, 4 * half + 8)) + 1
        ds = np.sort(rng.choice(np.arange(1, span + 1), half, replace=False))
        offs = np.concatenate([-ds[::-1], [0], ds])
        if offs.size < k:   # even k: one more positive offset
            extra = np.setdiff1d(np.arange(1, span + 2), ds)[:1]
            offs = np.sort(np.concatenate([offs, extra]))
        spec["offsets"] = offs.astype(np.int64)
    elif fam == "powerlaw":
        spec["exponent"] = float(rng.uniform(1.8, 2.5))
    return spec


def family_matrix(seed: int, n_min: int = 10_000, n_max: int = 2_000_000):
    """Returns (family name, n, rows, cols, vals) for selector sample `seed` (numpy, host).
    Rows come out non-decreasing; columns are not sorted within a row."""
    spec = family_spec(seed, n_min, n_max)
    fam, n, rng = spec["family"], spec["n"], spec["rng"]
    if fam == "banded":
        rows, cols = [], []
        for d in spec["offsets"].tolist():
            i = np.arange(max(0, -d), min(n, n - d), dtype=np.int64)
            rows.append(i)
            cols.append(i + d)
        r = np.concatenate(rows)
        c = np.concatenate(cols)
        order = np.argsort(r, kind="stable")
        r, c = r[order], c[order]
    elif fam == "uniform":
        lens = rng.integers(8, 65, n)
        r = np.repeat(np.arange(n, dtype=np.int64), lens)
        c = rng.integers(0, n, r.size)
    elif fam == "powerlaw":
        a = spec["exponent"]
        raw = (1.0 - rng.random(n)) ** (-1.0 / (a - 1.0))
        lens = np.clip(np.floor(raw * (16.0 / raw.mean())), 1, 20_000).astype(np.int64)
        r = np.repeat(np.arange(n, dtype=np.int64), lens)
        c = rng.integers(0, n, r.size)
    else:
        r = np.repeat(np.arange(n, dtype=np.int64), 32)
        c = (r // 32) * 32 + np.tile(np.arange(32, dtype=np.int64), n)
    v = rng.uniform(-1.0, 1.0, r.size)
    diag = r == c
    if diag.any():
        absrow = np.bincount(r, weights=np.abs(v), minlength=n)
        v[diag] = absrow[r[diag]] + 1.0
    return fam, n, r.astype(np.int32), c.astype(np.int32), v


def family_matrix_torch(seed: int, device, n_min: int = 10_000, n_max: int = 2_000_000):
    """The same families and sizes as family_matrix (same family_spec), with the bulk
    arrays drawn by torch on `device` from a generator seeded with `seed` (so the draws
    differ from the numpy ones; on one device type they are reproducible). For building
    thousands of large samples where host generation would dominate.
    Returns (family name, n, rows int32, cols int32, vals float64) as tensors on `device`."""
    import torch
    spec = family_spec(seed, n_min, n_max)
    fam, n = spec["family"], spec["n"]
    g = torch.Generator(device=device)
    g.manual_seed(1_000_003 + seed)
    kw = {"device": device}
    if fam == "banded":
        rows, cols = [], []
        for d in spec["offsets"].tolist():
            i = torch.arange(max(0, -d), min(n, n - d), dtype=torch.int64, **kw)
            rows.append(i)
            cols.append(i + d)
        r = torch.cat(rows)
        c = torch.cat(cols)
        r, order = torch.sort(r, stable=True)
        c = c[order]
    elif fam in ("uniform", "powerlaw"):
        if fam == "uniform":
            lens = torch.randint(8, 65, (n,), generator=g, dtype=torch.int64, **kw)
        else:
            a = spec["exponent"]
            u = torch.rand(n, generator=g, dtype=torch.float64, **kw)
            raw = (1.0 - u) ** (-1.0 / (a - 1.0))
            lens = torch.clamp(torch.floor(raw * (16.0 / raw.mean())), 1, 20_000).to(torch.int64)
        r = torch.repeat_interleave(torch.arange(n, dtype=torch.int64, **kw), lens)
        c = torch.randint(0, n, (r.numel(),), generator=g, dtype=torch.int64, **kw)
    else:
        r = torch.arange(n, dtype=torch.int64, **kw).repeat_interleave(32)
        c = (r // 32) * 32 + torch.arange(32, dtype=torch.int64, **kw).repeat(n)
    v = torch.rand(r.numel(), generator=g, dtype=torch.float64, **kw) * 2.0 - 1.0
    diag = r == c
    absrow = torch.zeros(n, dtype=torch.float64, **kw).index_add_(0, r, v.abs())
    v = torch.where(diag, absrow[r] + 1.0, v)
    return fam, n, r.to(torch.int32), c.to(torch.int32), v
