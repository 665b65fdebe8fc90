"""Host-side check of the row-block partition behind the paper's distributed HPCG (Sec. VI):
the g^3 stencil cut into P z-slabs, each slab's rows renumbered locally with its ghost columns
(the planes just below and above it) numbered after the local ones in order of first
appearance, split into a local and a remote part; the slabs' products y_s = A_local x_s +
A_remote x_ghost, put back together, equal A x. CPU only: the oracle's SpMV and split on
integer data, so every sum is exact and the comparison is bit for bit."""
import numpy as np
import pytest

import synth


def slab_matrix(g, z0, z1, rows, cols, vals):
    """The rows of planes [z0, z1) of the g^3 stencil, with local columns 0..n_s-1 (the
    slab's own cells in global order) and ghost columns n_s.. numbered by first appearance
    scanning rows in order and, within a row, columns in ascending global index. Returns
    (local rows, columns, values, n_s, ghost global indices in ghost order)."""
    lo, hi = z0 * g * g, z1 * g * g
    m = (rows >= lo) & (rows < hi)
    r, c, v = rows[m].astype(np.int64) - lo, cols[m].astype(np.int64), vals[m]
    own = (c >= lo) & (c < hi)
    keys = c[~own]
    uniq, first = np.unique(keys, return_index=True)
    order = np.argsort(first, kind="stable")
    gid = np.empty(uniq.size, np.int64)
    gid[order] = np.arange(uniq.size)
    n_s = hi - lo
    lc = np.empty_like(c)
    lc[own] = c[own] - lo
    lc[~own] = n_s + gid[np.searchsorted(uniq, keys)]
    ghosts = uniq[order]
    return r.astype(np.int32), lc.astype(np.int32), v, n_s, ghosts


@pytest.mark.parametrize("g,P", [(6, 2), (9, 3), (10, 4), (12, 5)])
def test_zslab_partition_reproduces_spmv(orc, g, P):
    n = g ** 3
    rows, cols, vals = synth.stencil27(g)
    A = orc.Matrix(orc.COO, n, n, rows.size, ai=rows, aj=cols, av=vals)
    x = np.random.default_rng(g * 10 + P).integers(-5, 6, n).astype(np.float64)
    want = orc.spmv(A, x)
    cuts = np.linspace(0, g, P + 1).round().astype(int)
    got = []
    for s in range(P):
        z0, z1 = cuts[s], cuts[s + 1]
        r, c, v, n_s, ghosts = slab_matrix(g, z0, z1, rows, cols, vals)
        # ghosts are exactly the cells of the neighbouring planes that the slab's rows touch
        expect = []
        if z0 > 0:
            expect.append(np.arange((z0 - 1) * g * g, z0 * g * g))
        if z1 < g:
            expect.append(np.arange(z1 * g * g, (z1 + 1) * g * g))
        expect = np.concatenate(expect) if expect else np.zeros(0, np.int64)
        assert np.array_equal(np.sort(ghosts), expect)
        S = orc.canonicalize(n_s, n_s + ghosts.size, r, c, v)
        loc, rem = orc.split_columns(S, n_s)
        # the local part is the slab's own 27-point stencil on a g x g x h grid
        h = z1 - z0
        assert loc.nnz == (3 * g - 2) ** 2 * (3 * h - 2) and loc.nnz + rem.nnz == S.nnz
        x_s = x[z0 * g * g:z1 * g * g]
        y_s = orc.spmv(loc, x_s) + (orc.spmv(rem, x[ghosts]) if rem.nnz else 0.0)
        got.append(y_s)
    assert np.array_equal(np.concatenate(got), want)


def test_zslab_halo_sizes_and_two_allreduce_terms(orc):
    """P slabs of a g^3 grid: an inner slab needs 2 g^2 ghost values per SpMV (one plane from
    each neighbour), an end slab g^2; the two dot products of a CG iteration are sums of the
    slabs' local dot products (exact on integer data)."""
    g, P = 8, 4
    n = g ** 3
    rows, cols, vals = synth.stencil27(g)
    cuts = np.linspace(0, g, P + 1).round().astype(int)
    p = np.random.default_rng(3).integers(-3, 4, n).astype(np.float64)
    q = np.random.default_rng(4).integers(-3, 4, n).astype(np.float64)
    parts = []
    for s in range(P):
        z0, z1 = cuts[s], cuts[s + 1]
        _, _, _, n_s, ghosts = slab_matrix(g, z0, z1, rows, cols, vals)
        assert ghosts.size == (2 if 0 < s < P - 1 else 1) * g * g
        sl = slice(z0 * g * g, z1 * g * g)
        parts.append(float(np.dot(p[sl], q[sl])))
    assert sum(parts) == float(np.dot(p, q))
