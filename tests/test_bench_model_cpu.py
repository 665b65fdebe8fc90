"""The benchmark's algorithmic byte model and DIA traffic bookkeeping, on the CPU.

The per-format GB/s, the HBM fractions and the roofline's `achieved` figure all divide the
byte model by a measured time, so the model is pinned here to counts made independently: the
stored arrays of each format as the oracle builds them (every index and value read once, x
read once, y written once), on small stencils and at the 128^3 benchmark size through the
closed-form entry count."""
import numpy as np
import pytest

import bench
import synth


def stored_bytes(orc, O, n, vbytes=8):
    """Bytes of the arrays one SpMV streams, counted from the oracle's structure."""
    xy = 16 * n   # x read once and y written once, FP64
    if O.fmt == orc.COO:
        return O.ai.nbytes + O.aj.nbytes + vbytes * O.nnz + xy
    if O.fmt == orc.CSR:
        return O.irp.nbytes + O.aj.nbytes + vbytes * O.nnz + xy
    # DIA: the slots of rows 0..n-1 of every diagonal (padding rows >= n are not streamed)
    return vbytes * O.ndiags * n + O.doff.nbytes + xy


@pytest.mark.parametrize("g", [4, 7, 12])
def test_byte_model_matches_the_stored_arrays(orc, g):
    n = g ** 3
    r, c, v = synth.stencil27(g)
    coo = orc.canonicalize(n, n, r, c, v)
    csr, dia = orc.coo_to_csr(coo), orc.coo_to_dia(coo)
    bm = bench.byte_model(n, coo.nnz, dia.ndiags)
    assert bm["coo"] == stored_bytes(orc, coo, n)
    assert bm["csr"] == stored_bytes(orc, csr, n)
    assert bm["dia"] == stored_bytes(orc, dia, n)
    for vb, vt in ((4, "f32"), (2, "bf16")):
        low = bench.byte_model(n, coo.nnz, dia.ndiags, vbytes=vb)
        assert low["dia"] == stored_bytes(orc, orc.with_values(dia, vt), n, vbytes=vb)


def test_byte_model_at_the_benchmark_size():
    """128^3: nnz = 382^3, 27 diagonals; the figures the per-format fractions rest on."""
    g = 128
    n, nnz = g ** 3, (3 * g - 2) ** 3
    bm = bench.byte_model(n, nnz, 27)
    assert nnz == 55_742_968
    assert bm["coo"] == 16 * nnz + 16 * n == 925_441_920
    assert bm["csr"] == 12 * nnz + 4 * (n + 1) + 16 * n == 710_858_660
    assert bm["dia"] == 8 * 27 * n + 4 * 27 + 16 * n == 486_539_372
    # one CG iteration: the DIA matrix once plus 88n bytes of FP64 vectors (the SpMV's p read
    # and q write, 16n; r -= alpha q with x += alpha p, 48n; p = r + beta p, 24n)
    assert bm["cg_iter"] == 8 * 27 * n + 4 * 27 + 88 * n


def test_dia_traffic_scales_by_rows_and_tracks_the_source():
    t = bench.DIA_TRAFFIC
    assert bench.dia_traffic(t["rows"]) == t["bytes"]
    assert bench.dia_traffic(2 * t["rows"]) == 2 * t["bytes"]
    # ncu's DRAM bytes for one 128^3 launch lie just below the algorithmic bytes (part of y
    # is still in L2 when the kernel ends): no re-reads
    assert 0.95 < t["bytes"] / bench.byte_model(128 ** 3, (3 * 128 - 2) ** 3, 27)["dia"] <= 1.0
