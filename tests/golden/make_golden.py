"""Writes the stored expected values under tests/golden/ from the CPU oracle alone.

Run from the repository root: python tests/golden/make_golden.py
Every value here comes from oracle/ (and the seeded generators in synth/); nothing comes
from the CUDA library. The fixtures are small text files:

  stencil4_dia.txt   DIA form (Sec. II-B-3) of the 27-point stencil on a 4^3 grid: offsets,
                     npad and the diagonal-major value array.
  cg_stencil8.txt    Unpreconditioned CG (Sec. VI) on the 8^3 stencil, b = A 1, x0 = 0,
                     tol 1e-10: iteration count and the relative residual after each iteration.
  rank_split_3x4x5.txt  The matrix of one interior process (3 x 4 x 5 block, Sec. VI's
                     distributed set-up) split into local and remote parts: sizes and the
                     remote part's triplets.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def stencil4_dia():
    g = 4
    r, c, v = synth.stencil27(g)
    D = oracle.coo_to_dia(oracle.canonicalize(g ** 3, g ** 3, r, c, v))
    return D


def cg_stencil8():
    g = 8
    n = g ** 3
    r, c, v = synth.stencil27(g)
    O = oracle.convert(oracle.canonicalize(n, n, r, c, v), "dia")
    b = oracle.spmv(O, np.ones(n))
    _, st, k, rel, hist, _ = oracle.cg(O, b, tol=1e-10, maxit=200)
    return st, k, rel, hist / hist[0]


def rank_split():
    r, c, v, n, ng = synth.hpcg_rank_matrix(3, 4, 5)
    O = oracle.canonicalize(n, n + ng, r, c, v)
    return n, ng, oracle.split_columns(O, n)


def main():
    D = stencil4_dia()
    with open(os.path.join(HERE, "stencil4_dia.txt"), "w") as f:
        f.write("# DIA form of the 27-point stencil, 4^3 grid (oracle); n ndiags npad, offsets, values\n")
        f.write(f"{D.nrows} {D.ndiags} {D.npad}\n")
        f.write(" ".join(str(int(o)) for o in D.doff) + "\n")
        for d in range(D.ndiags):
            f.write(" ".join(repr(float(a)) for a in D.av[d * D.npad:(d + 1) * D.npad]) + "\n")
    st, k, rel, hist = cg_stencil8()
    with open(os.path.join(HERE, "cg_stencil8.txt"), "w") as f:
        f.write("# CG on the 8^3 stencil, b = A 1, x0 = 0, tol 1e-10 (oracle); status iters relres, "
                "then ||r_k|| / ||r_0|| for k = 0..iters\n")
        f.write(f"{st} {k} {rel!r}\n")
        f.write("\n".join(repr(float(h)) for h in hist) + "\n")
    n, ng, (L, R) = rank_split()
    with open(os.path.join(HERE, "rank_split_3x4x5.txt"), "w") as f:
        f.write("# one interior process, 3x4x5 block (oracle split): n ghosts local_nnz remote_nnz, "
                "then remote triplets (row col value)\n")
        f.write(f"{n} {ng} {L.nnz} {R.nnz}\n")
        for i, j, a in zip(R.ai, R.aj, R.av):
            f.write(f"{int(i)} {int(j)} {float(a)!r}\n")


if __name__ == "__main__":
    oracle.build()
    main()
