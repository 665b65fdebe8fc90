"""Planted mistakes in the oracle must fail its pins.

Each case compiles a copy of ``oracle/oracle.c`` with one plausible mistake written into
it, loads that copy in place of the oracle library for the duration of the test, and
runs the pins of ``test_oracle_pins`` against it: at least one must fail. This checks that
the pins see the mistakes a restatement of the method could plausibly make: in the three
SpMV algorithms (an overwrite for an accumulation, an entry skipped, an off-by-one bound),
in CG (an inverted beta, a wrong vector or sign in an update) and in refinement and reliable
updates, which the paper does not define and which therefore have no printed values to
compare with (a swapped matrix, a dropped carry, a wrong sign). CPU only; needs gcc.
"""
from __future__ import annotations

import shutil
import subprocess

import pytest

import oracle
import test_oracle_pins as pins


def _compile_mutant(tmp_path, original: str, replacement: str, count: int) -> str:
    src = open(oracle._SRC).read()
    assert src.count(original) == count, f"anchor {original!r} not found {count} time(s)"
    (tmp_path / "oracle.c").write_text(src.replace(original, replacement))
    shutil.copy(oracle._HDR, tmp_path / "oracle.h")
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared",
                    "-fPIC", "-o", str(lib), str(tmp_path / "oracle.c"), "-lm"], check=True)
    return str(lib)


def _use(monkeypatch, lib: str) -> None:
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(oracle, "build", lambda force=False: lib)


def _fails(check) -> bool:
    try:
        check()
    except AssertionError:
        return True
    return False


@pytest.fixture(autouse=True)
def _gcc():
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")


IR_MUTANTS = {
    # the inner CG solves with the FP64 matrix instead of the rounded one
    "inner_on_A64": ("orc_cg(Alo, r, d,", "orc_cg(A64, r, d,", 1),
    # the outer residual is taken from the rounded matrix
    "residual_from_Alo": ("matvec(A64, x, r);", "matvec(Alo, x, r);", 1),
    # the correction is subtracted
    "update_sign": ("x[i] = x[i] + d[i];", "x[i] = x[i] - d[i];", 1),
}


@pytest.mark.parametrize("name", sorted(IR_MUTANTS))
def test_refinement_pins_catch_planted_mistake(tmp_path, monkeypatch, name):
    # the pin passes on the oracle as committed
    pins.check_refinement_outer_steps(oracle, "bf16")
    lib = _compile_mutant(tmp_path, *IR_MUTANTS[name])
    _use(monkeypatch, lib)
    assert _fails(lambda: pins.check_refinement_outer_steps(oracle, "bf16"))


RU_MUTANTS = {
    # the replaced residual (and the starting one) come from the rounded matrix
    "residual_from_Alo": ("matvec(A64, x, q);", "matvec(Alo, x, q);", 2),
    # rho is not carried to the next iteration
    "rho_not_carried": ("        rho = rr;\n", "\n", 1),
}


@pytest.mark.parametrize("name", sorted(RU_MUTANTS))
def test_reliable_update_pins_catch_planted_mistake(tmp_path, monkeypatch, name):
    lib = _compile_mutant(tmp_path, *RU_MUTANTS[name])
    _use(monkeypatch, lib)
    caught = (_fails(lambda: pins.test_cg_ru_iterates_match_exact_rational_cg(oracle))
              or _fails(lambda: pins.test_cg_ru_solves_the_fp64_system(oracle, "bf16"))
              or _fails(lambda: pins.test_cg_ru_solves_the_fp64_system(oracle, "f32")))
    assert caught


SPMV_MUTANTS = {
    # Algorithm 1 writes y(ai) instead of accumulating into it
    "coo_overwrites": ("y[ai[e]] += av[e] * x[aj[e]];", "y[ai[e]] = av[e] * x[aj[e]];", 1),
    # Algorithm 2 starts each row one entry late
    "csr_skips_first_entry": ("for (int32_t j = irp[i]; j < irp[i + 1]; j++) sum += av[j] * x[aj[j]];",
                              "for (int32_t j = irp[i] + 1; j < irp[i + 1]; j++) sum += av[j] * x[aj[j]];", 1),
    # Algorithm 3's bounds check excludes column 0
    "dia_bound_off_by_one": ("if (k >= 0 && k < n) sum += av[(int64_t)j * npad + i] * x[k];",
                             "if (k > 0 && k < n) sum += av[(int64_t)j * npad + i] * x[k];", 1),
}


@pytest.mark.parametrize("name", sorted(SPMV_MUTANTS))
def test_spmv_pins_catch_planted_mistake(tmp_path, monkeypatch, name):
    for c in pins.SMALL_CASES:   # the pins pass on the oracle as committed
        pins.test_spmv_matches_dense_brute_force(oracle, c)
    lib = _compile_mutant(tmp_path, *SPMV_MUTANTS[name])
    _use(monkeypatch, lib)
    caught = any(_fails(lambda c=c: pins.test_spmv_matches_dense_brute_force(oracle, c)) for c in pins.SMALL_CASES)
    assert caught


CG_MUTANTS = {
    # beta formed the wrong way round
    "beta_inverted": ("double beta = rho_new / rho;", "double beta = rho / rho_new;", 1),
    # the solution advanced along q instead of p
    "x_along_q": ("x[i] = x[i] + alpha * p[i];", "x[i] = x[i] + alpha * q[i];", 1),
    # the residual updated with the wrong sign (also in the reliable-update solver's copy)
    "residual_sign": ("r[i] = r[i] - alpha * q[i];", "r[i] = r[i] + alpha * q[i];", 2),
}


@pytest.mark.parametrize("name", sorted(CG_MUTANTS))
def test_cg_pins_catch_planted_mistake(tmp_path, monkeypatch, name):
    pins.test_cg_iterates_match_exact_rational_cg(oracle)   # passes on the oracle as committed
    pins.test_cg_recovers_ones(oracle, 8, "csr")
    lib = _compile_mutant(tmp_path, *CG_MUTANTS[name])
    _use(monkeypatch, lib)
    caught = (_fails(lambda: pins.test_cg_iterates_match_exact_rational_cg(oracle))
              or _fails(lambda: pins.test_cg_recovers_ones(oracle, 8, "csr")))
    assert caught
