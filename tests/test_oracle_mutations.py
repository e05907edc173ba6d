"""The oracle pins are sensitive: each plausible mistake planted in a
temporary copy of the oracle source makes at least one pin fail (CPU only;
the committed oracle is untouched)."""
import os
import subprocess

import numpy as np
import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "msd_oracle.c")

MUTANTS = {
    "exchange dropped": ("two += J * J - X;", "two += J * J;"),
    "pivot sign lost": ("det = -det;", "(void)det;"),
    "inverse transposed": ("w->Sinv[k * n + j]", "w->Sinv[j * n + k]"),
    "two-body half dropped": ("*energy = E + 0.5 * two;", "*energy = E + two;"),
    "CI coefficient dropped in G_T": ("+= cO * GI[j * M + q]", "+= O * GI[j * M + q]"),
    "exchange index order": ("X += w->GL[i * n + j] * w->GL[j * n + i];",
                             "X += w->GL[i * n + j] * w->GL[i * n + j];"),
}


def _run_pins():
    """True if every pin passes with the currently bound oracle."""
    try:
        for args in [(5, 2, 2, None, None, 0), (6, 3, 2, 60, None, 1)]:
            pins.test_brute_force_fock(*args)
        pins.test_hartree_fock_closed_form()
        pins.test_green_function_idempotent_and_trace()
        pins.test_per_determinant_overlap_is_the_determinant()
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found: {old}"
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared",
                           "-o", str(so), str(mut), "-lm"])
    saved = oracle._load()
    try:
        oracle._lib = oracle.bind(str(so))
        assert not _run_pins(), f"pins did not catch: {name}"
    finally:
        oracle._lib = saved
    assert _run_pins()
