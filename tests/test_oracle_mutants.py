"""Mutation test of the oracle's pins: each build of the oracle with one planted mistake
(a dropped sign, a wrong pivot, a transposed gather, a wrong weight, a dropped
compensation, a wrong cofactor sign, a transposed gradient scatter, a dropped flavour, a
wrong weight in dC/dw) must fail at least one pin.  The mistakes are planted in the
oracle, on the CPU, and never reach the library."""
import pytest

import oracle
import oracle_pins as P

MUTANTS = list(range(1, 10))


@pytest.mark.parametrize("k", MUTANTS)
def test_mutant_is_caught(k, tmp_path):
    path = oracle.build_mutant(k, str(tmp_path))
    failed = []
    with oracle.use_library(path):
        for check in P.ALL_CHECKS:
            try:
                check()
            except AssertionError:
                failed.append(check.__name__)
    assert failed, f"planted mistake {k} passed every pin"
