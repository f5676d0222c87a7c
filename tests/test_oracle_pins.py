"""Oracle pins (CPU): the oracle against the paper's identities, closed forms, exact
arithmetic and LAPACK on small inputs.  See tests/oracle_pins.py for each check."""
import pytest

import oracle_pins as P


@pytest.mark.parametrize("check", P.ALL_CHECKS, ids=lambda c: c.__name__)
def test_oracle_pin(check):
    check()
