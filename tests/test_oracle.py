"""The FP64 oracle against its pins (no GPU needed)."""
import pytest

import oracle
from tests import oracle_pins


@pytest.fixture(scope="module")
def L():
    return oracle.lib()


@pytest.mark.parametrize("check", oracle_pins.ALL_CHECKS, ids=lambda c: c.__name__)
def test_oracle_pin(L, check):
    check(L)
