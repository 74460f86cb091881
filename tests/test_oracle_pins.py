"""The FP64 oracle against closed forms, brute force and invariants."""
import pytest

import oracle.communicability as oc
from tests import pins


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda f: f.__name__)
def test_oracle_pin(check):
    check(oc)
