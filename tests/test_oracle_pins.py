"""The CPU oracle against its pins (closed forms, published constants,
library routines, exact invariants). CPU only."""
import pytest

import oracle_pins


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin()
