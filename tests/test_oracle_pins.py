"""The FP64 oracle against closed forms, libraries, invariants and hand-derived examples."""
import pytest

import pins


@pytest.mark.parametrize("pin", pins.ALL, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    pin(orc)
