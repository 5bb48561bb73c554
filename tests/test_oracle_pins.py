"""The FP64 oracle against closed forms, libraries, invariants and hand-derived examples."""
import pytest

import pins


@pytest.mark.parametrize("pin", pins.ALL, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    pin(orc)


@pytest.mark.parametrize("pin,fn", pins.py_pins(), ids=lambda v: v.__name__)
def test_python_oracle_pin(pin, fn):
    pin(fn)


def test_local_theta_pin(orc):
    from oracle import gp
    pins.pyo_local_theta(gp.local_theta, orc)
