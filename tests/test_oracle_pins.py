"""The FP64 oracle against its pins (closed forms, invariants, finite differences)."""
import pytest

import oracle
from tests import oracle_pins


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    err, tol = pin(oracle.get())
    assert err <= tol, f"{pin.__name__}: error {err:.3e} > tolerance {tol:.1e}"
