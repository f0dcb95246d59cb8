"""The irradiance oracle against its pins (closed forms, exact arithmetic,
symmetry, conservation, solid angle, superposition, grazing flags)."""
import pytest

import oracle
from tests import _pins


@pytest.mark.parametrize("pin", _pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(oracle.irradiance)
