"""The FP64 CPU oracle against its pins (CPU only)."""
import pytest

import oracle_pins as P
from oracle.oracle import get


@pytest.fixture(scope="module")
def orc():
    return get()


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=[p.__name__ for p in P.ALL_PINS])
def test_pin(orc, pin):
    pin(orc)


def test_penta_rejects_small_n(orc):
    import numpy as np
    with pytest.raises(ValueError):
        orc.penta_solve(1.0, np.ones(4))
