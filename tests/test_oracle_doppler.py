"""The oracle's Keplerian disk shading (Doppler and gravitational shift)
against the covariant closed form and the sign of the Doppler effect
(oracle_pins.DOPPLER)."""
import pytest

import oracle
import oracle_pins as P


@pytest.mark.parametrize("pin", P.DOPPLER, ids=[p.__name__ for p in P.DOPPLER])
def test_doppler_pin(pin):
    ok, detail = pin(oracle.load())
    assert ok, detail
