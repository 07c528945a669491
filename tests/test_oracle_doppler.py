"""The oracle's Keplerian disk shading (Doppler and gravitational shift)
against the covariant closed form and the sign of the Doppler effect
(oracle_pins.DOPPLER), and its image sky against the exactness of bilinear
interpolation on affine images (oracle_pins.SKY_TEXTURE)."""
import pytest

import oracle
import oracle_pins as P


@pytest.mark.parametrize("pin", P.DOPPLER + P.SKY_TEXTURE,
                         ids=[p.__name__ for p in P.DOPPLER + P.SKY_TEXTURE])
def test_doppler_pin(pin):
    ok, detail = pin(oracle.load())
    assert ok, detail
