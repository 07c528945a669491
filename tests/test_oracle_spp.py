"""The oracle's anti-aliased pixels (n x n stratified samples, box filter);
the check itself is oracle_pins.spp_mean, which the mutant tests also run
against an oracle with a shifted sample grid."""
import oracle
import oracle_pins as P


def test_spp_pixel_is_the_mean_of_its_samples():
    ok, detail = P.spp_mean(oracle.load())
    assert ok, detail
