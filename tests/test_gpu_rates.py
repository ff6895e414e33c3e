"""grins_unit_rates: the measured per-clock issue rates that the rooflines of
the bench divide by.  The rates are per SM clock, so they do not move with
the clock frequency; the bounds below are loose brackets around the unit
counts of a Blackwell SM (128 FP32 lanes, packed f32x2 instructions, a
special-function unit of 16 lanes for the reciprocal class), wide enough for any clock or driver, tight
enough to catch a probe that measured the wrong thing (a loop the compiler
removed reads as an absurd rate, a shared SM as half of one)."""
import pytest

pytestmark = pytest.mark.gpu


def test_unit_rates_are_plausible_and_repeatable():
    from paper_2503_18356_gb300 import api
    a = api.unit_rates()
    b = api.unit_rates()
    print(a)
    assert set(a) == set(api.UNIT_RATE_NAMES)
    assert 8.0 <= a["rcp"] <= 40.0
    assert 8.0 <= a["lg2"] <= 40.0
    assert a["rcp"] * 0.9 <= a["ex2"] <= 72.0          # ex2 at least the reciprocal rate
    # FP32 FMA lane operations: 128 lanes per SM, twice that at most where
    # the compiler packs independent FMAs into f32x2 instructions
    assert 64.0 <= a["ffma"] <= 272.0
    assert 0.1 <= a["dfma"] <= 72.0
    assert 0.1 <= a["dmul"] <= 72.0 and 0.1 <= a["dadd"] <= 72.0
    assert a["ffma"] > 4.0 * a["rcp"]
    for k in a:
        assert abs(a[k] - b[k]) <= 0.05 * a[k], (k, a[k], b[k])


def test_unit_rates_rejects_null():
    import ctypes as C
    from paper_2503_18356_gb300 import api
    st = api._lib.grins_unit_rates(C.cast(None, C.POINTER(C.c_double)), None)
    assert st == api.GRINS_E_INVALID_ARG
