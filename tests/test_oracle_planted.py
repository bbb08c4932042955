"""The pins catch planted mistakes.

Each case rebuilds the oracle with one deliberate mistake (XGO_PLANT in
oracle/xorgens_oracle.c), routes the oracle to it, and checks that the pin
aimed at that kind of mistake fails, and that the stored golden outputs no
longer reproduce.  The oracle proper is untouched."""
import pytest

import oracle as O
import test_oracle_pins as pins

CASES = {
    1: ("the lag-s term dropped", [lambda: pins.test_impulse_response_closed_form(0),
                                    lambda: pins.test_lag_dependency(0),
                                    lambda: pins.test_minimal_polynomial_irreducible_degree_4096(0)]),
    2: ("(I + R^b) shifting the wrong way", [lambda: pins.test_impulse_response_closed_form(0),
                                              lambda: pins.test_minimal_polynomial_irreducible_degree_4096(1)]),
    3: ("the operator pairs of the two lags swapped",
        [lambda: pins.test_impulse_response_closed_form(1),
         lambda: pins.test_minimal_polynomial_irreducible_degree_4096(0)]),
    4: ("the Weyl shift gamma off by one", [pins.test_weyl_combination_invariant]),
    5: ("the Weyl word used before it is advanced", [pins.test_weyl_combination_invariant]),
    6: ("63 xorshift outputs discarded in seeding",
        [lambda: pins.test_seed_procedure_recovered_through_the_warm_up(0)]),
    7: ("low halves of the xorshift outputs taken in seeding",
        [lambda: pins.test_seed_procedure_recovered_through_the_warm_up(1)]),
    8: ("xorshift triple (13, 7, 18) in seeding",
        [pins.test_seed_xorshift_is_marsaglia_13_7_17_full_period,
         lambda: pins.test_seed_procedure_recovered_through_the_warm_up(0)]),
    9: ("4r - 1 warm-up words discarded in seeding",
        [lambda: pins.test_seed_procedure_recovered_through_the_warm_up(0)]),
}


@pytest.mark.parametrize("plant", sorted(CASES))
def test_pins_catch_planted_mistake(plant):
    what, checks = CASES[plant]
    with O.planted(plant):
        for check in checks:
            with pytest.raises(AssertionError):
                check()
        with pytest.raises(AssertionError):
            pins.test_golden_regression()


def test_unplanted_oracle_passes_the_same_checks():
    for _, checks in CASES.values():
        for check in checks:
            check()
    pins.test_golden_regression()


CASES_W64 = {
    1: ["test_w64_impulse_response_closed_form", "test_w64_lag_dependency",
        "test_w64_minimal_polynomial_primitive_degree_4096"],
    2: ["test_w64_impulse_response_closed_form", "test_w64_minimal_polynomial_primitive_degree_4096"],
    3: ["test_w64_impulse_response_closed_form", "test_w64_minimal_polynomial_primitive_degree_4096"],
    4: ["test_w64_weyl_combination_invariant"],
    5: ["test_w64_weyl_combination_invariant"],
    6: ["test_w64_seed_procedure_recovered_through_the_warm_up"],
    7: ["test_w64_seed_procedure_recovered_through_the_warm_up"],
    8: ["test_w64_seed_xorshift_is_marsaglia_13_7_17_full_period",
        "test_w64_seed_procedure_recovered_through_the_warm_up"],
    9: ["test_w64_seed_procedure_recovered_through_the_warm_up"],
}


@pytest.mark.parametrize("plant", sorted(CASES_W64))
def test_w64_pins_catch_planted_mistake(plant):
    """The same mistakes planted in the 64-bit oracle (7: its ring filled
    newest first, there being no halves to take)."""
    import test_oracle_w64_pins as p64
    with O.planted(plant):
        for name in CASES_W64[plant]:
            with pytest.raises(AssertionError):
                getattr(p64, name)()
