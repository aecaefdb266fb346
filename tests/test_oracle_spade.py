"""The oracle's SPADE downsampling against its pins, and planted mistakes that the
pins must catch."""
import numpy as np
import pytest

import oracle
import spade_pins as pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_spade_pin(ref, pin):
    pin(ref)


MUTANTS = {
    "find_not_strict": ("found[j] = D < apprx;", "found[j] = D <= apprx;"),
    "no_skip_test": ("    if (dens[i] != 0) continue;  /* the skip test */\n", ""),
    "policy0_fills_only": ("if (policy == 0 || dens[j] == 0) dens[j] = (int32_t)c;",
                           "if (dens[j] == 0) dens[j] = (int32_t)c;"),
    "policy0_counts_apprx": ("c += policy == 0 ? (D < kernel) : (D < apprx || D < kernel);",
                             "c += (D < apprx || D < kernel);"),
    "squared_not_l1": ("for (int32_t t = 0; t < d; ++t) s += fabs((double)x[t] - (double)y[t]);",
                       "for (int32_t t = 0; t < d; ++t) s += ((double)x[t] - (double)y[t]) * ((double)x[t] - (double)y[t]);"),
    "dropped_column": ("for (int32_t t = 0; t < d; ++t) s += fabs((double)x[t] - (double)y[t]);",
                       "for (int32_t t = 1; t < d; ++t) s += fabs((double)x[t] - (double)y[t]);"),
    "policy1_own_density_missing": ("    if (policy == 1) dens[i] = (int32_t)c;\n", ""),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_spade_planted_mistake_is_caught(tmp_path, name):
    src = open(oracle._SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mpath = tmp_path / "kmref_mut.c"
    mpath.write_text(src.replace(old, new))
    mut = oracle.Oracle(oracle.bind(oracle.compile_oracle(str(mpath), str(tmp_path / "libkmref_mut.so"))))
    caught = []
    for pin in pins.ALL_PINS:
        try:
            pin(mut)
        except (AssertionError, ValueError):
            caught.append(pin.__name__)
    if name == "policy1_own_density_missing":
        # a reading check, not a mistake: with apprx > 0 an evaluated row always finds itself, so the
        # snippet's explicit own-density write changes nothing (the pins must agree with both builds)
        assert not caught, caught
        return
    assert caught, f"no pin caught the planted mistake {name}"


def test_spade_oracle_rejects_bad_args(ref):
    X = np.zeros((3, 2), np.float32)
    for a, w, p in ((0.0, 1.0, 0), (1.0, 0.0, 0), (-1.0, 1.0, 1), (1.0, 1.0, 2), (float("nan"), 1.0, 0)):
        with pytest.raises(ValueError):
            ref.spade(X, a, w, p)
