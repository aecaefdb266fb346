"""The oracle's keyed-reduce training (GDA, naive Bayes) against its pins, and
planted mistakes that the pins must catch."""
import numpy as np
import pytest

import keyed_pins as pins
import oracle


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_keyed_pin(ref, pin):
    pin(ref)


MUTANTS = {
    "gda_global_centre": ("const double* m = mu + (int64_t)y[i] * d;", "const double* m = mu;"),
    "gda_per_class_divisor": ("const double v = sigma[(int64_t)a * d + b] / (double)n;",
                              "const double v = sigma[(int64_t)a * d + b] / (double)(n - 1);"),
    "gda_upper_only": ("        sigma[(int64_t)b * d + a] = v;\n", ""),
    "gda_prior_unnormalised": ("phi[k] = (double)counts[k] / (double)n;", "phi[k] = (double)counts[k];"),
    "nb_denominator_plus_one": ("(total + (double)d)", "(total + 1.0)"),
    "nb_numerator_unsmoothed": ("s[t] = (s[t] + 1.0)", "s[t] = (s[t] + 0.0)"),
    "class_sums_wrong_stride": ("double* s = sums + (int64_t)c * d;", "double* s = sums + (int64_t)c;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_keyed_planted_mistake_is_caught(tmp_path, name):
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
    assert caught, f"no pin caught the planted mistake {name}"


def test_keyed_oracle_rejects_bad_labels(ref):
    X = np.zeros((3, 2), np.float32)
    with pytest.raises(ValueError):
        ref.gda(X, np.array([0, 2, 1], np.int32), 2)
    with pytest.raises(ValueError):
        ref.nb(X, np.array([0, -1, 1], np.int32), 2)
