"""The FP64 oracle against its pins, and planted mistakes that the pins must catch."""
import os
import shutil

import numpy as np
import pytest

import oracle
import oracle_pins as pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(ref, pin):
    pin(ref)


# Each mutant plants one plausible mistake in a copy of the oracle source.
MUTANTS = {
    "tie_highest_index": ("      if (D < b1) {", "      if (D <= b1) {"),
    "dropped_term": ("  for (int32_t t = 0; t < d; ++t) {\n    double diff", "  for (int32_t t = 1; t < d; ++t) {\n    double diff"),
    "wrong_sign": ("double diff = (double)x[t] - c[t];", "double diff = (double)x[t] + c[t];"),
    "transposed_stride": ("double D = sqdist(x, C + (int64_t)j * d, d);", "double D = sqdist(x, C + (int64_t)j, d);"),
    "empty_cluster_zeroed": ("s[t] / (double)counts[j] : cp[t];", "s[t] / (double)counts[j] : 0.0;"),
    "objective_new_centroids": ("*objective = kmref_objective(X, n, d, Cold, k, assign);",
                                "*objective = kmref_objective(X, n, d, C, k, assign);"),
    "mean_off_by_one": ("s[t] / (double)counts[j]", "s[t] / (double)(counts[j] + 1)"),
    "second_not_tracked": ("      } else if (D < b2) {\n        b2 = D; j2 = j;\n      }", "      }"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    src = open(oracle._SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mpath = tmp_path / "kmref_mut.c"
    mpath.write_text(src.replace(old, new))
    lib = oracle.bind(oracle.compile_oracle(str(mpath), str(tmp_path / "libkmref_mut.so")))
    mut = oracle.Oracle(lib)
    caught = []
    for pin in pins.ALL_PINS:
        try:
            pin(mut)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"no pin caught the planted mistake {name}"


def test_oracle_rejects_bad_args(ref):
    X = np.zeros((4, 2), np.float32)
    with pytest.raises(ValueError):
        ref.assign(X, np.zeros((5, 2)))  # k > n
    with pytest.raises(ValueError):
        ref.assign(np.zeros((0, 2), np.float32), np.zeros((1, 2)))
