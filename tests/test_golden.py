"""The oracle reproduces the fixtures of tests/golden (regression guard).

The fixtures were written by tests/golden/make_golden.py from the oracle
itself; they are not an independent pin (the closed-form and invariant pins
are in test_oracle_pins.py) but fail when the oracle's results change.
"""

import os

import numpy as np
import pytest

from tests.golden import make_golden

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    a = np.loadtxt(os.path.join(HERE, f"{name}_2x2x2x4.txt"))
    return a[:, 0] + 1j * a[:, 1]


@pytest.mark.parametrize("name", ["wilson_D", "clover_D", "schur_Dhat", "solution", "mobius_D", "mobius_Dhat_dag",
                                  "staggered_D", "staggered_Dhat", "mg_cycle", "mg_coarse_eo_solve"])
def test_oracle_matches_golden(name):
    got = np.asarray(make_golden.cases()[name]).reshape(-1)
    want = load(name)
    assert np.max(np.abs(got - want)) <= 1e-12 * max(1.0, np.max(np.abs(want)))
