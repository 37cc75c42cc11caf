"""The oracle still computes what tests/golden/oracle_regression.json recorded
(written by tests/golden/make_oracle_regression.py from the oracle alone): a
guard against unintended changes of the oracle's arithmetic (CPU)."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_oracle_regression  # noqa: E402


def test_oracle_matches_its_recorded_values():
    with open(os.path.join(HERE, "golden", "oracle_regression.json")) as f:
        want = json.load(f)
    got = make_oracle_regression.compute()
    assert set(got) == set(want)
    assert got["philox"] == want["philox"]  # integer: bit-exact
    for key in ("pair", "vertices", "poses", "score_grid", "score_exact", "coords"):
        a, b = np.asarray(got[key], dtype=np.float64), np.asarray(want[key], dtype=np.float64)
        # libm exp / sqrt may differ by an ulp between hosts
        assert np.allclose(a, b, rtol=1e-10, atol=1e-12), key
