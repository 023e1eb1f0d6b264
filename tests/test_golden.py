"""Regression fixtures of the seeded generator and the oracle (tests/golden).

The fixtures are oracle outputs written by tests/golden/make_golden.py; the
oracle's correctness is pinned separately (tests/test_oracle_pins.py).
These catch unintended changes to the generator's draw order or to the
oracle's arithmetic: a deliberate change regenerates them and says why.
"""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
FIX = json.load(open(os.path.join(HERE, "golden", "oracle_small.json")))


@pytest.mark.parametrize("entry", FIX["cases"], ids=lambda e: "x".join(map(str, e["case"])))
def test_oracle_reproduces_fixture(entry):
    import sys
    sys.path.insert(0, os.path.join(HERE, "golden"))
    from make_golden import case_values
    got = case_values(*entry["case"])
    for (n0, f0), (n1, f1) in zip(entry["inputs"], got["inputs"]):
        assert n1 == pytest.approx(n0, rel=1e-10) and f1 == pytest.approx(f0, rel=1e-10, abs=1e-14)
    for key in ("energy", "sigma_fro", "sigma1_fro", "sigma_00", "sigma1_00", "mp2"):
        assert got[key] == pytest.approx(entry[key], rel=1e-9, abs=1e-13), key
