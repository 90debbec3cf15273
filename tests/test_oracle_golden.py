"""The oracle still reproduces its stored regression values (tests/golden)."""
import json
import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def test_oracle_reproduces_golden_values():
    with open(os.path.join(HERE, "golden", "disk64_oracle.json")) as f:
        stored = json.load(f)["values"]
    now = make_golden.compute()
    for tag in stored:
        for key, val in stored[tag].items():
            if isinstance(val, dict):
                for k2, v2 in val.items():
                    assert now[tag][key][k2] == pytest.approx(v2, rel=1e-9, abs=1e-15)
            elif isinstance(val, list):
                assert now[tag][key] == pytest.approx(val, rel=1e-9, abs=1e-15)
            else:
                assert now[tag][key] == pytest.approx(val, rel=1e-9, abs=1e-15)
