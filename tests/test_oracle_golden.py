"""The oracle against its recorded outputs (tests/golden/oracle_regression.json, written by
tests/golden/make_oracle_golden.py from the oracle itself). This is a regression guard, not an independent
pin: the independent pins are in test_oracle_pins.py and test_oracle_retooled.py. A change to the oracle's
arithmetic must regenerate the file, and the commit must name the passage of the paper that justifies it."""
import json
import os

import numpy as np
import pytest

from golden.make_oracle_golden import CASES, SAMPLE, run

with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_regression.json")) as f:
    GOLD = json.load(f)


def test_fixture_matches_the_case_list():
    assert GOLD["sample_stride"] == SAMPLE
    assert sorted(GOLD["cases"]) == sorted(c[0] for c in CASES)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_oracle_reproduces_recorded_output(case):
    g = GOLD["cases"][case[0]]
    res = run(case)
    assert int(res.status) == g["status"] and int(res.iters) == g["iters"]
    assert [int(v) for v in res.block_iters] == g["block_iters"]
    x = res.X.ravel()[::SAMPLE]
    assert np.allclose(x, g["x_sample"], rtol=1e-10, atol=1e-13 * np.abs(x).max())   # BLAS rounding may differ by machine
    assert np.allclose(res.relres_recursive, g["relres_recursive"], rtol=1e-9, atol=1e-300)
