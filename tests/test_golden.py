"""The oracle reproduces the stored regression fixtures (written by
tests/golden/make_golden.py from the oracle alone). A change to the oracle's arithmetic
shows up here and must be justified by the passage of the paper it follows."""
import json
import os

import pytest

from tests.conftest import ROOT
from tests.golden import make_golden

with open(os.path.join(ROOT, "tests", "golden", "oracle_regression.json")) as f:
    GOLDEN = json.load(f)["cases"]


@pytest.mark.parametrize("name,prob", make_golden.CASES, ids=[c[0] for c in make_golden.CASES])
def test_oracle_regression(name, prob):
    assert make_golden.summarise(prob) == GOLDEN[name]
