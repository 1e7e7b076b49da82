"""The oracle against its stored expected values (tests/golden/, written by
tests/golden/make_golden.py from the oracle alone): a change to the oracle's
arithmetic shows up here and has to be justified by the paper."""
import json
import os

from tests.golden import make_golden

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_reproduces_golden_star3(oracle):
    with open(os.path.join(HERE, "golden", "star3_brownian.json")) as f:
        stored = json.load(f)
    assert make_golden.compute() == stored
    # the stored case is not degenerate: particles hit the vertex and exit
    assert sum(stored["hits"]) > 0 and sum(stored["exits"]) > 0
    assert sum(stored["histogram"]) == stored["case"]["n"]
