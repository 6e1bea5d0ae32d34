"""The oracle against closed forms, brute force, library routines and finite differences (CPU)."""
import json
import os

import pytest

import oracle_pins as P
from oracle.oracle import Params


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(oracle, pin):
    pin(oracle)


def test_defaults_match_paper_constants():
    with open(os.path.join(P.GOLDEN, "paper_constants.json")) as f:
        g = json.load(f)
    assert Params().sigma == g["sigma"]["value"]
