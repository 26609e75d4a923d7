"""The stored oracle fixtures under tests/golden/ (written by
tests/golden/make_golden.py): the oracle as it stands must reproduce them,
so a change to its arithmetic shows here as well as in the pins."""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NAMES = sorted(f[:-5] for f in os.listdir(GOLDEN) if f.endswith(".json"))


def load(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        return json.load(f)


def test_fixtures_exist():
    assert NAMES


@pytest.mark.parametrize("name", NAMES)
def test_oracle_reproduces_fixture(name):
    g = load(name)
    x = {k: np.asarray(v) for k, v in g["inputs"].items()}
    r, eps = g["r"], g["eps"]
    O = oracle.forward(x["p_l"], x["I_l"], x["I_h"], r, eps)
    dp, dil, dih = oracle.backward(x["R"], x["p_l"], x["I_l"], x["I_h"], r, eps)
    for got, key in ((O, "O_h"), (dp, "dp_l"), (dil, "dI_l"), (dih, "dI_h")):
        ref = np.asarray(g["expected"][key])
        assert got.shape == ref.shape
        assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref))), key
