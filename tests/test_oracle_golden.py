"""The oracle reproduces its committed regression fixture
(tests/golden/oracle_icosphere.json, written by tests/golden/make_golden.py
from the oracle alone)."""
import json
import os

import numpy as np
import pytest

import oracle as O
from tests.golden import make_golden as G

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("name,fn", [("icosphere", G.icosphere_fixture),
                                     ("icosphere_absorbing", G.absorbing_fixture)])
def test_oracle_matches_golden(name, fn):
    with open(os.path.join(HERE, "golden", "oracle_icosphere.json")) as f:
        gold = json.load(f)[name]
    now = fn()
    assert now["counters"] == gold["counters"]
    np.testing.assert_allclose(now["image_sum"], gold["image_sum"], rtol=1e-12)
    for k, v in gold["pixels"].items():
        np.testing.assert_allclose(now["pixels"][k], v, rtol=1e-12, atol=1e-15)


def test_oracle_matches_golden_with_absorption_fields():
    with open(os.path.join(HERE, "golden", "oracle_icosphere.json")) as f:
        gold = json.load(f)["icosphere_textured"]
    now = G.textured_fixture()
    for name in ("grid", "hash_texture"):
        assert now[name]["counters"] == gold[name]["counters"]
        np.testing.assert_allclose(now[name]["image_sum"], gold[name]["image_sum"], rtol=1e-12)
        for k, v in gold[name]["pixels"].items():
            np.testing.assert_allclose(now[name]["pixels"][k], v, rtol=1e-12, atol=1e-15)
