"""The oracle reproduces its frozen 8^3 outputs (tests/golden/oracle_steps.json).

The paper prints no worked example, so the fixture was written by
tests/golden/make_golden.py from the oracle alone.  This test makes any
change to the oracle's arithmetic visible: regenerate the fixture only with a
change that names the passage (or the reading of it) that justifies it.
"""
import json
import os

import numpy as np
import pytest

from .golden import make_golden

FIXTURE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_steps.json")


def _close(got, want, rtol, path):
    if isinstance(want, dict):
        assert set(got) == set(want), path
        for k in want:
            _close(got[k], want[k], rtol, f"{path}.{k}")
    elif isinstance(want, list):
        assert len(got) == len(want), path
        for i, (g, w) in enumerate(zip(got, want)):
            _close(g, w, rtol, f"{path}[{i}]")
    elif isinstance(want, bool) or want is None or isinstance(want, int):
        assert got == want, (path, got, want)
    else:
        assert abs(got - want) <= rtol * max(abs(want), 1e-300), (path, got, want)


@pytest.mark.parametrize("name", sorted(make_golden.CASES))
def test_oracle_matches_frozen_outputs(name):
    with open(FIXTURE) as f:
        data = json.load(f)
    want = data["cases"][name]
    got = json.loads(json.dumps(make_golden.run_case(name)))
    for s_got, s_want in zip(got["steps"], want["steps"]):
        assert s_got["iters"] == s_want["iters"]
    _close(got, want, 1e-10, name)


def test_fixture_states_its_source():
    with open(FIXTURE) as f:
        data = json.load(f)
    assert "oracle/" in data["source"] and "make_golden" in data["source"]
    assert np.isfinite(data["cases"]["barotropic"]["steps"][0]["dt"])
