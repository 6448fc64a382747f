"""The mixed serving bench's comparison of a sampled request with the
oracle's solve at the served accuracy (bench.serving_case), on CPU."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _ref(converged, certified, pobj=10.0):
    return {"converged": converged, "certified": certified, "pobj": pobj}


def test_same_outcome_passes():
    c = bench.serving_case(3, "pendulum", True, True, 10.0 + 1e-6, _ref(True, True))
    assert c["pass"] and abs(c["rel_obj"] - 1e-6 / 11.0) < 1e-15
    # both stopped at the iteration limit: the same outcome, verdicts aside
    assert bench.serving_case(4, "pendulum", False, False, 3.0, _ref(False, False))["pass"]
    assert bench.serving_case(5, "cartpole", True, False, 12.0, _ref(True, False, 12.0))["pass"]


def test_different_outcome_fails():
    assert not bench.serving_case(6, "pendulum", True, True, 10.0, _ref(False, False))["pass"]
    assert not bench.serving_case(7, "pendulum", False, False, 10.0, _ref(True, True))["pass"]
    assert not bench.serving_case(8, "pendulum", True, False, 10.0, _ref(True, True))["pass"]
