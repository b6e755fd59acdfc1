"""The oracle against its stored results (tests/golden/, written by
tests/golden/make_golden.py, which calls only the oracle): a guard against
unintended change of the oracle's arithmetic.  Fixed rho and gamma, so no
discrete adapt decision can turn on rounding."""
import json
import os

import numpy as np
import pytest

from oracle import parsdmm as P
from paper_1902_09699_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FILES = sorted(f for f in os.listdir(GOLDEN) if f.endswith(".json"))


def _model(spec):
    if spec["kind"] == "layered":
        return W.layered(tuple(spec["n"]), n_layers=spec["n_layers"], seed=spec["seed"])
    return W.grf(tuple(spec["n"]), seed=spec["seed"])


def test_golden_files_present():
    assert len(FILES) >= 2


@pytest.mark.parametrize("name", FILES)
def test_oracle_reproduces_its_stored_result(name):
    with open(os.path.join(GOLDEN, name)) as f:
        g = json.load(f)
    case, want = g["case"], g["result"]
    res = P.parsdmm(_model(case["model"]), case["grid"], case["sets"], P.options(**case["opts"]))
    x = np.asarray(want["x"])
    assert np.linalg.norm(res["x"] - x) <= 1e-12 * np.linalg.norm(x)
    assert int(res["cg_steps"]) == want["cg_steps"]
