"""Writes the stored oracle results under tests/golden/ (run from the
repository root: python tests/golden/make_golden.py).  Calls only oracle/
and the seeded input generators; the paper prints no worked numeric example
of a projection (its results are figures and timing tables), so these files
pin the oracle against unintended change, not against the paper."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import parsdmm as P                   # noqa: E402
from paper_1902_09699_gb300 import workloads as W  # noqa: E402

CASES = {
    "small_grid_three_sets": dict(
        grid={"n": [8, 6]},
        model=dict(kind="layered", n=[8, 6], n_layers=3, seed=71),
        sets=[{"op": "I", "type": "bounds", "lo": 2.0, "hi": 4.0},
              {"op": "TV", "type": "l1", "sigma_rel": 0.5},
              {"op": "DZ", "type": "bounds", "lo": 0.0, "hi": 1e300}],
        opts=dict(max_iter=50, cg_iters=5, adapt=0, rho0=1.0, gamma0=1.5)),
    "small_grid_blur_data_fit": dict(
        grid={"n": [9, 7]},
        model=dict(kind="grf", n=[9, 7], seed=72),
        sets=[{"op": "BLUR", "axis": "x", "taps": [0.4, 0.2, 0.1], "type": "bounds", "lo": 2.6, "hi": 3.4},
              {"op": "I", "type": "bounds", "lo": 1.5, "hi": 4.5}],
        opts=dict(max_iter=40, cg_iters=5, adapt=0, rho0=1.0, gamma0=1.5)),
}


def model(spec):
    if spec["kind"] == "layered":
        return W.layered(tuple(spec["n"]), n_layers=spec["n_layers"], seed=spec["seed"])
    return W.grf(tuple(spec["n"]), seed=spec["seed"])


def compute(case):
    res = P.parsdmm(model(case["model"]), case["grid"], case["sets"], P.options(**case["opts"]))
    return {"x": [float(v) for v in res["x"]], "rho": [float(v) for v in res["rho"]],
            "cg_steps": int(res["cg_steps"])}


def main():
    for name, case in CASES.items():
        out = dict(case=case, result=compute(case))
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
