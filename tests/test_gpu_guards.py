"""The debug build with device index guards (libsip_guarded.so, SIP_GUARDS=1).

Every kernel of that build checks its work item against its array (grid
points, segment rows, selection jobs, final-pass and per-line blocks) and the
x indices the set pass gathers; a failed check records SIP_ERR_INTERNAL, the
check and the index in the plan's error word and skips the access, and the
call returns SIP_ERR_INTERNAL.  This test runs the guarded build in a fresh
process over projections that reach every guarded kernel (2D and 3D, FP32
and FP64, selections, ties, per-line sets, a batch, multilevel) and checks
that no guard fires and the results still match the oracle.  No test plants
a bad index on the GPU.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import os, sys
import numpy as np, torch
sys.path.insert(0, %(root)r)
from paper_1902_09699_gb300 import sip, workloads as W
from oracle import parsdmm as P
assert sip.LIB_PATH.endswith("libsip_guarded.so"), sip.LIB_PATH
def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
cases = []
c = W.layered_2d(n=(96, 128), seed=77)
cases.append((c["grid"], c["sets"], dict(c["opts"], max_iter=40), "f64", {}))
cases.append((c["grid"], [s_ for s_ in c["sets"] if s_["type"] != "card"], dict(c["opts"], max_iter=40), "f32", {}))
g3 = W.grf_3d(n=(24, 20, 12), seed=5)
cases.append((g3["grid"], g3["sets"], dict(g3["opts"], max_iter=30), "f64", {}))
cases.append((g3["grid"], g3["sets"], dict(g3["opts"], max_iter=20, levels=2, coarse_iter=10), "f64", {}))
s2 = W.small_2d(n=(40, 36), seed=3)
lines = [s2["sets"][0], {"op": "DZ", "type": "card", "k": 3, "scope": "z"}, {"op": "DX", "type": "l1", "sigma": 0.5, "scope": "x"}]
cases.append((s2["grid"], lines, dict(s2["opts"], max_iter=30), "f64", {}))
for grid, sets, opts, dt, kw in cases:
    pr = sip.Projector(grid, sets, dtype=dt, **opts)
    m = torch.as_tensor(W.grf(grid["n"], seed=9) if "levels" not in opts else g3["m"], device="cuda",
                        dtype=torch.float64 if dt == "f64" else torch.float32)
    x, info = pr.project(m)
    pr.close()
    o = {k: v for k, v in opts.items() if k not in ("levels", "coarse_iter")}
    mm = m.double().cpu().numpy()
    ref = P.ml_parsdmm(mm, grid, sets, P.options(**o), levels=opts["levels"], coarse_iter=opts["coarse_iter"]) \
        if "levels" in opts else P.parsdmm(mm, grid, sets, P.options(**o))
    e = rel(x.double().cpu().numpy(), ref["x"])
    assert e <= (1e-10 if dt == "f64" else 1e-2), (grid, dt, e)
rb = W.ragged_batch(count=4, lo=16, hi=40, seed=5)
bp = sip.BatchProjector([(it["grid"], it["sets"]) for it in rb["instances"]], dtype="f64",
                        **dict(rb["opts"], max_iter=20))
xs, infos = bp.project([it["m"] for it in rb["instances"]])
bp.close()
print("guarded ok", len(cases) + 1)
'''


def test_guarded_build_runs_clean():
    from paper_1902_09699_gb300 import build
    if not os.path.exists(build.OUT_GUARDED):
        build.build(guarded=True)
    env = dict(os.environ, SIP_GUARDS="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT % {"root": ROOT}], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "guarded ok" in r.stdout
