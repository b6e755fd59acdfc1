"""Parallel Dykstra baseline (Appendix A) through the C ABI: sweeps of
per-set projections, each computed by single-set PARSDMM iterations (the
paper's sub-problem solver), against the oracle's Algorithm
Parallel-DYKSTRA with the oracle's single-set PARSDMM as the projectors."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import operators as O                 # noqa: E402
from oracle import parsdmm as P                   # noqa: E402
from oracle.dykstra import parallel_dykstra       # noqa: E402
from paper_1902_09699_gb300 import sip            # noqa: E402
from paper_1902_09699_gb300 import workloads as W  # noqa: E402

TD = {"f64": torch.float64, "f32": torch.float32}


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def problem(n=(24, 20), seed=8):
    """The paper's first comparison set list: bounds, anisotropic TV l1
    ball, vertical monotonicity (absolute radius from the model)."""
    grid = {"n": n}
    m = W.grf(n, seed=seed)
    tv = float(np.abs(O.apply(grid, "TV", m)).sum())
    sets = [{"op": "I", "type": "bounds", "lo": 2.2, "hi": 3.8},
            {"op": "TV", "type": "l1", "sigma": 0.5 * tv},
            {"op": "DZ", "type": "bounds", "lo": 0.0, "hi": math.inf}]
    return grid, m, sets


@pytest.mark.parametrize("dt,bar", [("f64", 1e-10), ("f32", 1e-4)])
def test_dykstra_matches_oracle(dt, bar):
    grid, m, sets = problem()
    if dt == "f32":
        m = torch.as_tensor(m, dtype=torch.float32).double().numpy()
    inner = dict(max_iter=30, cg_iters=5, adapt=0, rho0=1.0, gamma0=1.0)
    projs = [lambda v, s=s: P.parsdmm(v, grid, [s], P.options(**inner))["x"] for s in sets]
    ref = parallel_dykstra(m, projs, 4)
    dk = sip.Dykstra(grid, sets, dtype=dt, **inner)
    x, info = dk.project(torch.as_tensor(m, dtype=TD[dt], device="cuda"), 4)
    dk.close()
    assert rel(x.double().cpu().numpy(), ref) <= bar
    assert info["sweeps"] == 4
    assert info["l1_projections"] == 4 * 30
    assert 0 < info["cg_steps"] <= 4 * 30 * 5


def test_dykstra_and_parsdmm_reach_the_same_projection():
    """Convex intersection: both methods approach its unique projection, and
    Dykstra's error shrinks with the sweeps."""
    grid, m, sets = problem((20, 16), seed=9)
    pr = sip.Projector(grid, sets, dtype="f64", max_iter=4000, adapt=1, gamma0=1.5)
    x_pd, _ = pr.project(torch.as_tensor(m, device="cuda"))
    pr.close()
    dk = sip.Dykstra(grid, sets, dtype="f64", max_iter=300, cg_iters=5, adapt=1, gamma0=1.5)
    err = []
    for sweeps in (20, 200):
        x_dk, _ = dk.project(torch.as_tensor(m, device="cuda"), sweeps)
        err.append(rel(x_dk.cpu().numpy(), x_pd.cpu().numpy()))
    dk.close()
    assert err[1] < err[0] and err[1] < 2e-2, err


def test_dykstra_rejects_relative_radii():
    grid, m, sets = problem()
    with pytest.raises(sip.SipError):
        sip.Dykstra(grid, [{"op": "TV", "type": "l1", "sigma_rel": 0.5}], dtype="f64")
