"""The annulus set and per-line sets (every column, row or fiber of A x on
its own) through the C ABI, against the FP64 oracle.

Bars as in the loop parity tests: 1e-10 in FP64 (the GPU's own
adapt-rho-gamma), 1e-4 in FP32 (fixed rho: no threshold decision can flip
on one-ulp differences).  Per-line card sets keep the k largest entries of
each line by per-thread lists for k <= 8 and by a radix selection in shared
memory above; per-line l1 sets sort each line in shared memory; lines longer
than SIP_MAX_LINE are rejected.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import parsdmm as P                   # noqa: E402
from paper_1902_09699_gb300 import sip            # noqa: E402
from paper_1902_09699_gb300 import workloads as W  # noqa: E402

TD = {"f64": torch.float64, "f32": torch.float32}


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run_gpu(m, grid, sets, dt, opts):
    pr = sip.Projector(grid, sets, dtype=dt, **opts)
    x, info = pr.project(torch.as_tensor(m, dtype=TD[dt], device="cuda"))
    out = x.double().cpu().numpy(), info
    pr.close()
    return out


def model(n, seed):
    return W.layered(n, n_layers=6, seed=seed)


BOUNDS = {"op": "I", "type": "bounds", "lo": 1.5, "hi": 4.5}

LINE_CASES = {
    # the paper's per-row / per-column cardinality of D_x / D_z
    "card-dz-columns": ({"op": "DZ", "type": "card", "k": 3, "scope": "z"}, (48, 36)),
    "card-dx-rows": ({"op": "DX", "type": "card", "k": 2, "scope": "x"}, (48, 36)),
    "card-frac-columns": ({"op": "DZ", "type": "card", "k_frac": 0.1, "scope": "z"}, (40, 30)),
    # k above the per-thread top-k path's limit: the radix selection per line
    "card-dz-columns-k12": ({"op": "DZ", "type": "card", "k": 12, "scope": "z"}, (48, 36)),
    "card-frac-rows-large": ({"op": "DX", "type": "card", "k_frac": 0.3, "scope": "x"}, (40, 30)),
    "l2-columns": ({"op": "I", "type": "l2", "sigma": 18.0, "scope": "z"}, (48, 36)),
    "l1-rows": ({"op": "DX", "type": "l1", "sigma": 0.6, "scope": "x"}, (48, 36)),
    "annulus-rows": ({"op": "I", "type": "annulus", "lo": 11.0, "hi": 13.0, "scope": "x"}, (48, 36)),
    "card-dy-fibers": ({"op": "DY", "type": "card", "k": 2, "scope": "y"}, (12, 10, 9)),
    "l2-columns-3d": ({"op": "DX", "type": "l2", "sigma": 0.4, "scope": "z"}, (12, 10, 9)),
}


@pytest.mark.parametrize("name", sorted(LINE_CASES))
def test_per_line_set_fp64_matches_oracle(name):
    s, n = LINE_CASES[name]
    m = model(n, 3) if len(n) == 2 else W.grf(n, seed=3)
    grid = {"n": n}
    sets = [BOUNDS, s]
    opts = dict(max_iter=40, cg_iters=5, adapt=1, rho0=1.0, gamma0=1.5)
    ref = P.parsdmm(m, grid, sets, P.options(**opts))
    x, info = run_gpu(m, grid, sets, "f64", opts)
    assert rel(x, ref["x"]) <= 1e-10
    for a, b in zip(info["r_feas"], ref["r_feas"]):
        assert a == pytest.approx(b, rel=1e-8, abs=1e-13)


@pytest.mark.parametrize("name", ["card-dz-columns", "l1-rows", "annulus-rows", "l2-columns-3d"])
def test_per_line_set_fp32(name):
    s, n = LINE_CASES[name]
    m = model(n, 4) if len(n) == 2 else W.grf(n, seed=4)
    m32 = torch.as_tensor(m, dtype=torch.float32).double().numpy()
    grid = {"n": n}
    sets = [BOUNDS, s]
    opts = dict(max_iter=30, cg_iters=5, adapt=0, rho0=1.0, gamma0=1.5)
    ref = P.parsdmm(m32, grid, sets, P.options(**opts))
    x, _ = run_gpu(m32, grid, sets, "f32", opts)
    assert rel(x, ref["x"]) <= 1e-4


@pytest.mark.parametrize("dt,bar", [("f64", 1e-10), ("f32", 1e-4)])
def test_annulus_whole_set(dt, bar):
    n = (40, 32)
    m = model(n, 5)
    if dt == "f32":
        m = torch.as_tensor(m, dtype=torch.float32).double().numpy()
    grid = {"n": n}
    nrm = float(np.linalg.norm(m))
    sets = [{"op": "I", "type": "annulus", "lo": 1.05 * nrm, "hi": 1.2 * nrm},
            {"op": "DZ", "type": "bounds", "lo": -0.2, "hi": 0.4}]
    opts = dict(max_iter=40, cg_iters=5, adapt=1 if dt == "f64" else 0, rho0=1.0, gamma0=1.5)
    ref = P.parsdmm(m, grid, sets, P.options(**opts))
    x, info = run_gpu(m, grid, sets, dt, opts)
    assert rel(x, ref["x"]) <= bar
    if dt == "f64":
        for a, b in zip(info["r_feas"], ref["r_feas"]):
            assert a == pytest.approx(b, rel=1e-8, abs=1e-13)


def test_short_and_degenerate_lines():
    """Lines of one entry (D_z on n_z = 2), k >= line length, k = 0."""
    m = W.grf((2, 30), seed=6)
    grid = {"n": (2, 30)}
    for s in ({"op": "DZ", "type": "card", "k": 1, "scope": "z"},
              {"op": "DZ", "type": "card", "k": 0, "scope": "z"},
              {"op": "DX", "type": "card", "k": 40, "scope": "x"},
              {"op": "DX", "type": "l1", "sigma": 0.0, "scope": "x"}):
        sets = [BOUNDS, s]
        opts = dict(max_iter=20, cg_iters=5, adapt=0, rho0=1.0, gamma0=1.5)
        ref = P.parsdmm(m, grid, sets, P.options(**opts))
        x, _ = run_gpu(m, grid, sets, "f64", opts)
        assert rel(x, ref["x"]) <= 1e-10, s


def test_line_limits_rejected():
    with pytest.raises(sip.SipError):
        sip.Projector({"n": (4097, 3)}, [{"op": "I", "type": "card", "k": 3, "scope": "z"}], dtype="f64")
    with pytest.raises(sip.SipError):
        sip.Projector({"n": (8, 8)}, [{"op": "TV", "type": "l1", "sigma": 1.0, "scope": "z"}], dtype="f64")
    with pytest.raises(sip.SipError):
        sip.Projector({"n": (8, 8)}, [{"op": "I", "type": "l2", "sigma_rel": 0.5, "scope": "x"}], dtype="f64")
    with pytest.raises(sip.SipError):
        sip.Projector({"n": (8, 8)}, [{"op": "I", "type": "annulus", "lo": 2.0, "hi": 1.0}], dtype="f64")
    # l2 lines have no length limit
    pr = sip.Projector({"n": (5000, 2)}, [{"op": "I", "type": "l2", "sigma": 1.0, "scope": "z"}], dtype="f32")
    pr.close()


# ---------------------------------------------------------------- point-wise data fit
def _inpainting(n=(48, 40), seed=21, frac=0.4):
    """Observed entries of a layered model under a random mask, with noise;
    the data-fit set {-0.05 <= M x - d <= 0.05} (M the mask) as per-entry
    bounds d +- 0.05 on observed entries and +-inf elsewhere."""
    g = np.random.default_rng(seed)
    truth = model(n, seed)
    obs = g.uniform(size=truth.size) < frac
    d = truth + 0.02 * g.standard_normal(truth.size)
    lo = np.where(obs, d - 0.05, -math.inf)
    hi = np.where(obs, d + 0.05, math.inf)
    m = np.where(obs, d, float(d[obs].mean()))
    grid = {"n": n}
    tv = float(np.abs(O_apply(grid, "TV", truth)).sum())
    sets = [{"op": "I", "type": "bounds", "lo": lo, "hi": hi},
            {"op": "TV", "type": "l1", "sigma": tv},
            {"op": "I", "type": "bounds", "lo": 1.5, "hi": 4.5}]
    return grid, m, sets, obs, d


def O_apply(grid, op, x):
    from oracle import operators as O
    return O.apply(grid, op, x)


@pytest.mark.parametrize("dt,bar", [("f64", 1e-10), ("f32", 1e-4)])
def test_data_fit_inpainting(dt, bar):
    grid, m, sets, obs, d = _inpainting()
    if dt == "f32":
        m = torch.as_tensor(m, dtype=torch.float32).double().numpy()
    opts = dict(max_iter=60, cg_iters=5, adapt=1 if dt == "f64" else 0, rho0=1.0, gamma0=1.5)
    ref = P.parsdmm(m, grid, sets, P.options(**opts))
    x, info = run_gpu(m, grid, sets, dt, opts)
    assert rel(x, ref["x"]) <= bar
    if dt == "f64":
        for a, b in zip(info["r_feas"], ref["r_feas"]):
            assert a == pytest.approx(b, rel=1e-8, abs=1e-13)


def test_data_fit_on_a_derivative_and_equalities():
    """Per-entry bounds on D_z x (some entries pinned: lo = hi) and a
    desaturation-style identity data fit with clipped ranges."""
    n = (32, 24)
    grid = {"n": n}
    g = np.random.default_rng(22)
    m = model(n, 22)
    Mz = (n[0] - 1) * n[1]
    lo = g.uniform(-0.3, 0.0, Mz)
    hi = lo + g.uniform(0.0, 0.4, Mz)
    hi[::7] = lo[::7]
    d = np.clip(m, 2.0, 3.5)
    lo_x = np.where(d <= 2.0, -math.inf, np.where(d >= 3.5, 3.5, d))
    hi_x = np.where(d <= 2.0, 2.0, np.where(d >= 3.5, math.inf, d))
    sets = [{"op": "DZ", "type": "bounds", "lo": lo, "hi": hi},
            {"op": "I", "type": "bounds", "lo": lo_x, "hi": hi_x}]
    opts = dict(max_iter=50, cg_iters=5, adapt=1, rho0=1.0, gamma0=1.5)
    ref = P.parsdmm(m, grid, sets, P.options(**opts))
    x, _ = run_gpu(m, grid, sets, "f64", opts)
    assert rel(x, ref["x"]) <= 1e-10


def test_data_fit_vectors_validated():
    with pytest.raises(sip.SipError):   # lo > hi at one entry
        sip.Projector({"n": (4, 4)}, [{"op": "I", "type": "bounds", "lo": np.r_[np.zeros(15), 2.0], "hi": 1.0}],
                      dtype="f64")
    with pytest.raises(sip.SipError):   # vectors only for bounds
        sip.Projector({"n": (4, 4)}, [{"op": "I", "type": "l2", "sigma": 1.0, "lo": np.zeros(16)}], dtype="f64")


@pytest.mark.parametrize("dt,bar", [("f64", 1e-10), ("f32", 1e-4)])
def test_l2_data_fit_ball(dt, bar):
    """{||M (x - d)|| <= sigma} (noise-level radius) with TV and bounds:
    the l2 data-fit formulation of the paper with a mask (NaN centers)."""
    g = np.random.default_rng(23)
    n = (40, 36)
    truth = model(n, 23)
    d = truth + 0.05 * g.standard_normal(truth.size)
    obs = g.uniform(size=truth.size) < 0.5
    d[~obs] = np.nan
    sigma = 0.05 * math.sqrt(obs.sum())
    m = np.where(obs, d, 3.0)
    if dt == "f32":
        m = torch.as_tensor(m, dtype=torch.float32).double().numpy()
    grid = {"n": n}
    tv = float(np.abs(O_apply(grid, "TV", truth)).sum())
    sets = [{"op": "I", "type": "l2", "sigma": sigma, "center": d},
            {"op": "TV", "type": "l1", "sigma": tv},
            {"op": "I", "type": "bounds", "lo": 1.5, "hi": 4.5}]
    opts = dict(max_iter=60, cg_iters=5, adapt=1 if dt == "f64" else 0, rho0=1.0, gamma0=1.5)
    ref = P.parsdmm(m, grid, sets, P.options(**opts))
    x, info = run_gpu(m, grid, sets, dt, opts)
    assert rel(x, ref["x"]) <= bar
    if dt == "f64":
        # the ball's r_feas is ||s - d|| - sigma over ||s||: a difference of
        # nearly equal numbers, so rounding is amplified by their ratio
        for a, b in zip(info["r_feas"], ref["r_feas"]):
            assert a == pytest.approx(b, rel=1e-6, abs=1e-13)


def test_l2_data_fit_validated():
    with pytest.raises(sip.SipError):   # a center needs an l2 set
        sip.Projector({"n": (4, 4)}, [{"op": "I", "type": "l1", "sigma": 1.0, "center": np.zeros(16)}], dtype="f64")
    with pytest.raises(sip.SipError):   # and an absolute radius
        sip.Projector({"n": (4, 4)}, [{"op": "I", "type": "l2", "sigma_rel": 0.5, "center": np.zeros(16)}],
                      dtype="f64")
