"""Warm-started window selection of the cardinality sets' top-k.

The projection onto {card(A x) <= k} keeps the k entries of largest
magnitude (Sec. Notation); the library finds the k-th magnitude either by
radix passes over all entries or, when the k-th value of the previous
iteration predicts a window that holds the new one, from the window's
candidates alone.  Both give the same key, so with deterministic sums
(fixed rho: no binary64 atomics on the x path) the results are bitwise
equal with the window on and off; the window path must actually be taken
(hits counted) and must handle ties at the k-th value.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import parsdmm as P                   # noqa: E402
from paper_1902_09699_gb300 import sip            # noqa: E402
from paper_1902_09699_gb300 import workloads as W  # noqa: E402

TD = {"f64": torch.float64, "f32": torch.float32}

CARD_SETS = [
    {"op": "I", "type": "bounds", "lo": 1.5, "hi": 4.5},
    {"op": "DZ", "type": "card", "k_frac": 0.03},
    {"op": "DX", "type": "card", "k_frac": 0.05},
    {"op": "TV", "type": "card", "k_frac": 0.04},
    {"op": "DZ", "type": "bounds", "lo": -0.2, "hi": 0.6},
]


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run(m, grid, sets, dt, **opts):
    pr = sip.Projector(grid, sets, dtype=dt, **opts)
    x, info = pr.project(torch.as_tensor(m, dtype=TD[dt], device="cuda"))
    out = x.cpu().numpy(), info
    pr.close()
    return out


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("mode", ["graph", "persistent"])
def test_window_equals_radix(dt, mode):
    n = (80, 120)
    m = W.layered(n, seed=5)
    grid = {"n": n}
    opts = dict(max_iter=80, cg_iters=5, adapt=0, rho0=1.0, gamma0=1.5, exec=mode)
    x1, i1 = run(m, grid, CARD_SETS, dt, select_window=1, **opts)
    x0, i0 = run(m, grid, CARD_SETS, dt, select_window=0, **opts)
    assert i0["window_hits"] == 0
    # three card sets over 80 iterations: most selections come from the window
    assert i1["window_hits"] >= 120, i1["window_hits"]
    assert np.array_equal(x1, x0)


def test_window_matches_oracle_fp64():
    n = (64, 96)
    m = W.layered(n, seed=9)
    grid = {"n": n}
    opts = dict(max_iter=60, cg_iters=5, adapt=0, rho0=1.0, gamma0=1.5)
    ref = P.parsdmm(m, grid, CARD_SETS, P.options(**opts))
    x, info = run(m, grid, CARD_SETS, "f64", **opts)
    assert info["window_hits"] > 0
    assert rel(x, ref["x"]) <= 1e-10


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_window_ties_at_kth_value(dt):
    """A laterally invariant model with only I and D_z sets stays laterally
    invariant, so every |D_z x| value occurs n_x times and a k that is not a
    multiple of n_x cuts through a tie at the k-th value."""
    nz, nx = 48, 40
    col = W.layered((nz, 1), n_layers=8, noise=0.0, blob_amp=0.0, seed=3)
    m = np.tile(col, nx)
    grid = {"n": (nz, nx)}
    sets = [{"op": "I", "type": "bounds", "lo": 1.8, "hi": 4.2},
            {"op": "DZ", "type": "card", "k": 5 * nx + 17}]
    opts = dict(max_iter=50, cg_iters=5, adapt=0, rho0=1.0, gamma0=1.5)
    x1, i1 = run(m, grid, sets, dt, select_window=1, **opts)
    x0, i0 = run(m, grid, sets, dt, select_window=0, **opts)
    assert i1["window_hits"] > 0
    assert np.array_equal(x1, x0)
    if dt == "f64":
        ref = P.parsdmm(m, grid, sets, P.options(**opts))
        assert rel(x1, ref["x"]) <= 1e-10


def test_window_in_a_batch():
    g = np.random.default_rng(4)
    inst = [({"n": (40, 33)}, CARD_SETS),
            ({"n": (130, 3)}, [{"op": "DZ", "type": "card", "k_frac": 0.05},
                               {"op": "I", "type": "l2", "sigma_rel": 0.6}]),
            ({"n": (25, 25)}, [{"op": "TV", "type": "l1", "sigma_rel": 0.2}]),
            ({"n": (64, 20)}, CARD_SETS[:3])]
    models = [W.layered(gr["n"], n_layers=6, seed=20 + i) + 0.05 * g.standard_normal(int(np.prod(gr["n"])))
              for i, (gr, _) in enumerate(inst)]
    opts = dict(max_iter=50, adapt=0, rho0=1.0, gamma0=1.5)
    out = {}
    for sw in (1, 0):
        bp = sip.BatchProjector(inst, dtype="f64", select_window=sw, **opts)
        xs, infos = bp.project(models)
        out[sw] = ([x.cpu().numpy() for x in xs], infos)
        bp.close()
    for i in range(len(inst)):
        if i in (0, 3):  # bounds and card sets only: no binary64 atomics
            assert np.array_equal(out[1][0][i], out[0][0][i]), i
        else:             # l1 / l2 norms: equal up to the atomics' rounding order
            assert rel(out[1][0][i], out[0][0][i]) <= 1e-12, i
        assert out[0][1][i]["window_hits"] == 0
    assert out[1][1][0]["window_hits"] > 0 and out[1][1][3]["window_hits"] > 0
    assert out[1][1][2]["window_hits"] == 0  # no card set
    for i, ((grid, sets), m) in enumerate(zip(inst, models)):
        ref = P.parsdmm(m, grid, sets, P.options(**opts))
        assert rel(out[1][0][i], ref["x"]) <= 1e-10, i
