"""Single-step parity: each CUDA step against the FP64 oracle on identical
inputs, through the C ABI.

Tolerances: stencils and the system matrix differ from the oracle only in
rounding order (a few ulp): 1e-13 relative in FP64, 2e-6 in FP32.  Clip and
cardinality are decided exactly on identical inputs: bit-exact.  The l1
threshold: 1e-12 relative (FP64 running sums in both precisions, so FP32 is
held to 1e-12 relative to the FP32 inputs' exact values as well).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import operators as O          # noqa: E402
from oracle import parsdmm as P            # noqa: E402
from oracle import prox as X               # noqa: E402
from paper_1902_09699_gb300 import sip     # noqa: E402

TOL = {"f64": 1e-13, "f32": 2e-6}
EPS64 = np.finfo(np.float64).eps
TD = {"f64": torch.float64, "f32": torch.float32}

GRIDS = [
    {"n": (7, 5), "h": (1.0, 1.0)},
    {"n": (64, 64), "h": (1.0, 1.0)},
    {"n": (300, 37), "h": (0.5, 2.0)},          # ragged tails, non-unit spacing
    {"n": (9, 6, 5), "h": (1.0, 1.0, 1.0)},
    {"n": (33, 17, 9), "h": (1.0, 0.5, 2.0)},
]


def cuda(a, dt):
    return torch.as_tensor(np.asarray(a), dtype=TD[dt], device="cuda")


def host(t):
    return t.double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("gi", range(len(GRIDS)))
@pytest.mark.parametrize("op", ["I", "DZ", "DX", "DY", "TV"])
def test_operator_and_adjoint(dt, gi, op):
    grid = GRIDS[gi]
    if op == "DY" and len(grid["n"]) == 2:
        pytest.skip("2D")
    g = np.random.default_rng(gi)
    x = g.standard_normal(O.grid_size(grid))
    xin = host(cuda(x, dt))                 # the exact values the GPU sees
    s = sip.apply_op(grid, op, cuda(xin, dt))
    assert rel(host(s), O.apply(grid, op, xin)) <= TOL[dt]
    y = host(cuda(g.standard_normal(O.out_size(grid, op)), dt))
    xt = sip.apply_op_t(grid, op, cuda(y, dt))
    assert rel(host(xt), O.apply_t(grid, op, y)) <= 4 * TOL[dt]


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("gi", range(len(GRIDS)))
def test_system_matrix(dt, gi):
    grid = GRIDS[gi]
    ops = ["I", "TV", "DZ", "DX"] + (["DY"] if len(grid["n"]) == 3 else [])
    rhos = [0.7, 1.3, 2.1, 0.4, 3.0][:len(ops)]
    x = host(cuda(np.random.default_rng(10 + gi).standard_normal(O.grid_size(grid)), dt))
    out = sip.system_apply(grid, ops, rhos, 1.25, cuda(x, dt))
    assert rel(host(out), O.system_apply(grid, ops, rhos, 1.25, x)) <= 8 * TOL[dt]


SIZES = [1, 2, 31, 1000, 1024, 1025, 4097, 300001]


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("n", SIZES)
def test_bounds_and_l2(dt, n):
    g = np.random.default_rng(n)
    w = host(cuda(g.standard_normal(n) * 3, dt))
    y, _ = sip.project_set({"type": "bounds", "lo": -0.5, "hi": 1.25}, cuda(w, dt))
    assert np.array_equal(host(y), host(cuda(X.proj_bounds(w, -0.5, 1.25), dt)))
    y, _ = sip.project_set({"type": "bounds", "lo": 0.0, "hi": math.inf}, cuda(w, dt))
    assert np.array_equal(host(y), np.maximum(w, 0.0))
    for frac in (0.3, 2.0):
        sigma = frac * np.linalg.norm(w)
        y, scale = sip.project_set({"type": "l2", "sigma": sigma}, cuda(w, dt))
        assert rel(host(y), X.proj_l2(w, sigma)) <= TOL[dt]


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("n", SIZES)
def test_l1_ball_threshold(dt, n):
    g = np.random.default_rng(100 + n)
    w = host(cuda(g.standard_normal(n) * g.uniform(0.1, 10.0), dt))
    for frac in (0.0, 1e-4, 0.05, 0.5, 0.999, 1.0, 1.5):
        tau = frac * float(np.abs(w).sum())
        y, theta = sip.project_set({"type": "l1", "sigma": tau}, cuda(w, dt))
        ref = X.proj_l1(w, tau)
        if 0.0 < frac < 1.0:
            th_ref = X.l1_threshold(w, tau)
            # theta = (S - tau) / c with S the sum of the c entries above it:
            # both sides sum S in binary64 in different orders, so they may
            # differ by the recursive-summation bound 2 (n - 1) eps S / c
            a = np.abs(w)
            c = int(np.sum(a > th_ref))
            bound = 2 * max(n - 1, 1) * np.finfo(np.float64).eps * float(a[a > th_ref].sum()) / max(c, 1)
            assert abs(theta - th_ref) <= max(bound, 1e-15 * th_ref)
        if dt == "f64":
            assert np.allclose(host(y), ref, rtol=0, atol=1e-12 * max(np.abs(w).max(), 1e-300))
        else:  # y = sign(w) max(|w| - theta, 0) evaluated in binary32
            assert np.allclose(host(y), ref, rtol=0, atol=2e-6 * max(np.abs(w).max(), 1e-300))
        if dt == "f64":  # support identical (entries above theta)
            assert np.array_equal(host(y) != 0, ref != 0)


def test_l1_ball_with_ties_and_zeros():
    w = np.array([0.0, 2.0, -2.0, 2.0, 0.0, 1.0, -1.0, 0.5] * 400)
    for dt in ("f64", "f32"):
        for tau in (1.0, 100.0, 1500.0, 2500.0):
            y, theta = sip.project_set({"type": "l1", "sigma": tau}, cuda(w, dt))
            assert np.allclose(host(y), X.proj_l1(w, tau), atol=1e-5)


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("n", SIZES)
def test_cardinality_support_bit_exact(dt, n):
    g = np.random.default_rng(200 + n)
    w = host(cuda(g.standard_normal(n), dt))
    for k in sorted({0, 1, max(n // 50, 1), n // 2, n - 1, n, n + 5}):
        if k < 0:
            continue
        y, _ = sip.project_set({"type": "card", "k": k}, cuda(w, dt))
        assert np.array_equal(host(y), X.proj_card(w, k)), (n, k)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_cardinality_tie_rule(dt):
    # many exact ties at the k-th magnitude, spread over several tiles
    g = np.random.default_rng(5)
    n = 20000
    w = g.choice([0.25, -0.25, 0.5, -1.0, 0.0], size=n, p=[0.3, 0.3, 0.2, 0.1, 0.1])
    for k in (1, 1999, 2000, 2001, 5000, 9000, 15000, 19999):
        y, _ = sip.project_set({"type": "card", "k": k}, cuda(w, dt))
        assert np.array_equal(host(y), X.proj_card(w, k)), k


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("gi", range(len(GRIDS)))
def test_norms_for_relative_radii(dt, gi):
    grid = GRIDS[gi]
    m = host(cuda(np.random.default_rng(gi).standard_normal(O.grid_size(grid)) + 3, dt))
    for op, t in (("TV", "l1"), ("DX", "l2"), ("I", "l1"), ("DZ", "l2")):
        got = sip.op_norm(grid, op, t, cuda(m, dt))
        # FP32 differences are rounded to binary32 before the binary64 sum
        assert got == pytest.approx(O.norm_of(grid, op, t, m), rel=1e-12 if dt == "f64" else 1e-6)


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("grid", [{"n": (16, 12), "h": (1.0, 1.0)}, {"n": (17, 9), "h": (1.0, 2.0)},
                                  {"n": (8, 6, 6), "h": (1.0, 1.0, 1.0)}, {"n": (12, 10, 7), "h": (1.0, 1.0, 1.0)}])
def test_restrict_and_prolong(dt, grid):
    g = np.random.default_rng(3)
    m = host(cuda(g.standard_normal(O.grid_size(grid)), dt))
    mc = sip.restrict(grid, cuda(m, dt))
    assert rel(host(mc), P.restrict(grid, m)) <= TOL[dt]
    gc = P.coarse_grid(grid)
    ops = ["I", "DZ", "DX", "TV"] + (["DY"] if len(grid["n"]) == 3 else [])
    for op in ops:
        uc = host(cuda(g.standard_normal(O.out_size(gc, op)), dt))
        uf = sip.prolong(grid, op, cuda(uc, dt))
        assert rel(host(uf), P.prolong(gc, grid, op, uc)) <= 4 * TOL[dt], op
