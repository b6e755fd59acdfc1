"""Pins for oracle/parsdmm.py: CG, adapt-rho-gamma, stopping quantities, the
PARSDMM fixed point and ML-PARSDMM.

What fixes the answers (none of it re-runs the oracle's own formulas):
* CG: a dense solve of the explicit system matrix (Eq. sys_mat).
* PARSDMM: the projection problem itself (Eq. proj_intersect) -- closed-form
  projections for single sets, column-wise isotonic regression (pool
  adjacent violators) for vertical monotonicity, parallel Dykstra
  (Appendix A) on convex intersections, a general-purpose constrained
  solver (SLSQP) on tiny grids, and the KKT conditions of the Lagrangian
  (Eq. aug_lag).
* adapt-rho-gamma: inputs built so each of the four cases of the algorithm's
  table is hit with known spectral step sizes.
* ML: exactness of restriction / prolongation on linear fields.
"""
import math

import numpy as np
import pytest

from oracle import operators as ops
from oracle import parsdmm as P
from oracle import prox
from oracle.dykstra import parallel_dykstra


# ---------------------------------------------------------------- helpers
def pava_increasing(y):
    """Pool-adjacent-violators: least-squares non-decreasing fit (textbook
    isotonic regression)."""
    vals, wts = [], []
    for v in y:
        vals.append(float(v))
        wts.append(1.0)
        while len(vals) > 1 and vals[-2] > vals[-1]:
            w = wts[-2] + wts[-1]
            v2 = (vals[-2] * wts[-2] + vals[-1] * wts[-1]) / w
            vals[-2:] = [v2]
            wts[-2:] = [w]
    out = []
    for v, w in zip(vals, wts):
        out.extend([v] * int(round(w)))
    return np.array(out)


def proj_dz_nonneg(grid, x):
    """Projection onto {D_z x >= 0}: isotonic regression of every column."""
    nz = grid["n"][0]
    X = np.asarray(x).reshape(-1, nz)
    return np.vstack([pava_increasing(c) for c in X]).reshape(-1)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dense_C(grid, opsl, rhos, c_id):
    N = ops.grid_size(grid)
    return np.stack([ops.system_apply(grid, opsl, rhos, c_id, e) for e in np.eye(N)], axis=1)


# ---------------------------------------------------------------- CG
def test_cg_matches_dense_solve():
    grid = {"n": (6, 5), "h": (1.0, 1.0)}
    opsl, rhos = ["TV", "DZ", "I"], [1.3, 0.7, 2.0]
    C = dense_C(grid, opsl, rhos, 0.0)
    g = np.random.default_rng(0)
    b = g.standard_normal(30)
    x_ref = np.linalg.solve(C, b)
    apply_c = lambda z: ops.system_apply(grid, opsl, rhos, 0.0, z)
    x, steps = P.cg(apply_c, b, np.zeros(30), 200, 0)
    assert rel(x, x_ref) < 1e-10
    # Krylov: exact after at most N steps in exact arithmetic
    x, steps = P.cg(apply_c, b, g.standard_normal(30), 30, 0)
    assert rel(x, x_ref) < 1e-8


def test_cg_adaptive_stop_rule():
    grid = {"n": (8, 8), "h": (1.0, 1.0)}
    opsl, rhos = ["TV", "I"], [3.0, 1.0]
    apply_c = lambda z: ops.system_apply(grid, opsl, rhos, 0.0, z)
    g = np.random.default_rng(1)
    b = g.standard_normal(64)
    x0 = g.standard_normal(64)
    r0 = np.linalg.norm(b - apply_c(x0))
    x, steps = P.cg(apply_c, b, x0, 0, 100)
    assert np.linalg.norm(b - apply_c(x)) < 0.1 * r0 * (1 + 1e-9)
    x1, _ = P.cg(apply_c, b, x0, steps - 1, 0)
    assert np.linalg.norm(b - apply_c(x1)) >= 0.1 * r0 * (1 - 1e-9)
    # zero residual: no step
    xs = np.linalg.solve(dense_C(grid, opsl, rhos, 0.0), b)
    _, st = P.cg(apply_c, apply_c(xs), xs, 5, 0)
    assert st <= 1


# ---------------------------------------------------------------- adapt
def test_adapt_case_both_correlated():
    o = P.options(adapt=2)
    # dv-hat = 3 dh exactly (corr 1): MG = SD = 3 -> alpha = 3
    # dv = 12 dg exactly: beta = 12 -> rho = 6, gamma = 1 + 2*6/15
    dh = np.array([1.0, -2.0, 0.5]); dvh = 3 * dh
    dg = np.array([0.2, 0.1, -0.3]); dv = 12 * dg
    dots = (dh @ dvh, dh @ dh, dvh @ dvh, dg @ dv, dg @ dg, dv @ dv)
    r, gm, case = P.adapt_rho_gamma(dots, 1.0, 1.0, o)
    assert case == 1
    assert r == pytest.approx(6.0, rel=1e-14)
    assert gm == pytest.approx(1.0 + 2.0 * 6.0 / 15.0, rel=1e-14)


def test_adapt_case_alpha_only_uses_sd_branch():
    o = P.options(adapt=2)
    # dh = (1, 0), dvh = (1, 2): corr = 1/sqrt(5) > 0.3
    # MG = 1/1 = 1, SD = 5/1 = 5; 2 MG <= SD -> alpha = SD - MG/2 = 4.5
    dh = np.array([1.0, 0.0]); dvh = np.array([1.0, 2.0])
    dg = np.array([1.0, 0.0]); dv = np.array([0.0, 1.0])  # corr 0
    dots = (dh @ dvh, dh @ dh, dvh @ dvh, dg @ dv, dg @ dg, dv @ dv)
    r, gm, case = P.adapt_rho_gamma(dots, 1.0, 1.0, o)
    assert (case, r, gm) == (2, 4.5, 1.9)


def test_adapt_case_beta_only_and_neither():
    o = P.options(adapt=2)
    zero = (0.0, 0.0, 0.0)
    dg = np.array([2.0, 1.0]); dv = np.array([4.0, 2.0])  # MG = 2 = SD
    r, gm, case = P.adapt_rho_gamma(zero + (dg @ dv, dg @ dg, dv @ dv), 1.0, 1.0, o)
    assert (case, r, gm) == (3, 2.0, 1.1)
    r, gm, case = P.adapt_rho_gamma(zero + zero, 0.7, 1.3, o)
    assert (case, r, gm) == (4, 0.7, 1.5)
    # anti-correlated: negative correlation is "not > eps"
    dh = np.array([1.0, 0.0]); dvh = -dh
    r, gm, case = P.adapt_rho_gamma((dh @ dvh, 1.0, 1.0) + zero, 0.7, 1.3, o)
    assert case == 4


def test_adapt_gamma_stays_below_two_and_rho_only_mode():
    dh = np.array([1.0, 2.0]); dg = np.array([1.0, 1.0])
    dots = (dh @ (5 * dh), dh @ dh, 25 * dh @ dh, dg @ (5 * dg), dg @ dg, 25 * dg @ dg)
    r, gm, _ = P.adapt_rho_gamma(dots, 1.0, 1.0, P.options(adapt=2))
    assert r == pytest.approx(5.0) and gm == 1.99      # AM-GM equality gives 2
    r, gm, _ = P.adapt_rho_gamma(dots, 1.0, 1.5, P.options(adapt=1))
    assert r == pytest.approx(5.0) and gm == 1.5


# ---------------------------------------------------------------- stopping
def test_feasibility_and_evolution_closed_forms():
    s = np.array([3.0, 4.0])
    spec = {"type": "l2", "sigma": 1.0}
    # ||s - P(s)|| = ||s|| - sigma for the l2 ball
    assert P.feasibility(s, spec) == pytest.approx((5.0 - 1.0) / 5.0)
    assert P.feasibility(s, {"type": "bounds", "lo": 0.0, "hi": 10.0}) == 0.0
    x = np.array([1.0, 0.0])
    hist = [np.array([1.0, 0.5]), np.array([0.0, 0.0]), np.array([1.0, 0.1])]
    assert P.evolution(x, hist) == pytest.approx(1.0)


# ---------------------------------------------------------------- PARSDMM
GRID = {"n": (8, 6), "h": (1.0, 1.0)}


def model(grid, seed=0):
    n = ops.grid_size(grid)
    g = np.random.default_rng(seed)
    return 3.0 + g.standard_normal(n)


def run(m, grid, sets, iters=3000, **kw):
    o = P.options(max_iter=iters, adapt=1, gamma0=1.5, rho0=1.0)
    o.update(kw)
    return P.parsdmm(m, grid, sets, o)


def test_single_bounds_set_gives_clip():
    m = model(GRID)
    res = run(m, GRID, [{"op": "I", "type": "bounds", "lo": 2.5, "hi": 3.5}], iters=400)
    assert rel(res["x"], np.clip(m, 2.5, 3.5)) < 1e-8


def test_single_l2_set_gives_radial_scaling():
    m = model(GRID, 1)
    sigma = 0.5 * np.linalg.norm(m)
    res = run(m, GRID, [{"op": "I", "type": "l2", "sigma": sigma}], iters=400)
    assert rel(res["x"], m * sigma / np.linalg.norm(m)) < 1e-8


def test_single_l1_set_gives_soft_threshold():
    m = model(GRID, 2)
    tau = 0.4 * np.abs(m).sum()
    a = np.abs(m)
    lo, hi = 0.0, a.max()
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if np.maximum(a - mid, 0).sum() > tau else (lo, mid)
    expect = np.sign(m) * np.maximum(a - 0.5 * (lo + hi), 0)
    res = run(m, GRID, [{"op": "I", "type": "l1", "sigma": tau}], iters=600)
    assert rel(res["x"], expect) < 1e-7


def test_single_card_set_from_feasible_start_keeps_top_k():
    # non-convex: from x = y = m (feasible warm start) the loop must keep the
    # k largest entries (the projection for tie-free m)
    m = model(GRID, 3)
    k = 10
    expect = np.zeros_like(m)
    idx = np.argsort(-np.abs(m))[:k]
    expect[idx] = m[idx]
    o = P.options(max_iter=400, adapt=0, rho0=1.0, gamma0=1.0)
    init = (m.copy(), [expect.copy(), m.copy()], [np.zeros_like(m), np.zeros_like(m)])
    res = P.parsdmm(m, GRID, [{"op": "I", "type": "card", "k": k}], o, init=init)
    assert rel(res["x"], expect) < 1e-8


def test_vertical_monotonicity_is_isotonic_regression():
    m = model(GRID, 4)
    res = run(m, GRID, [{"op": "DZ", "type": "bounds", "lo": 0.0, "hi": math.inf}], iters=3000)
    assert rel(res["x"], proj_dz_nonneg(GRID, m)) < 1e-6


def test_convex_intersection_matches_parallel_dykstra():
    m = model(GRID, 5)
    sigma = 0.95 * np.linalg.norm(np.clip(m, 2.5, 3.7))
    projs = [lambda z: np.clip(z, 2.5, 3.7),
             lambda z: proj_dz_nonneg(GRID, z),
             lambda z: z if np.linalg.norm(z) <= sigma else z * sigma / np.linalg.norm(z)]
    ref = parallel_dykstra(m, projs, 200000, tol=1e-15)
    sets = [{"op": "I", "type": "bounds", "lo": 2.5, "hi": 3.7},
            {"op": "DZ", "type": "bounds", "lo": 0.0, "hi": math.inf},
            {"op": "I", "type": "l2", "sigma": sigma}]
    res = run(m, GRID, sets, iters=4000)
    assert rel(res["x"], ref) < 1e-5


def test_bounds_tv_monotone_matches_general_qp_solver():
    """The config-1 set list on a 5 x 4 grid against SLSQP on the QP
    min 1/2||x-m||^2 s.t. 2 <= x <= 4, ||TV x||_1 <= tau, D_z x >= 0,
    with the l1 constraint split as -t <= TV x <= t, sum t <= tau."""
    opt = pytest.importorskip("scipy.optimize")
    grid = {"n": (5, 4), "h": (1.0, 1.0)}
    N = ops.grid_size(grid)
    g = np.random.default_rng(8)
    m = 3.0 + 0.8 * g.standard_normal(N)
    T = np.stack([ops.apply(grid, "TV", e) for e in np.eye(N)], axis=1)
    Dz = np.stack([ops.apply(grid, "DZ", e) for e in np.eye(N)], axis=1)
    tau = 0.5 * np.abs(T @ m).sum()
    nt = T.shape[0]

    def f(z):
        return 0.5 * np.sum((z[:N] - m) ** 2)

    def fg(z):
        gr = np.zeros_like(z)
        gr[:N] = z[:N] - m
        return gr
    cons = [
        {"type": "ineq", "fun": lambda z: z[N:] - T @ z[:N], "jac": lambda z: np.hstack([-T, np.eye(nt)])},
        {"type": "ineq", "fun": lambda z: z[N:] + T @ z[:N], "jac": lambda z: np.hstack([T, np.eye(nt)])},
        {"type": "ineq", "fun": lambda z: np.array([tau - z[N:].sum()]),
         "jac": lambda z: np.hstack([np.zeros((1, N)), -np.ones((1, nt))])},
        {"type": "ineq", "fun": lambda z: Dz @ z[:N], "jac": lambda z: np.hstack([Dz, np.zeros((Dz.shape[0], nt))])},
    ]
    z0 = np.concatenate([np.full(N, 3.0), np.full(nt, tau / nt)])
    bnds = [(2.0, 4.0)] * N + [(0.0, None)] * nt
    sol = opt.minimize(f, z0, jac=fg, bounds=bnds, constraints=cons, method="SLSQP",
                       options={"maxiter": 2000, "ftol": 1e-13})
    assert sol.success
    sets = [{"op": "I", "type": "bounds", "lo": 2.0, "hi": 4.0},
            {"op": "TV", "type": "l1", "sigma": tau},
            {"op": "DZ", "type": "bounds", "lo": 0.0, "hi": math.inf}]
    res = run(m, grid, sets, iters=6000)
    assert rel(res["x"], sol.x[:N]) < 1e-5


def test_kkt_certificate_from_duals():
    """At the fixed point of the paper's form: x = m + sum_{i<=p} A_i^T v_i
    (stationarity of Eq. aug_lag with y_i = A_i x), and -v_i lies in the
    normal cone of C_i at A_i x."""
    m = model(GRID, 6)
    sets = [{"op": "I", "type": "bounds", "lo": 2.5, "hi": 3.5},
            {"op": "TV", "type": "l1", "sigma": 0.1 * ops.norm_of(GRID, "TV", "l1", m)},
            {"op": "DZ", "type": "bounds", "lo": 0.0, "hi": math.inf}]
    res = run(m, GRID, sets, iters=6000)
    # the l1 ball is active at the solution
    assert ops.norm_of(GRID, "TV", "l1", res["x"]) == pytest.approx(sets[1]["sigma"], rel=1e-5)
    x, v = res["x"], res["v"]
    recon = m + sum(ops.apply_t(GRID, s["op"], v[i]) for i, s in enumerate(sets))
    assert rel(recon, x) < 1e-6
    scale = np.abs(v[0]).max() + 1e-12
    s0 = x
    # bounds: v <= 0 at the upper bound, v >= 0 at the lower one, 0 inside
    inside = (s0 > 2.5 + 1e-6) & (s0 < 3.5 - 1e-6)
    assert np.abs(v[0][inside]).max(initial=0) < 1e-5 * scale + 1e-8
    # l1 ball: -v = lambda * sign(s) on the support with one lambda >= 0
    s1 = ops.apply(GRID, "TV", x)
    sup = np.abs(s1) > 1e-6 * np.abs(s1).max()
    lam = -v[1][sup] * np.sign(s1[sup])
    assert lam.min() >= -1e-9 * lam.max()
    assert (lam.max() - lam.min()) <= 1e-4 * lam.max()


def test_idempotent_on_feasible_model():
    grid = {"n": (6, 5), "h": (1.0, 1.0)}
    iz = np.tile(np.arange(6), 5)
    m = 2.5 + 0.1 * iz                            # in [2, 4] and D_z m >= 0
    sets = [{"op": "I", "type": "bounds", "lo": 2.0, "hi": 4.0},
            {"op": "TV", "type": "l1", "sigma_rel": 1.0},
            {"op": "DZ", "type": "bounds", "lo": 0.0, "hi": math.inf}]
    res = run(m, grid, sets, iters=500)
    assert rel(res["x"], m) < 1e-8
    x1 = res["x"]
    sets_abs = P.resolve_sets(grid, sets, m)
    res2 = run(x1, grid, sets_abs, iters=500)
    assert rel(res2["x"], x1) < 1e-8


def test_paper_form_and_direct_form_agree():
    m = model(GRID, 7)
    sets = [{"op": "I", "type": "bounds", "lo": 2.5, "hi": 3.5},
            {"op": "TV", "type": "l1", "sigma": 0.4 * ops.norm_of(GRID, "TV", "l1", m)}]
    a = run(m, GRID, sets, iters=5000, form="alg1")
    b = run(m, GRID, sets, iters=5000, form="direct")
    assert rel(a["x"], b["x"]) < 1e-6


def test_feasibility_reported_below_eps_and_stop_rule():
    m = model(GRID, 9)
    sets = [{"op": "I", "type": "bounds", "lo": 2.5, "hi": 3.5},
            {"op": "DZ", "type": "bounds", "lo": 0.0, "hi": math.inf}]
    res = run(m, GRID, sets, iters=3000, stop=1)
    assert res["stop_reason"] == 1
    assert res["iters"] % 5 == 0 and res["iters"] < 3000
    assert all(f < 1e-3 for f in res["r_feas"]) and res["r_evol"] < 1e-2
    # recomputed from scratch on the returned x
    for i, s in enumerate(res["sets"]):
        assert P.feasibility(ops.apply(GRID, s["op"], res["x"]), s) == pytest.approx(res["r_feas"][i], rel=1e-9, abs=1e-15)


def test_schedule_replay_reproduces_adaptive_run():
    m = model(GRID, 10)
    sets = [{"op": "I", "type": "bounds", "lo": 2.5, "hi": 3.5},
            {"op": "TV", "type": "l1", "sigma": 0.5 * ops.norm_of(GRID, "TV", "l1", m)}]
    a = run(m, GRID, sets, iters=60, adapt=2)
    rs = np.array([t["rho"] for t in a["trace"]])
    gs = np.array([t["gamma"] for t in a["trace"]])
    assert np.ptp(rs) > 0           # rho really moved
    b = P.parsdmm(m, GRID, sets, P.options(max_iter=60, adapt=0), rho_schedule=rs, gamma_schedule=gs)
    assert np.array_equal(a["x"], b["x"])


# ---------------------------------------------------------------- ML
def test_restriction_of_linear_field_is_cell_centre_value():
    for n in ((8, 6), (8, 6, 4)):
        grid = {"n": n, "h": (1.0,) * len(n)}
        sh = ops.grid_shape(grid)
        iy, ix, iz = np.meshgrid(*[np.arange(s) for s in sh], indexing="ij")
        f = lambda z, x, y: 0.5 * z - 1.5 * x + 2.0 * y + 1.0
        m = f(iz, ix, iy).reshape(-1)
        c = P.restrict(grid, m)
        gc = P.coarse_grid(grid)
        csh = ops.grid_shape(gc)
        jy, jx, jz = np.meshgrid(*[np.arange(s) for s in csh], indexing="ij")
        ey = (2 * jy + 0.5) if len(n) == 3 else jy * 0
        assert np.allclose(c, f(2 * jz + 0.5, 2 * jx + 0.5, ey).reshape(-1), atol=1e-13)


@pytest.mark.parametrize("op", ["I", "DZ", "DX", "DY", "TV"])
def test_prolongation_reproduces_linear_fields(op):
    # every coarse output axis keeps >= 2 samples (a single coarse sample can
    # only be extended as a constant)
    n = (8, 6, 6)
    gf = {"n": n, "h": (1.0, 1.0, 1.0)}
    gc = P.coarse_grid(gf)
    f = lambda z, x, y: 0.25 * z + 0.75 * x - 0.5 * y + 2.0

    def sample(grid, name, scale):
        # values of f at the positions of the op's outputs, in fine-cell units
        if name == "I":
            shp, st = ops.grid_shape(grid), None
        else:
            shp, st = ops.diff_shape(grid, name), {"DZ": 2, "DX": 1, "DY": 0}[name]
        idx = np.meshgrid(*[np.arange(s) + (0.5 if st == a else 0.0) for a, s in enumerate(shp)], indexing="ij")
        pos = [scale * idx[a] + (0.5 * (scale - 1)) for a in range(3)]   # (y, x, z)
        return f(pos[2], pos[1], pos[0]).reshape(-1)
    names = ops.tv_parts(gf) if op == "TV" else [op]
    uc = np.concatenate([sample(gc, d, 2) for d in names])
    uf = np.concatenate([sample(gf, d, 1) for d in names])
    assert np.allclose(P.prolong(gc, gf, op, uc), uf, atol=1e-12)


@pytest.mark.parametrize("levels", [2, 3])
def test_multilevel_reaches_single_level_solution(levels):
    """Convex sets: the projection is unique, so ML-PARSDMM from any coarse
    warm start reaches the single-level solution."""
    grid = {"n": (16, 12), "h": (1.0, 1.0)}
    m = model(grid, 11)
    sets = [{"op": "I", "type": "bounds", "lo": 2.5, "hi": 3.5},
            {"op": "DZ", "type": "bounds", "lo": 0.0, "hi": math.inf}]
    o = P.options(max_iter=3000, adapt=1, gamma0=1.5)
    ml = P.ml_parsdmm(m, grid, sets, o, levels=levels, coarse_iter=300)
    sl = P.parsdmm(m, grid, sets, o)
    assert rel(ml["x"], sl["x"]) < 1e-5
    assert len(ml["levels"]) == levels
    assert [len(r["x"]) for r in ml["levels"]] == [int(np.prod(g)) for g in
                                                    [((16 >> j) + 0, (12 >> j) + 0) for j in range(levels - 1, -1, -1)]]


def test_single_per_column_l2_set_gives_columnwise_scaling():
    """One per-line set on A = I: the projection of m onto it, i.e. every
    column scaled into its own l2 ball."""
    m = model(GRID, 12)
    nz, nx = GRID["n"][0], GRID["n"][1]
    X = m.reshape(nx, nz).T
    sigma = 0.8 * float(np.median(np.linalg.norm(X, axis=0)))
    expect = X * np.minimum(1.0, sigma / np.linalg.norm(X, axis=0))[None, :]
    res = run(m, GRID, [{"op": "I", "type": "l2", "sigma": sigma, "scope": "z"}], iters=400)
    assert rel(res["x"], expect.T.reshape(-1)) < 1e-8


def test_single_annulus_set_gives_radial_scaling():
    m = model(GRID, 13)
    n = float(np.linalg.norm(m))
    res = run(m, GRID, [{"op": "I", "type": "annulus", "lo": 1.3 * n, "hi": 2.0 * n}], iters=400)
    assert rel(res["x"], m * 1.3) < 1e-8


def test_per_line_sets_reject_unsupported_forms():
    m = model(GRID, 14)
    with pytest.raises(ValueError):
        P.resolve_sets(GRID, [{"op": "TV", "type": "l1", "sigma": 1.0, "scope": "z"}], m)
    with pytest.raises(ValueError):
        P.resolve_sets(GRID, [{"op": "I", "type": "l2", "sigma_rel": 0.5, "scope": "x"}], m)
    with pytest.raises(ValueError):
        P.resolve_sets(GRID, [{"op": "I", "type": "l2", "sigma": 1.0, "scope": "y"}], m)
    r = P.resolve_sets(GRID, [{"op": "DZ", "type": "card", "k_frac": 0.25, "scope": "z"}], m)[0]
    assert r["k"] == int(0.25 * (GRID["n"][0] - 1))


def test_single_vector_bounds_set_gives_entrywise_clip():
    """A per-entry bounds set on A = I alone: the projection is the clip of
    m to its own interval at every entry."""
    m = model(GRID, 15)
    g = np.random.default_rng(15)
    lo = m - g.uniform(0.0, 0.5, m.size) - 0.2
    hi = lo + g.uniform(0.0, 0.4, m.size)
    res = run(m, GRID, [{"op": "I", "type": "bounds", "lo": lo, "hi": hi}], iters=400)
    assert rel(res["x"], np.clip(m, lo, hi)) < 1e-8


def test_single_l2_data_set_gives_the_ball_projection():
    """A lone l2 data-fit set on A = I: the projection of m onto the ball
    around the observed values (masked entries free)."""
    m = model(GRID, 16)
    g = np.random.default_rng(16)
    d = m + 0.5 * g.standard_normal(m.size)
    d[g.uniform(size=m.size) < 0.25] = np.nan
    sigma = 0.3 * float(np.linalg.norm((m - d)[~np.isnan(d)]))
    res = run(m, GRID, [{"op": "I", "type": "l2", "sigma": sigma, "center": d}], iters=400)
    from oracle import prox as PX
    assert rel(res["x"], PX.proj_l2_data(m, d, sigma)) < 1e-8


def test_blur_data_fit_matches_general_qp_solver():
    """The projection-as-inverse-problem form with a blurring forward
    operator (Sec. "Introduction", data-fit formulation): min 1/2||x - m||^2
    s.t. l <= F x - d <= u on the observed samples (a restriction of the blur,
    +-inf elsewhere) and 2 <= x <= 4, against SLSQP with F built from
    scipy's zero-padded convolution."""
    opt = pytest.importorskip("scipy.optimize")
    nd = pytest.importorskip("scipy.ndimage")
    grid = {"n": (8, 6), "h": (1.0, 1.0)}
    N = ops.grid_size(grid)
    taps = (0.4, 0.2, 0.1)
    kfull = np.array(taps[::-1] + taps[1:])
    F = np.stack([nd.convolve1d(e.reshape(6, 8), kfull, axis=0, mode="constant").reshape(-1)
                  for e in np.eye(N)], axis=1)   # blur along x (axis 0 of the (nx, nz) array)
    g = np.random.default_rng(21)
    truth = 3.0 + 0.6 * g.standard_normal(N)
    obs = g.uniform(size=N) < 0.5
    d = F @ truth + g.uniform(-0.05, 0.05, N)
    lo = np.where(obs, d - 0.08, -math.inf)
    hi = np.where(obs, d + 0.08, math.inf)
    m = truth + 0.7 * g.standard_normal(N)
    Fo = F[obs]
    cons = [{"type": "ineq", "fun": lambda x: hi[obs] - Fo @ x, "jac": lambda x: -Fo},
            {"type": "ineq", "fun": lambda x: Fo @ x - lo[obs], "jac": lambda x: Fo}]
    sol = opt.minimize(lambda x: 0.5 * np.sum((x - m) ** 2), np.clip(m, 2.0, 4.0), jac=lambda x: x - m,
                       bounds=[(2.0, 4.0)] * N, constraints=cons, method="SLSQP",
                       options={"maxiter": 2000, "ftol": 1e-14})
    assert sol.success
    sets = [{"op": "BLUR", "axis": "x", "taps": taps, "type": "bounds", "lo": lo, "hi": hi},
            {"op": "I", "type": "bounds", "lo": 2.0, "hi": 4.0}]
    res = run(m, grid, sets, iters=6000)
    assert rel(res["x"], sol.x) < 1e-5
    # the data fit binds: some observed samples sit on their bounds
    s = F @ res["x"]
    assert np.sum(obs & ((np.abs(s - lo) < 1e-5) | (np.abs(s - hi) < 1e-5))) > 0


def test_blur_rejected_with_levels_and_lines():
    m = model(GRID, 22)
    blur = {"op": "BLUR", "axis": "z", "taps": (0.5, 0.25), "type": "bounds", "lo": 0.0, "hi": 9.0}
    with pytest.raises(ValueError):
        P.ml_parsdmm(m, GRID, [blur], P.options(max_iter=5), levels=2)
    with pytest.raises(ValueError):
        P.parsdmm(m, GRID, [dict(blur, type="l2", sigma=1.0, scope="z")], P.options(max_iter=5))


def test_blur_l2_data_ball_matches_general_qp_solver():
    """The l2 data-fit ball with a blurring forward operator, min 1/2||x - m||^2
    s.t. ||M (F x - d)||_2 <= sigma (M the observation mask: NaN in d),
    against SLSQP with F from scipy's zero-padded convolution."""
    opt = pytest.importorskip("scipy.optimize")
    nd = pytest.importorskip("scipy.ndimage")
    grid = {"n": (7, 6), "h": (1.0, 1.0)}
    N = ops.grid_size(grid)
    taps = (0.5, 0.25)
    kfull = np.array(taps[::-1] + taps[1:])
    F = np.stack([nd.convolve1d(e.reshape(6, 7), kfull, axis=1, mode="constant").reshape(-1)
                  for e in np.eye(N)], axis=1)   # blur along z (axis 1 of the (nx, nz) array)
    g = np.random.default_rng(31)
    truth = 3.0 + 0.5 * g.standard_normal(N)
    d = F @ truth + 0.1 * g.standard_normal(N)
    obs = g.uniform(size=N) < 0.6
    d[~obs] = np.nan
    m = truth + 0.8 * g.standard_normal(N)
    Fo, do = F[obs], d[obs]
    sigma = 0.3 * float(np.linalg.norm(Fo @ m - do))
    cons = [{"type": "ineq", "fun": lambda x: sigma ** 2 - np.sum((Fo @ x - do) ** 2),
             "jac": lambda x: -2.0 * (Fo @ x - do) @ Fo}]
    sol = opt.minimize(lambda x: 0.5 * np.sum((x - m) ** 2), m.copy(), jac=lambda x: x - m,
                       constraints=cons, method="SLSQP", options={"maxiter": 1000, "ftol": 1e-15})
    assert sol.success
    sets = [{"op": "BLUR", "axis": "z", "taps": taps, "type": "l2", "sigma": sigma, "center": d}]
    res = run(m, grid, sets, iters=4000)
    assert rel(res["x"], sol.x) < 1e-5
    # the ball binds
    assert float(np.linalg.norm(Fo @ res["x"] - do)) == pytest.approx(sigma, rel=1e-5)


def test_init_rho_gamma_equal_the_uniform_starting_values():
    """Starting penalties given per block reproduce the rho0 / gamma0 runs
    when they are uniform (with and without adaptation)."""
    m = model(GRID, 41)
    sets = [{"op": "I", "type": "bounds", "lo": 2.5, "hi": 3.5},
            {"op": "TV", "type": "l1", "sigma_rel": 0.4}]
    for adapt in (0, 1):
        base = P.parsdmm(m, GRID, sets, P.options(max_iter=30, adapt=adapt, rho0=2.5, gamma0=1.3))
        nb = len(base["blocks"])
        same = P.parsdmm(m, GRID, sets, P.options(max_iter=30, adapt=adapt, rho0=1.0, gamma0=1.0),
                         init_rho=[2.5] * nb, init_gamma=[1.3] * nb)
        assert np.array_equal(same["x"], base["x"])
    with pytest.raises(ValueError):
        P.parsdmm(m, GRID, sets, P.options(max_iter=3), init_rho=[1.0])


def test_warm_start_from_the_fixed_point_stays_there():
    """Started from its own converged iterates (x, y_i, v_i) and penalties,
    the iteration is at a fixed point: a convex problem's solution does not
    move (the state a warm start hands over is the whole ADMM state)."""
    m = model(GRID, 42)
    sets = [{"op": "I", "type": "bounds", "lo": 2.5, "hi": 3.5},
            {"op": "TV", "type": "l1", "sigma": 0.2 * ops.norm_of(GRID, "TV", "l1", m)}]
    conv = run(m, GRID, sets, iters=6000, adapt=0)
    again = P.parsdmm(m, GRID, sets, P.options(max_iter=20, adapt=0, rho0=1.0, gamma0=1.5),
                      init=(conv["x"], conv["y"], conv["v"]))
    assert rel(again["x"], conv["x"]) < 1e-9
    cold = P.parsdmm(m, GRID, sets, P.options(max_iter=20, adapt=0, rho0=1.0, gamma0=1.5))
    assert rel(cold["x"], conv["x"]) > 1e-6   # 20 cold iterations are not there yet


def test_warm_start_with_adapt_state_continues_the_run():
    """A run of 2K iterations equals K iterations followed by a warm start
    that carries x, y_i, v_i, rho_i, gamma_i and the quantities Algorithm
    adapt-rho-gamma saved at its last call (K even: the continued run's adapt
    calls fall on the same iterations).  Without the saved quantities the
    continuation differs (its first call only saves)."""
    grid = {"n": (9, 7)}
    m = model(grid, seed=4)
    sets = [{"op": "I", "type": "bounds", "lo": 2.0, "hi": 4.0},
            {"op": "TV", "type": "l1", "sigma_rel": 0.4},
            {"op": "DZ", "type": "bounds", "lo": 0.0, "hi": math.inf}]
    o = P.options(max_iter=60, adapt=2, adapt_every=2, rho0=1.0, gamma0=1.5)
    full = P.parsdmm(m, grid, sets, o)
    half = P.parsdmm(m, grid, sets, dict(o, max_iter=30))
    init = (half["x"], half["y"], half["v"])
    cont = P.parsdmm(m, grid, sets, dict(o, max_iter=30), init=init, init_rho=half["rho"],
                     init_gamma=half["gamma"], init_k0=half["k0"])
    np.testing.assert_allclose(cont["x"], full["x"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(cont["rho"], full["rho"], rtol=1e-13)
    cold = P.parsdmm(m, grid, sets, dict(o, max_iter=30), init=init, init_rho=half["rho"],
                     init_gamma=half["gamma"])
    assert not np.allclose(cold["rho"], full["rho"], rtol=1e-6)
