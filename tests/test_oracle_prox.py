"""Pins for oracle/prox.py against brute force and optimality conditions.

The set table (Sec. "Software and numerical examples") defines the sets;
Eq. proj_prob defines the projection as the nearest point; Eq. prox_sq_dist
gives the prox of the squared distance in closed form.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import prox


def _rand(n, seed):
    return np.random.default_rng(seed).standard_normal(n) * 2.0


def test_bounds_is_nearest_point_per_entry():
    w = _rand(50, 1)
    y = prox.proj_bounds(w, -0.5, 1.25)
    for wi, yi in zip(w, y):
        cands = np.linspace(-0.5, 1.25, 2001)
        best = cands[np.argmin(np.abs(cands - wi))]
        assert abs(yi - wi) <= abs(best - wi) + 1e-12
        assert -0.5 <= yi <= 1.25
    assert np.array_equal(prox.proj_bounds(w, 0.0, math.inf), np.maximum(w, 0.0))
    with pytest.raises(ValueError):
        prox.proj_bounds(w, 1.0, 0.0)


def test_l2_ball_projection_optimality():
    g = np.random.default_rng(2)
    for n, sigma in ((1, 0.3), (5, 1.0), (40, 3.0)):
        w = g.standard_normal(n) * 3
        y = prox.proj_l2(w, sigma)
        assert np.linalg.norm(y) <= sigma * (1 + 1e-14) or np.allclose(y, w)
        # variational inequality: <w - y, z - y> <= 0 for all z in the ball
        for _ in range(200):
            z = g.standard_normal(n)
            z *= g.uniform(0, sigma) / np.linalg.norm(z)
            assert float((w - y) @ (z - y)) <= 1e-12
    w = np.array([3.0, 4.0])
    assert np.allclose(prox.proj_l2(w, 1.0), [0.6, 0.8])
    assert np.array_equal(prox.proj_l2(w, 5.0), w)


def _theta_by_bisection(w, tau):
    """theta >= 0 with sum max(|w| - theta, 0) = tau, by bisection (an
    independent route to the l1-ball KKT conditions)."""
    a = np.abs(w)
    if a.sum() <= tau:
        return 0.0
    lo, hi = 0.0, float(a.max())
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.maximum(a - mid, 0).sum() > tau:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 10, 64])
def test_l1_threshold_matches_bisection(n):
    for seed in range(5):
        w = _rand(n, 100 + seed)
        for frac in (0.0, 0.1, 0.5, 0.9, 1.0, 1.5):
            tau = frac * float(np.abs(w).sum())
            th = prox.l1_threshold(w, tau)
            ref = _theta_by_bisection(w, tau)
            assert th == pytest.approx(ref, rel=1e-12, abs=1e-12)
            y = prox.proj_l1(w, tau)
            if frac < 1.0:
                assert np.abs(y).sum() == pytest.approx(tau, rel=1e-12, abs=1e-12)
            else:
                assert np.array_equal(y, w)


def test_l1_projection_brute_force_support_enumeration():
    """For n <= 8 enumerate every support set S and sign pattern fixed by w:
    on S, y = sign(w)(|w| - t) with t = (sum_S |w| - tau)/|S|; keep the
    feasible candidate nearest to w (the projection is unique)."""
    g = np.random.default_rng(11)
    for n in range(1, 9):
        for _ in range(10):
            w = g.standard_normal(n) * 2
            tau = g.uniform(0.05, 0.95) * np.abs(w).sum()
            best, best_d = None, np.inf
            for r in range(1, n + 1):
                for S in itertools.combinations(range(n), r):
                    S = list(S)
                    t = (np.abs(w[S]).sum() - tau) / r
                    if t < 0:
                        continue
                    y = np.zeros(n)
                    y[S] = np.sign(w[S]) * (np.abs(w[S]) - t)
                    if np.any(np.sign(y[S]) != np.sign(w[S])) or np.any(np.abs(w[S]) < t):
                        continue
                    d = np.linalg.norm(y - w)
                    if np.abs(y).sum() <= tau * (1 + 1e-12) and d < best_d:
                        best, best_d = y, d
            y = prox.proj_l1(w, tau)
            assert np.allclose(y, best, atol=1e-12)


def test_l1_special_cases():
    w = np.array([1.0, -2.0, 3.0])
    assert np.array_equal(prox.proj_l1(w, 0.0), np.zeros(3))
    assert np.array_equal(prox.proj_l1(w, 10.0), w)
    # tau = 1 against sorted |w| = 3, 2, 1: theta = 2, only the 3 survives
    assert np.allclose(prox.proj_l1(w, 1.0), [0.0, 0.0, 1.0])
    # ties in |w| do not matter for the threshold
    assert np.allclose(prox.proj_l1(np.array([2.0, -2.0]), 2.0), [1.0, -1.0])


def test_card_brute_force_over_subsets():
    g = np.random.default_rng(5)
    for n in range(1, 11):
        for k in range(0, n + 2):
            w = g.standard_normal(n)
            best_S, best_d = None, np.inf
            for S in itertools.combinations(range(n), min(k, n)):
                y = np.zeros(n)
                y[list(S)] = w[list(S)]
                d = np.linalg.norm(y - w)
                if d < best_d:
                    best_S, best_d = set(S), d
            assert set(prox.card_support(w, k).tolist()) == best_S
            assert np.linalg.norm(prox.proj_card(w, k) - w) == pytest.approx(best_d, abs=1e-14)


def test_card_tie_rule_prefers_lower_index():
    w = np.array([1.0, -3.0, 3.0, 0.5, -3.0])
    assert prox.card_support(w, 2).tolist() == [1, 2]
    assert prox.card_support(w, 3).tolist() == [1, 2, 4]
    assert prox.card_support(w, 0).tolist() == []
    assert np.array_equal(prox.proj_card(w, 9), w)


def test_prox_dist_is_minimiser():
    g = np.random.default_rng(9)
    m, w = g.standard_normal(20), g.standard_normal(20)
    for rho in (0.1, 1.0, 7.5):
        z = prox.prox_dist(w, m, rho)
        # gradient of 1/2||z - m||^2 + rho/2 ||z - w||^2 vanishes at z
        assert np.allclose((z - m) + rho * (z - w), 0, atol=1e-14)


def test_annulus_nearest_point_and_special_cases():
    """Annulus {lo <= ||w|| <= hi}: nearest point over sampled members; with
    lo = 0 it is the l2 ball."""
    g = np.random.default_rng(7)
    for n, lo, hi in ((2, 1.0, 2.0), (3, 0.5, 0.8), (6, 2.0, 2.0)):
        for scale in (0.1, 1.0, 1.5, 5.0):
            w = g.standard_normal(n)
            w *= scale * (lo + hi) / 2 / np.linalg.norm(w)
            y = prox.proj_annulus(w, lo, hi)
            ny = np.linalg.norm(y)
            assert lo * (1 - 1e-14) <= ny <= hi * (1 + 1e-14)
            # no sampled member of the annulus is closer
            for _ in range(300):
                z = g.standard_normal(n)
                z *= g.uniform(lo, hi) / np.linalg.norm(z)
                assert np.linalg.norm(z - w) >= np.linalg.norm(y - w) - 1e-12
        w = g.standard_normal(n)
        assert np.allclose(prox.proj_annulus(w, 0.0, 0.7), prox.proj_l2(w, 0.7), rtol=0, atol=1e-15)
    assert np.allclose(prox.proj_annulus(np.array([0.3, 0.4]), 1.0, 2.0), [0.6, 0.8])
    assert np.allclose(prox.proj_annulus(np.array([3.0, 4.0]), 1.0, 2.0), [1.2, 1.6])
    assert np.array_equal(prox.proj_annulus(np.zeros(3), 1.0, 2.0), np.zeros(3))
    with pytest.raises(ValueError):
        prox.proj_annulus(np.ones(2), 2.0, 1.0)


def test_lines_follow_the_array_layout():
    """Lines against numpy views of the z-fastest layout: X = w.reshape(nx, nz).T
    is the n_z x n_x model, its columns X[:, j] and rows X[i, :]."""
    nz, nx = 4, 3
    w = np.arange(nz * nx, dtype=float)
    X = w.reshape(nx, nz).T
    cols = prox.lines((1, nx, nz), "z")
    rows = prox.lines((1, nx, nz), "x")
    assert len(cols) == nx and len(rows) == nz
    for j in range(nx):
        assert np.array_equal(w[cols[j]], X[:, j])
    for i in range(nz):
        assert np.array_equal(w[rows[i]], X[i, :])
    ny = 2
    w3 = np.arange(nz * nx * ny, dtype=float)
    V = w3.reshape(ny, nx, nz)   # V[iy, ix, iz]
    fib = prox.lines((ny, nx, nz), "y")
    assert len(fib) == nz * nx
    assert any(np.array_equal(w3[f], V[:, 1, 2]) for f in fib)


def test_per_line_card_is_nearest_point_of_the_product_set():
    """card(X[:, j]) <= k for every column j: brute force over all supports
    of all columns at once (the set is their Cartesian product)."""
    g = np.random.default_rng(8)
    nz, nx, k = 3, 3, 1
    w = g.standard_normal(nz * nx)
    spec = {"type": "card", "k": k, "scope": "z", "shape": (1, nx, nz)}
    y = prox.project(spec, w)
    best = np.inf
    for S in itertools.product(itertools.combinations(range(nz), k), repeat=nx):
        z = np.zeros_like(w)
        for j, sj in enumerate(S):
            for i in sj:
                z[j * nz + i] = w[j * nz + i]
        best = min(best, float(np.linalg.norm(z - w)))
    assert float(np.linalg.norm(y - w)) == pytest.approx(best, abs=1e-14)
    assert all(np.count_nonzero(y[j * nz:(j + 1) * nz]) <= k for j in range(nx))


def test_per_line_l2_and_l1_row_constraints():
    """Rows X[i, :] each in an l2 ball / l1 ball: every row satisfies its
    constraint, and rows already inside are unchanged."""
    g = np.random.default_rng(9)
    nz, nx = 5, 7
    w = g.standard_normal(nz * nx) * 2
    X = w.reshape(nx, nz).T
    for t, norm in (("l2", lambda r: np.linalg.norm(r)), ("l1", lambda r: np.abs(r).sum())):
        sigma = float(np.median([norm(X[i, :]) for i in range(nz)]))
        y = prox.project({"type": t, "sigma": sigma, "scope": "x", "shape": (1, nx, nz)}, w)
        Y = y.reshape(nx, nz).T
        for i in range(nz):
            assert norm(Y[i, :]) <= sigma * (1 + 1e-12)
            if norm(X[i, :]) <= sigma:
                assert np.array_equal(Y[i, :], X[i, :])


def test_vector_bounds_nearest_point_and_data_fit_reading():
    """Per-entry bounds: the clip is the nearest point entry by entry; with
    l + d, u + d as bounds it is the projection onto {l <= w - d <= u}, and
    +-inf leaves an entry free (an unobserved pixel of a mask)."""
    g = np.random.default_rng(11)
    n = 40
    w = g.standard_normal(n) * 2
    d = g.standard_normal(n)
    lo = np.where(g.uniform(size=n) < 0.5, d - 0.3, -math.inf)
    hi = np.where(np.isfinite(lo), d + 0.2, math.inf)
    y = prox.proj_bounds(w, lo, hi)
    for i in range(n):
        if np.isfinite(lo[i]):
            cands = np.linspace(lo[i], hi[i], 1001)
            assert abs(y[i] - w[i]) <= np.min(np.abs(cands - w[i])) + 1e-12
            assert -0.3 - 1e-15 <= y[i] - d[i] <= 0.2 + 1e-15
        else:
            assert y[i] == w[i]
    with pytest.raises(ValueError):
        prox.proj_bounds(w, np.zeros(n), -np.ones(n))


def test_l2_data_ball_nearest_point_and_reduction():
    """{||M (w - d)|| <= sigma}: the nearest point over sampled members (the
    free entries equal w's, the observed ones on or inside the ball around
    d); with no NaN and d = 0 it is the l2 ball."""
    g = np.random.default_rng(12)
    n = 6
    for trial in range(20):
        w = g.standard_normal(n) * 2
        d = g.standard_normal(n)
        d[g.uniform(size=n) < 0.3] = np.nan
        obs = ~np.isnan(d)
        sigma = 0.7
        y = prox.proj_l2_data(w, d, sigma)
        assert np.array_equal(y[~obs], w[~obs])
        assert np.linalg.norm(y[obs] - d[obs]) <= sigma * (1 + 1e-14) + 1e-15
        for _ in range(200):
            z = w.copy()
            u = g.standard_normal(obs.sum())
            z[obs] = d[obs] + u * (g.uniform(0, sigma) / max(np.linalg.norm(u), 1e-300))
            assert np.linalg.norm(z - w) >= np.linalg.norm(y - w) - 1e-12
    w = g.standard_normal(10)
    assert np.allclose(prox.proj_l2_data(w, np.zeros(10), 0.5), prox.proj_l2(w, 0.5), atol=1e-15, rtol=0)
