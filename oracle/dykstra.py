"""Algorithm Parallel-DYKSTRA (Appendix A) -- an independent cross-check.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Used by the tests to pin the PARSDMM fixed point on convex intersections
whose per-set projections P_{V_i} are known in closed form (bounds, l2 ball
of x, vertical monotonicity via isotonic regression).
"""
import numpy as np


def parallel_dykstra(m, projectors, iters, weights=None, tol=0.0):
    """Parallel Dykstra's algorithm for argmin 1/2||x - m||^2 s.t. x in all V_i.

    Initialise x = m and one auxiliary copy per set, v_i = x; then repeat:
    y_i = P_{V_i}(v_i); x = sum_i w_i y_i with weights summing to one;
    v_i = x + v_i - y_i.  Stops after ``iters`` sweeps or when x changes by
    less than ``tol`` (relative).
    """
    m = np.asarray(m, dtype=np.float64).reshape(-1)
    p = len(projectors)
    w = np.full(p, 1.0 / p) if weights is None else np.asarray(weights, dtype=np.float64)
    if abs(float(np.sum(w)) - 1.0) > 1e-12:
        raise ValueError("weights must sum to one")
    x = m.copy()
    v = [x.copy() for _ in range(p)]
    for _ in range(int(iters)):
        y = [P(vi) for P, vi in zip(projectors, v)]
        x_new = np.zeros_like(x)
        for wi, yi in zip(w, y):
            x_new = x_new + wi * yi
        v = [x_new + vi - yi for vi, yi in zip(v, y)]
        done = tol > 0.0 and np.linalg.norm(x_new - x) <= tol * max(np.linalg.norm(x_new), 1e-300)
        x = x_new
        if done:
            break
    return x
