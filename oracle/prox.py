"""Projections onto the simple sets C_i and the prox of the squared distance.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Every function takes and returns flat float64 vectors.  The sets are those of
the set table (Sec. "Software and numerical examples"); the projection is the
Euclidean one of Eq. proj_prob.
"""
import numpy as np


def proj_bounds(w, lo, hi):
    """Bounds {l[i] <= w[i] <= u[i]}: the projection is the element-wise
    clip (set table, "bounds").  l and u are scalars or vectors of w's
    length; vectors give the point-wise data-fit set {l <= F x - d_obs <= u}
    of the paper's projection-as-inverse-problem formulation, with F the
    set's operator and d_obs folded into the bounds (l + d_obs, u + d_obs),
    and +-inf where nothing is observed."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    if np.any(lo > hi):
        raise ValueError("proj_bounds: lo > hi")
    return np.minimum(np.maximum(np.asarray(w, dtype=np.float64), lo), hi)


def proj_l2(w, sigma):
    """l2 ball {||w||_2 <= sigma}: radial scaling by min(1, sigma/||w||_2)
    (set table, "l2")."""
    w = np.asarray(w, dtype=np.float64)
    nrm = float(np.sqrt(np.sum(w * w)))
    if nrm <= sigma:
        return w.copy()
    return w * (sigma / nrm)


def proj_l2_data(w, center, sigma):
    """Data-fit l2 ball {||M (w - d)||_2 <= sigma} around observed values d
    (the paper's l2 data-fit set {||F x - d_obs|| <= sigma} with F the
    set's operator, here together with a binary mask M): ``center`` holds d,
    NaN where nothing is observed.  Observed entries move radially toward d
    when outside the ball; unobserved entries are not constrained and stay."""
    w = np.asarray(w, dtype=np.float64)
    c = np.asarray(center, dtype=np.float64)
    obs = ~np.isnan(c)
    y = w.copy()
    r = w[obs] - c[obs]
    nrm = float(np.sqrt(np.sum(r * r)))
    if nrm > sigma:
        y[obs] = c[obs] + r * (sigma / nrm)
    return y


def proj_annulus(w, lo, hi):
    """Annulus {sigma_l <= ||w||_2 <= sigma_u} (set table, "annulus"):
    radial scaling onto the nearer sphere when ||w||_2 lies outside
    [sigma_l, sigma_u].  The set is not convex for sigma_l > 0.  Reading:
    w = 0 has no nearest point of a unique direction; it is returned
    unchanged."""
    if not (0.0 <= lo <= hi):
        raise ValueError("proj_annulus: need 0 <= lo <= hi")
    w = np.asarray(w, dtype=np.float64)
    nrm = float(np.sqrt(np.sum(w * w)))
    if nrm > hi:
        return w * (hi / nrm)
    if 0.0 < nrm < lo:
        return w * (lo / nrm)
    return w.copy()


def lines(shape, scope):
    """Index arrays of the lines of an array of shape (ny, nx, nz) (z
    fastest, Sec. "Notation") that a per-line set applies to: "z" the
    lines along z (the columns X[:, j] of a 2D model), "x" the lines along x
    (the rows X[i, :]), "y" the lines along y (the fibers of a 3D model).
    Each array lists its line's linear indices in increasing order."""
    ny, nx, nz = shape
    idx = np.arange(ny * nx * nz).reshape(ny, nx, nz)
    if scope == "z":
        return list(idx.reshape(ny * nx, nz))
    if scope == "x":
        return list(np.transpose(idx, (0, 2, 1)).reshape(ny * nz, nx))
    if scope == "y":
        return list(np.transpose(idx, (1, 2, 0)).reshape(nx * nz, ny))
    raise ValueError("unknown scope %r" % (scope,))


def l1_threshold(w, tau):
    """Soft-threshold level theta of the l1-ball projection, by sorting
    (Duchi et al. 2008, the l1-ball projection the paper uses, Sec.
    "Parallel Dykstra versus PARSDMM").

    Sort |w| in decreasing order into u, form the running sums c_j, take the
    largest j with u_j > (c_j - tau)/j and return theta = (c_j - tau)/j.
    Returns 0 when ||w||_1 <= tau (w is already inside the ball).  For
    tau = 0 the ball is {0} and theta = max|w|.
    """
    if tau < 0:
        raise ValueError("l1_threshold: tau < 0")
    a = np.abs(np.asarray(w, dtype=np.float64))
    if a.size == 0 or float(np.sum(a)) <= tau:
        return 0.0
    if tau == 0.0:
        return float(np.max(a))
    u = np.sort(a)[::-1]
    c = np.cumsum(u)
    j = np.arange(1, u.size + 1)
    ok = u > (c - tau) / j
    rho = int(np.nonzero(ok)[0][-1]) + 1
    return float((c[rho - 1] - tau) / rho)


def proj_l1(w, tau):
    """l1 ball {||w||_1 <= tau} (set table, "l1"):
    y = sign(w) * max(|w| - theta, 0) with theta from ``l1_threshold``."""
    w = np.asarray(w, dtype=np.float64)
    theta = l1_threshold(w, tau)
    if theta == 0.0:
        return w.copy()
    return np.sign(w) * np.maximum(np.abs(w) - theta, 0.0)


def card_support(w, k):
    """Indices kept by the cardinality projection {card(w) <= k} (set table,
    "cardinality"): the k entries of largest |w|.

    Reading (the set is non-convex, so the projection is not unique at
    ties, Sec. "Notation"): order by |w| decreasing, ties broken by the lower
    linear index; keep exactly min(k, len(w)) entries.
    """
    w = np.asarray(w, dtype=np.float64)
    k = int(k)
    if k < 0:
        raise ValueError("card_support: k < 0")
    order = np.argsort(-np.abs(w), kind="stable")
    return np.sort(order[:min(k, w.size)])


def proj_card(w, k):
    """Cardinality projection: keep the entries of ``card_support``, zero the
    rest."""
    w = np.asarray(w, dtype=np.float64)
    y = np.zeros_like(w)
    idx = card_support(w, k)
    y[idx] = w[idx]
    return y


def prox_dist(w, m, rho):
    """Prox of f(z) = 1/2 ||z - m||^2 with weight rho (Eq. prox_sq_dist):
    (m + rho w) / (1 + rho), point-wise."""
    return (np.asarray(m, dtype=np.float64) + rho * np.asarray(w, dtype=np.float64)) / (1.0 + rho)


def project(set_spec, w):
    """Projection P_C(w) for a set specification dict with key "type" in
    {"bounds", "l1", "l2", "card", "annulus"} and the resolved parameters
    "lo"/"hi", "sigma" or "k".  With "scope" in {"z", "x", "y"} the set
    constrains every line of that direction on its own (the per-column,
    per-row and per-fiber sets of Sec. "Software and numerical examples"),
    so the projection is the simple set's projection of each line; "shape"
    gives the (ny, nx, nz) array shape of w."""
    scope = set_spec.get("scope", "all")
    if scope != "all":
        w = np.asarray(w, dtype=np.float64)
        y = np.empty_like(w)
        base = dict(set_spec, scope="all")
        for ln in lines(set_spec["shape"], scope):
            y[ln] = project(base, w[ln])
        return y
    t = set_spec["type"]
    if t == "annulus":
        return proj_annulus(w, set_spec["lo"], set_spec["hi"])
    if t == "bounds":
        return proj_bounds(w, set_spec["lo"], set_spec["hi"])
    if t == "l2":
        if set_spec.get("center") is not None:
            return proj_l2_data(w, set_spec["center"], set_spec["sigma"])
        return proj_l2(w, set_spec["sigma"])
    if t == "l1":
        return proj_l1(w, set_spec["sigma"])
    if t == "card":
        return proj_card(w, set_spec["k"])
    raise ValueError("unknown set type %r" % (t,))
