"""Algorithm PARSDMM, adapt-rho-gamma, stopping quantities and ML-PARSDMM.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Notation follows the paper.  Blocks i = 1..p are the user's sets (A_i, C_i);
in the paper's form ("alg1", Eqs. PARSDMM_1, PARSDMM_2, conc_variables) a
block p+1 with A_{p+1} = I_N and the prox of the squared distance to m is
appended.  The sign convention is the one of the augmented Lagrangian
(Eq. aug_lag): v_i^T (y_i - A_i x).

Sets are dicts: {"op": "I"|"DZ"|"DX"|"DY"|"TV"|"BLUR", "type": "bounds"|"l1"|
"l2"|"card", "lo", "hi", "sigma", "sigma_rel", "k", "k_frac"}; a "BLUR"
operator takes "axis" ("z", "x" or "y") and "taps" (k_0..k_R, see
``operators.blur_op``).  A radius given as
``sigma_rel`` is resolved against the model being projected
(sigma = sigma_rel * ||A m|| in the set's norm); a cardinality given as
``k_frac`` is resolved as floor(k_frac * N) with N the grid size.
"""
import math

import numpy as np

from . import operators as ops
from . import prox

DEFAULTS = dict(
    max_iter=200,        # iterations of the WHILE loop of Algorithm PARSDMM
    cg_iters=5,          # > 0: fixed CG steps per x-update; 0: Eq. cg_stop rule
    cg_max=100,          # cap on CG steps under the Eq. cg_stop rule
    eps_feas=1e-3,       # Eq. stopping_conditions, value used in the paper
    eps_evol=1e-2,       # Eq. stopping_conditions, value used in the paper
    check_every=5,       # feasibility tested every few iterations ("typically 5")
    evol_hist=5,         # s in Eq. obj_stop
    stop=0,              # 0: run max_iter; 1: Eq. stopping_conditions; 2: feasibility only
    adapt=0,             # 0: fixed rho/gamma; 1: adapt rho only; 2: rho and gamma
    adapt_every=2,       # "update-frequency" of Algorithm PARSDMM
    rho0=1.0,
    gamma0=1.0,
    eps_corr=0.3,        # Algorithm adapt-rho-gamma
    rho_ratio_max=1e3,   # safeguard on rho_i relative to rho_{p+1}
    gamma_max=1.99,      # gamma_i kept in [1, 2)
    form="alg1",         # "alg1": identity block p+1; "direct": distance term in the x-step
)


def options(**kw):
    o = dict(DEFAULTS)
    for k, v in kw.items():
        if k not in o:
            raise KeyError("unknown option %r" % (k,))
        o[k] = v
    return o


_SCOPE_AXIS = {"z": 2, "x": 1, "y": 0}   # axis of the (ny, nx, nz) shape


def resolve_sets(grid, sets, m):
    """Resolve relative radii / cardinalities against the model m.

    Per-line sets ("scope" "z", "x" or "y"): readings.  Their radius applies
    to every line and is absolute (a relative radius is rejected); k_frac
    resolves against the line length; the TV stack is rejected (its parts
    live on different grids)."""
    out = []
    N = ops.grid_size(grid)
    for s in sets:
        r = dict(s)
        if r["op"] == "BLUR":
            r["op"] = ops.blur_op(r.pop("axis"), r.pop("taps"))
        r.setdefault("lo", -math.inf)
        r.setdefault("hi", math.inf)
        if r["type"] == "bounds" and (np.ndim(r["lo"]) or np.ndim(r["hi"])):
            # per-entry bounds (point-wise data fit): one value per row of A
            M = ops.out_size(grid, r["op"])
            r["lo"] = np.broadcast_to(np.asarray(r["lo"], dtype=np.float64), (M,)).copy()
            r["hi"] = np.broadcast_to(np.asarray(r["hi"], dtype=np.float64), (M,)).copy()
        scope = r.setdefault("scope", "all")
        if scope != "all":
            if r["op"] == "TV" or ops.is_blur(r["op"]):
                raise ValueError("per-line sets need I or a difference operator")
            if r.get("sigma_rel", 0.0):
                raise ValueError("per-line sets take absolute radii")
            r["shape"] = ops.grid_shape(grid) if r["op"] == "I" else ops.diff_shape(grid, r["op"])
            if r["shape"][_SCOPE_AXIS[scope]] < 1 or (scope == "y" and len(grid["n"]) < 3):
                raise ValueError("no lines along %s" % scope)
        if r.get("center") is not None:
            # l2 data fit: one observed value (or NaN) per row of A
            if r["type"] != "l2" or r.get("sigma_rel", 0.0) or scope != "all":
                raise ValueError("a center goes with an absolute l2 radius on the whole set")
            r["center"] = np.asarray(r["center"], dtype=np.float64).reshape(-1).copy()
            if r["center"].size != ops.out_size(grid, r["op"]):
                raise ValueError("center needs one value per row of A")
        if r["type"] in ("l1", "l2"):
            if r.get("sigma_rel", 0.0):
                r["sigma"] = r["sigma_rel"] * ops.norm_of(grid, r["op"], r["type"], m)
            r["sigma"] = float(r["sigma"])
        if r["type"] == "annulus":
            r["lo"], r["hi"] = float(r["lo"]), float(r["hi"])
        if r["type"] == "card":
            if r.get("k_frac", 0.0):
                n = N if scope == "all" else r["shape"][_SCOPE_AXIS[scope]]
                r["k"] = int(math.floor(r["k_frac"] * n))
            r["k"] = int(r["k"])
        out.append(r)
    return out


# --------------------------------------------------------------------------
# x-update: conjugate gradient on the normal equations (Sec. "Solving the
# linear system and automatic parameter selection"; Eq. cg_stop)
# --------------------------------------------------------------------------
def cg(apply_c, b, x0, n_fixed, cg_max):
    """Plain conjugate gradient from the warm start x0.

    n_fixed > 0: run that many steps.  n_fixed == 0: Eq. cg_stop, read as
    "stop once ||r_j|| / ||b|| < 0.1 ||r_0|| / ||b||" with r_0 the residual
    of the warm start, at most ``cg_max`` steps.  Both modes stop early when
    r = 0 or p^T C p <= 0.  Returns (x, steps).
    """
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - apply_c(x)
    p = r.copy()
    rr = float(r @ r)
    r0 = math.sqrt(rr)
    limit = n_fixed if n_fixed > 0 else cg_max
    steps = 0
    for _ in range(limit):
        if n_fixed == 0 and math.sqrt(rr) < 0.1 * r0:
            break
        if rr == 0.0:
            break
        q = apply_c(p)
        pq = float(p @ q)
        if pq <= 0.0:
            break
        alpha = rr / pq
        x = x + alpha * p
        r = r - alpha * q
        rr_new = float(r @ r)
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        steps += 1
    return x, steps


# --------------------------------------------------------------------------
# Algorithm adapt-rho-gamma
# --------------------------------------------------------------------------
def _corr(a_b, a_a, b_b):
    # Reading: a zero denominator gives correlation 0 ("not > eps_corr").
    d = a_a * b_b
    return a_b / math.sqrt(d) if d > 0.0 else 0.0


def _spectral(num_ab, aa, bb):
    """Hybrid of the minimum-gradient and steepest-descent spectral step
    sizes of Algorithm adapt-rho-gamma: MG = a.b/a.a, SD = b.b/a.b; keep MG
    when 2 MG > SD, else SD - MG/2."""
    mg = num_ab / aa
    sd = bb / num_ab
    return mg if 2.0 * mg > sd else sd - 0.5 * mg


def adapt_rho_gamma(dots, rho, gamma, opts):
    """One block's (rho, gamma) update from the six inner products of
    Algorithm adapt-rho-gamma.

    ``dots`` = (dh.dvh, dh.dh, dvh.dvh, dg.dv, dg.dg, dv.dv) with
    dh = s^{k+1} - s^{k0}, dvh = vhat^{k+1} - vhat^{k0},
    dg = -(y^{k+1} - y^{k0}), dv = v^{k+1} - v^{k0}.
    Returns (rho_new, gamma_new, case) with case in 1..4 for the four rows
    of the algorithm's (rho, gamma) table.  With ``adapt == 1`` gamma keeps
    its value; gamma is capped at ``gamma_max`` so it stays below 2 (the
    relaxation range [1, 2) of Sec. "The iterations").
    """
    hv, hh, vhvh, gv, gg, vv = dots
    eps = opts["eps_corr"]
    a_corr = _corr(hv, hh, vhvh)
    b_corr = _corr(gv, gg, vv)
    a_ok = a_corr > eps
    b_ok = b_corr > eps
    if a_ok:
        a_hat = _spectral(hv, hh, vhvh)
    if b_ok:
        b_hat = _spectral(gv, gg, vv)
    if a_ok and b_ok:
        r = math.sqrt(a_hat * b_hat)
        g, case = 1.0 + 2.0 * r / (a_hat + b_hat), 1
    elif a_ok:
        r, g, case = a_hat, 1.9, 2
    elif b_ok:
        r, g, case = b_hat, 1.1, 3
    else:
        r, g, case = rho, 1.5, 4
    if opts["adapt"] == 1:
        g = gamma
    g = min(g, opts["gamma_max"])
    return r, g, case


# --------------------------------------------------------------------------
# Stopping quantities (Eqs. feas_stop, obj_stop)
# --------------------------------------------------------------------------
def feasibility(s, set_spec):
    """r_feas_i = ||A_i x - P_Ci(A_i x)|| / ||A_i x|| (Eq. feas_stop), given
    s = A_i x.  Reading: when ||A_i x|| = 0 the unnormalised distance is
    returned."""
    d = float(np.linalg.norm(s - prox.project(set_spec, s)))
    n = float(np.linalg.norm(s))
    return d / n if n > 0.0 else d


def evolution(x, history):
    """r_evol = max_j ||x^k - x^{k-j}|| / ||x^k|| over the stored previous
    iterates (Eq. obj_stop).  Reading: 0 when ||x^k|| = 0 and no history."""
    n = float(np.linalg.norm(x))
    if not history:
        return 0.0
    d = max(float(np.linalg.norm(x - h)) for h in history)
    return d / n if n > 0.0 else d


# --------------------------------------------------------------------------
# Algorithm PARSDMM
# --------------------------------------------------------------------------
def _blocks(grid, sets, form):
    blocks = [dict(s) for s in sets]
    if form == "alg1":
        blocks.append({"op": "I", "type": "dist"})
    elif form != "direct":
        raise ValueError("unknown form %r" % (form,))
    for b in blocks:
        b["M"] = ops.out_size(grid, b["op"])
    return blocks


def parsdmm(m, grid, sets, opts=None, init=None, rho_schedule=None,
            gamma_schedule=None, resolve=True, init_rho=None, init_gamma=None,
            init_k0=None):
    """Project m onto the intersection of {x : A_i x in C_i}, Algorithm
    PARSDMM with the iterations of Eq. SDMM_adaptive.

    Per iteration k = 1, 2, ... (the paper's x^{k+1} is called x^(k) here):
      1. b = sum_i A_i^T (rho_i y_i + v_i); x = CG(C, b, warm start x).
         Form "direct" (distance term kept in the x-step, no block p+1):
         C = I + sum_i rho_i A_i^T A_i, b = m + sum_i A_i^T(rho_i y_i + v_i).
      2. for every block: s_i = A_i x; xbar_i = gamma_i s_i + (1-gamma_i) y_i;
         y_i = prox_i(xbar_i - v_i / rho_i); v_i += rho_i (y_i - xbar_i).
      3. when k % check_every == 0: r_feas_i (Eq. feas_stop) and r_evol
         (Eq. obj_stop); stop if requested and Eq. stopping_conditions holds.
      4. when adapting and k % adapt_every == 1 % adapt_every: Algorithm
         adapt-rho-gamma for every block, then C follows from the new rho
         (Eq. C_update; here C is rebuilt from its definition, Eq. sys_mat).

    Readings: the initial state is all zeros (x, y_i, v_i), as the paper
    states for the coarsest multilevel grid, unless ``init`` gives
    (x, [y_i], [v_i]); the denominator typo of the identity-block prox in
    Algorithm PARSDMM is read as (1 + rho_{p+1}) per Eq. prox_sq_dist; the
    first adapt-rho-gamma call only stores the k0 quantities; after every
    adapt step rho_i (i <= p) is clipped to [rho_{p+1}/R, rho_{p+1} R]
    (direct form: [1/R, R]) with R = rho_ratio_max.

    ``rho_schedule`` / ``gamma_schedule`` ([max_iter, blocks]) replay the
    values used in each iteration instead of adapting them.  ``init_rho`` /
    ``init_gamma`` (one value per block) replace rho0 / gamma0 as the
    starting values of a warm start that carries the penalties over
    (reading: adapt-rho-gamma then proceeds from them as from rho0).
    ``init_k0`` (one (vhat, v, s, y) tuple per block, as returned in ``k0``)
    gives the quantities Algorithm adapt-rho-gamma saved at its last call
    ("save for next call"), so that the first call of this run forms its
    differences against them instead of only saving.
    Returns a dict with x, y, v, rho, gamma, iters, cg_steps, stop_reason,
    r_feas, r_evol, k0 (the saved quantities at the end) and a per-iteration
    ``trace``.
    """
    o = options() if opts is None else dict(opts)
    m = np.asarray(m, dtype=np.float64).reshape(-1)
    N = ops.grid_size(grid)
    if m.size != N:
        raise ValueError("m has %d entries, grid has %d" % (m.size, N))
    rsets = resolve_sets(grid, sets, m) if resolve else [dict(s) for s in sets]
    blocks = _blocks(grid, rsets, o["form"])
    nb = len(blocks)
    p = len(rsets)
    alg1 = o["form"] == "alg1"

    if init is None:
        x = np.zeros(N)
        y = [np.zeros(b["M"]) for b in blocks]
        v = [np.zeros(b["M"]) for b in blocks]
    else:
        x = np.array(init[0], dtype=np.float64).reshape(-1)
        y = [np.array(a, dtype=np.float64).reshape(-1) for a in init[1]]
        v = [np.array(a, dtype=np.float64).reshape(-1) for a in init[2]]
    rho = np.full(nb, float(o["rho0"])) if init_rho is None else np.array(init_rho, dtype=np.float64)
    gamma = np.full(nb, float(o["gamma0"])) if init_gamma is None else np.array(init_gamma, dtype=np.float64)
    if rho.shape != (nb,) or gamma.shape != (nb,):
        raise ValueError("init_rho / init_gamma need one value per block")
    k0 = [None] * nb              # saved (vhat, v, s, y) of the last adapt call
    if init_k0 is not None:
        if len(init_k0) != nb:
            raise ValueError("init_k0 needs one tuple per block")
        k0 = [None if t is None else tuple(np.array(a, dtype=np.float64).reshape(-1) for a in t)
              for t in init_k0]
    history = []                  # previous iterates for Eq. obj_stop
    trace = []
    cg_total = 0
    stop_reason = 0
    r_feas = [float("nan")] * p
    r_evol = float("nan")
    it = 0
    for k in range(1, int(o["max_iter"]) + 1):
        it = k
        if rho_schedule is not None:
            rho = np.array(rho_schedule[k - 1], dtype=np.float64)
        if gamma_schedule is not None:
            gamma = np.array(gamma_schedule[k - 1], dtype=np.float64)
        rho_used = rho.copy()
        gamma_used = gamma.copy()

        # 1. x-update
        b = np.zeros(N)
        for i, blk in enumerate(blocks):
            b = b + ops.apply_t(grid, blk["op"], rho[i] * y[i] + v[i])
        c_id = 0.0 if alg1 else 1.0
        if not alg1:
            b = b + m
        cg_ops = [blk["op"] for blk in blocks]
        apply_c = lambda z: ops.system_apply(grid, cg_ops, rho, c_id, z)
        x_prev = x
        x, steps = cg(apply_c, b, x, int(o["cg_iters"]), int(o["cg_max"]))
        cg_total += steps

        # 2. per-block relaxation, prox and dual update
        s_all, y_old, v_old = [], y, v
        y_new, v_new = [], []
        for i, blk in enumerate(blocks):
            s = ops.apply(grid, blk["op"], x)
            xbar = gamma[i] * s + (1.0 - gamma[i]) * y[i]
            w = xbar - v[i] / rho[i]
            if blk["type"] == "dist":
                yi = prox.prox_dist(w, m, rho[i])
            else:
                yi = prox.project(blk, w)
            vi = v[i] + rho[i] * (yi - xbar)
            s_all.append(s)
            y_new.append(yi)
            v_new.append(vi)
        y, v = y_new, v_new

        # 3. stopping quantities
        history.append(x_prev)
        history = history[-int(o["evol_hist"]):]
        rec = {"k": k, "rho": rho_used, "gamma": gamma_used, "cg_steps": steps}
        if k % int(o["check_every"]) == 0:
            r_feas = [feasibility(s_all[i], blocks[i]) for i in range(p)]
            r_evol = evolution(x, history)
            rec["r_feas"] = list(r_feas)
            rec["r_evol"] = r_evol
            feas_ok = all(f < o["eps_feas"] for f in r_feas)
            if (o["stop"] == 1 and feas_ok and r_evol < o["eps_evol"]) or \
               (o["stop"] == 2 and feas_ok):
                trace.append(rec)
                stop_reason = 1
                break
        trace.append(rec)

        # 4. Algorithm adapt-rho-gamma
        f = int(o["adapt_every"])
        if o["adapt"] and rho_schedule is None and k % f == 1 % f:
            new_rho = rho.copy()
            new_gamma = gamma.copy()
            cases = []
            for i in range(nb):
                vhat = v_old[i] + rho[i] * (y_old[i] - s_all[i])
                cur = (vhat, v[i], s_all[i], y[i])
                if k0[i] is not None:
                    vh0, v0, s0, y0 = k0[i]
                    dvh = vhat - vh0
                    dv = v[i] - v0
                    dh = s_all[i] - s0
                    dg = -(y[i] - y0)
                    dots = (float(dh @ dvh), float(dh @ dh), float(dvh @ dvh),
                            float(dg @ dv), float(dg @ dg), float(dv @ dv))
                    new_rho[i], new_gamma[i], c = adapt_rho_gamma(dots, rho[i], gamma[i], o)
                    cases.append(c)
                k0[i] = cur
            R = float(o["rho_ratio_max"])
            ref = new_rho[p] if alg1 else 1.0
            for i in range(p):
                new_rho[i] = min(max(new_rho[i], ref / R), ref * R)
            rho, gamma = new_rho, new_gamma
            rec["adapt_cases"] = cases

    return dict(x=x, y=y, v=v, rho=rho, gamma=gamma, iters=it,
                cg_steps=cg_total, stop_reason=stop_reason, r_feas=r_feas,
                r_evol=r_evol, trace=trace, sets=rsets, blocks=blocks, k0=k0)


# --------------------------------------------------------------------------
# ML-PARSDMM (Algorithm ML-PARSDMM, Sec. "Multilevel PARSDMM")
# --------------------------------------------------------------------------
def coarse_grid(grid):
    """Coarsen every axis by 2 (n_c = ceil(n/2)); the spacing doubles.

    Reading: the paper fixes neither the coarsening factor nor the coarse
    spacing; factor 2 and h_c = 2 h keep derivative quantities on the same
    physical scale on both levels."""
    n = tuple(int(v) for v in grid["n"])
    h = tuple(float(v) for v in grid.get("h", (1.0,) * len(n)))
    return {"n": tuple((v + 1) // 2 for v in n), "h": tuple(2.0 * v for v in h)}


def restrict(grid, m):
    """Coarse model m_l: anti-alias filter plus subsampling, read as the
    average over each 2 x 2 (x 2) block of fine cells (a box filter followed
    by taking one sample per block).  Odd sizes: the last block averages the
    cells it has."""
    fs = ops.grid_shape(grid)
    cg_ = coarse_grid(grid)
    cs = ops.grid_shape(cg_)
    M = np.asarray(m, dtype=np.float64).reshape(fs)
    out = np.zeros(cs)
    cnt = np.zeros(cs)
    nd = len(grid["n"])
    for dy in ((0, 1) if nd > 2 else (0,)):
        for dx in (0, 1):
            for dz in (0, 1):
                sub = M[dy::2 if nd > 2 else 1, dx::2, dz::2]
                out[:sub.shape[0], :sub.shape[1], :sub.shape[2]] += sub
                cnt[:sub.shape[0], :sub.shape[1], :sub.shape[2]] += 1.0
    return (out / cnt).reshape(-1)


def _interp_axis(A, axis, n_fine, staggered):
    """Linear interpolation along one axis from a coarse to a fine grid.

    Positions in fine-cell units: fine sample i sits at i (+ 1/2 for a
    staggered, difference-output axis); coarse sample j sits at 2 j + 1/2
    (+ 1 for a staggered axis), the centre of the fine cells it covers.
    The two nearest coarse samples are combined linearly, extrapolating
    linearly past the ends, so linear fields are reproduced exactly."""
    nc = A.shape[axis]
    A = np.moveaxis(A, axis, -1)
    if nc == 1:
        out = np.repeat(A, n_fine, axis=-1)
        return np.moveaxis(out, -1, axis)
    off = 0.5 if staggered else 0.0
    pf = np.arange(n_fine) + off
    t = (pf - 0.5 - 2.0 * off) / 2.0          # continuous coarse index
    j0 = np.clip(np.floor(t).astype(np.int64), 0, nc - 2)
    f = t - j0
    out = A[..., j0] * (1.0 - f) + A[..., j0 + 1] * f
    return np.moveaxis(out, -1, axis)


def prolong(grid_c, grid_f, op, u):
    """Interpolate a vector living on the output grid of operator ``op`` at
    the coarse level to the same operator's output grid at the fine level
    ("interpolate y_i and v_i as images", Sec. "Multilevel PARSDMM").
    Separable (bi/tri)linear interpolation; the differenced axis of a D
    operator is staggered by half a cell."""
    u = np.asarray(u, dtype=np.float64).reshape(-1)
    if op == "TV":
        parts = []
        off = 0
        for d in ops.tv_parts(grid_c):
            mc = ops.out_size(grid_c, d)
            parts.append(prolong(grid_c, grid_f, d, u[off:off + mc]))
            off += mc
        return np.concatenate(parts)
    if op == "I":
        cshape, fshape, stag = ops.grid_shape(grid_c), ops.grid_shape(grid_f), None
    else:
        cshape, fshape = ops.diff_shape(grid_c, op), ops.diff_shape(grid_f, op)
        stag = {"DZ": 2, "DX": 1, "DY": 0}[op]
    A = u.reshape(cshape)
    for ax in range(3):
        A = _interp_axis(A, ax, fshape[ax], stag == ax)
    return A.reshape(-1)


def ml_parsdmm(m, grid, sets, opts=None, levels=2, coarse_iter=None):
    """Algorithm ML-PARSDMM: solve from the coarsest grid to the finest
    without cycling; every level starts from the interpolated x, y_i, v_i
    of the level below; the coarsest starts from zeros.

    Readings: m_l comes from ``restrict``; set radii and cardinalities are
    resolved per level from m_l (relative parameters) and the level's grid
    size; rho and gamma restart from rho0 / gamma0 on every level;
    ``coarse_iter`` (default: the fine max_iter) iterations on coarse levels.
    """
    o = options() if opts is None else dict(opts)
    if levels > 1 and any(s["op"] == "BLUR" or ops.is_blur(s["op"]) for s in sets):
        # reading: the paper's multilevel scheme interpolates y_i, v_i as
        # images; a blur's taps have no stated coarse-grid counterpart
        raise ValueError("a blur operator runs on one level only")
    grids = [grid]
    ms = [np.asarray(m, dtype=np.float64).reshape(-1)]
    for _ in range(levels - 1):
        ms.append(restrict(grids[-1], ms[-1]))
        grids.append(coarse_grid(grids[-1]))
    init = None
    res = None
    per_level = []
    for lev in range(levels - 1, -1, -1):
        ol = dict(o)
        if lev > 0 and coarse_iter is not None:
            ol["max_iter"] = int(coarse_iter)
        res = parsdmm(ms[lev], grids[lev], sets, ol, init=init)
        per_level.append(res)
        if lev > 0:
            gc, gf = grids[lev], grids[lev - 1]
            x_f = prolong(gc, gf, "I", res["x"])
            y_f = [prolong(gc, gf, b["op"], yy) for b, yy in zip(res["blocks"], res["y"])]
            v_f = [prolong(gc, gf, b["op"], vv) for b, vv in zip(res["blocks"], res["v"])]
            init = (x_f, y_f, v_f)
    res = dict(res)
    res["levels"] = per_level
    return res
