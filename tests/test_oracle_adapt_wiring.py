"""Pin for how oracle/parsdmm.py feeds Algorithm adapt-rho-gamma.

adapt_rho_gamma() itself (the correlations, spectral steps and the four
cases of the algorithm's table) is pinned in test_oracle_parsdmm.py.  This
file pins its inputs: which iterates form v-hat and the four differences,
and what is kept from the previous call (the k0 quantities).

The check is a second PARSDMM loop written here with a different structure:
it keeps every iterate x^k, y_i^k, v_i^k, s_i^k = A_i x^k in a list and, at
an adapt iteration, forms the algorithm's quantities straight from their
definitions by indexing that list, with k0 the previous adapt iteration:

    vhat^{k+1} = v^k + rho^k (y^k - s^{k+1})
    dvh = vhat^{k+1} - vhat^{k0},  dv = v^{k+1} - v^{k0}
    dh  = s^{k+1} - s^{k0},        dg = -(y^{k+1} - y^{k0})

The first call only records (reading of the first call), rho_i is kept in
[rho_{p+1}/R, rho_{p+1} R] after every call (reading of the rho safeguard).
The oracle's rho / gamma trajectory must equal this loop's.  The case is
chosen so that each of these slips changes the trajectory: y^{k+1} in
place of y^k in vhat, v^{k+1} in place of v^k in vhat, and the k0 copy
stored before the differences are formed.
"""
import numpy as np
import pytest

from oracle import operators as ops
from oracle import parsdmm as P
from oracle import prox


def hand_loop(m, grid, sets, o):
    rs = P.resolve_sets(grid, sets, m)
    blocks = rs + [{"op": "I", "type": "dist"}]
    nb, p = len(blocks), len(rs)
    N = ops.grid_size(grid)
    X = [np.zeros(N)]
    Y = [[np.zeros(ops.out_size(grid, b["op"])) for b in blocks]]
    V = [[np.zeros(ops.out_size(grid, b["op"])) for b in blocks]]
    S = [None]
    rho = np.full(nb, float(o["rho0"]))
    gamma = np.full(nb, float(o["gamma0"]))
    used = [None]          # (rho, gamma) used in iteration k
    calls = []             # adapt iterations so far
    cases = {}
    f = int(o["adapt_every"])
    for k in range(1, int(o["max_iter"]) + 1):
        used.append((rho.copy(), gamma.copy()))
        opl = [b["op"] for b in blocks]
        b = sum(ops.apply_t(grid, opl[i], rho[i] * Y[k - 1][i] + V[k - 1][i]) for i in range(nb))
        x, _ = P.cg(lambda z: ops.system_apply(grid, opl, rho, 0.0, z), b, X[k - 1], int(o["cg_iters"]),
                    int(o["cg_max"]))
        s = [ops.apply(grid, opl[i], x) for i in range(nb)]
        yk, vk = [], []
        for i, blk in enumerate(blocks):
            xbar = gamma[i] * s[i] + (1.0 - gamma[i]) * Y[k - 1][i]
            w = xbar - V[k - 1][i] / rho[i]
            yi = prox.prox_dist(w, m, rho[i]) if blk["type"] == "dist" else prox.project(blk, w)
            yk.append(yi)
            vk.append(V[k - 1][i] + rho[i] * (yi - xbar))
        X.append(x)
        Y.append(yk)
        V.append(vk)
        S.append(s)
        if k % f != 1 % f:
            continue
        calls.append(k)
        if len(calls) < 2:
            continue
        k0 = calls[-2]

        def vhat(j, i):
            return V[j - 1][i] + used[j][0][i] * (Y[j - 1][i] - S[j][i])
        new_rho, new_gamma = rho.copy(), gamma.copy()
        for i in range(nb):
            dvh = vhat(k, i) - vhat(k0, i)
            dv = V[k][i] - V[k0][i]
            dh = S[k][i] - S[k0][i]
            dg = -(Y[k][i] - Y[k0][i])
            dots = (dh @ dvh, dh @ dh, dvh @ dvh, dg @ dv, dg @ dg, dv @ dv)
            new_rho[i], new_gamma[i], cases[(k, i)] = P.adapt_rho_gamma(dots, rho[i], gamma[i], o)
        R = float(o["rho_ratio_max"])
        for i in range(p):
            new_rho[i] = min(max(new_rho[i], new_rho[p] / R), new_rho[p] * R)
        rho, gamma = new_rho, new_gamma
    return X[-1], used[1:], cases


CASE = dict(n=(4, 3), seed=3)


def _case(rho_ratio_max=1e3):
    grid = {"n": CASE["n"], "h": (1.0, 1.0)}
    rg = np.random.default_rng(CASE["seed"])
    m = 3.0 + 1.2 * rg.standard_normal(int(np.prod(CASE["n"])))
    sets = [{"op": "I", "type": "bounds", "lo": 2.0, "hi": 4.0},
            {"op": "TV", "type": "l1", "sigma_rel": 0.3}]
    o = P.options(max_iter=8, cg_iters=5, adapt=2, adapt_every=2, rho0=1.0, gamma0=1.5,
                  rho_ratio_max=rho_ratio_max)
    return m, grid, sets, o


@pytest.mark.parametrize("rho_ratio_max", [1e3, 1.5])
def test_adapt_inputs_follow_the_algorithm(rho_ratio_max):
    m, grid, sets, o = _case(rho_ratio_max)
    res = P.parsdmm(m, grid, sets, o)
    x_h, used, cases = hand_loop(m, grid, sets, o)
    assert len(res["trace"]) == len(used) == o["max_iter"]
    for rec, (rh, gh) in zip(res["trace"], used):
        np.testing.assert_allclose(rec["rho"], rh, rtol=1e-12, atol=0)
        np.testing.assert_allclose(rec["gamma"], gh, rtol=1e-12, atol=0)
    np.testing.assert_allclose(res["x"], x_h, rtol=1e-12, atol=1e-12)
    # the trajectory must actually move: some block leaves case 4 (no
    # correlation) and changes rho and gamma, so a slip in the inputs shows
    assert any(c != 4 for c in cases.values())
    assert not np.allclose(used[-1][0], used[0][0])
    assert not np.allclose(used[-1][1], used[0][1])


def test_rho_safeguard_binds_in_the_clamped_case():
    """With R = 1.5 the safeguard must act at least once (otherwise the
    clamped case would not test it)."""
    m, grid, sets, o = _case(1.5)
    _, used_c, _ = hand_loop(m, grid, sets, o)
    m, grid, sets, o = _case(1e3)
    _, used_f, _ = hand_loop(m, grid, sets, o)
    assert not np.allclose(used_c[-1][0], used_f[-1][0])
    for rh, _ in used_c:
        assert np.all(rh[:-1] <= rh[-1] * 1.5 * (1 + 1e-15))
        assert np.all(rh[:-1] >= rh[-1] / 1.5 * (1 - 1e-15))
