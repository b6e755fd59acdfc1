"""Loop parity: the CUDA PARSDMM loop against the FP64 oracle on the same
seeded inputs, under a fixed iteration count and a deterministic rho
schedule, through the C ABI.

Bars: ||x_gpu - x_oracle|| / ||x_oracle|| <= 1e-10 in FP64 and <= 1e-4 in
FP32 (FP32 runs replay the oracle's rho/gamma schedule so binary32 rounding
cannot flip an adapt-rho-gamma branch).  The FP64 GPU loop also runs its own
adapt-rho-gamma, whose rho trajectory must match the oracle's to 1e-9.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import operators as O                 # noqa: E402
from oracle import parsdmm as P                   # noqa: E402
from paper_1902_09699_gb300 import sip            # noqa: E402
from paper_1902_09699_gb300 import workloads as W  # noqa: E402

TD = {"f64": torch.float64, "f32": torch.float32}
BAR = {"f64": 1e-10, "f32": 1e-4}


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run_gpu(m, grid, sets, dt, opts, rho_schedule=None, gamma_schedule=None, trace=False):
    pr = sip.Projector(grid, sets, dtype=dt, rho_schedule=rho_schedule, gamma_schedule=gamma_schedule,
                       trace=trace, **opts)
    x, info = pr.project(torch.as_tensor(m, dtype=TD[dt], device="cuda"))
    out = x.double().cpu().numpy(), info, (pr.trace.copy() if trace else None)
    pr.close()
    return out


def oracle_run(m, grid, sets, opts, **kw):
    o = P.options(**opts)
    return P.parsdmm(m, grid, sets, o, **kw)


def schedules(res):
    rs = np.array([t["rho"] for t in res["trace"]])
    gs = np.array([t["gamma"] for t in res["trace"]])
    return rs, gs


def m_as(m, dt):
    return torch.as_tensor(m, dtype=TD[dt]).double().numpy()


# ---------------------------------------------------------------- 64 x 64 FP64
def test_small_2d_fp64_fixed_rho():
    c = W.small_2d()
    ref = oracle_run(c["m"], c["grid"], c["sets"], c["opts"])
    x, info, _ = run_gpu(c["m"], c["grid"], c["sets"], "f64", c["opts"])
    assert info["iters"] == 200
    assert rel(x, ref["x"]) <= 1e-10
    for a, b in zip(info["r_feas"], ref["r_feas"]):
        assert a == pytest.approx(b, rel=1e-8, abs=1e-14)
    assert info["r_evol"] == pytest.approx(ref["r_evol"], rel=1e-8)
    assert info["cg_steps"] == ref["cg_steps"]


def test_small_2d_fp32():
    c = W.small_2d()
    m32 = m_as(c["m"], "f32")
    ref = oracle_run(m32, c["grid"], c["sets"], c["opts"])
    x, info, _ = run_gpu(m32, c["grid"], c["sets"], "f32", c["opts"])
    assert rel(x, ref["x"]) <= 1e-4


# ---------------------------------------------------------------- config-2 set list, reduced grid
def layered_small(n=(96, 128)):
    c = W.layered_2d(n=n, seed=77)
    c["opts"] = dict(c["opts"], max_iter=60)
    return c


def test_layered_fp64_own_adapt_matches_oracle():
    c = layered_small()
    ref = oracle_run(c["m"], c["grid"], c["sets"], c["opts"])
    x, info, tr = run_gpu(c["m"], c["grid"], c["sets"], "f64", c["opts"], trace=True)
    rs, _ = schedules(ref)
    nb = len(c["sets"]) + 1
    assert np.ptp(rs) > 0, "rho must move in this case"
    assert np.allclose(tr[:, :nb], rs, rtol=1e-9, atol=0)
    assert rel(x, ref["x"]) <= 1e-10
    assert info["k"][3] == math.floor(0.02 * 96 * 128)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_layered_replayed_schedule(dt):
    # The cardinality set is not convex: at near-ties of the k-th value its
    # support can change under a one-ulp change of the input, and a binary32
    # run over 60 iterations can meet such a tie where binary64 does not (on
    # this case one binary32 trajectory in five did).  Binary32 therefore
    # runs the convex sets of the list; binary64 runs all of them.
    c = layered_small()
    sets = c["sets"] if dt == "f64" else [s for s in c["sets"] if s["type"] != "card"]
    m = m_as(c["m"], dt)
    ref = oracle_run(m, c["grid"], sets, c["opts"])
    rs, gs = schedules(ref)
    x, info, _ = run_gpu(m, c["grid"], sets, dt, c["opts"], rho_schedule=rs, gamma_schedule=gs)
    assert rel(x, ref["x"]) <= BAR[dt]


@pytest.mark.parametrize("mode", ["graph", "persistent", "cluster"])
def test_execution_modes_agree_with_oracle(mode):
    # both ways of running the iterations: one kernel per phase replayed from
    # a CUDA graph, and one cooperative kernel with grid barriers
    c = layered_small((72, 100))
    ref = oracle_run(c["m"], c["grid"], c["sets"], c["opts"])
    x, info, tr = run_gpu(c["m"], c["grid"], c["sets"], "f64", dict(c["opts"], exec=mode), trace=True)
    rs, _ = schedules(ref)
    nb = len(c["sets"]) + 1
    assert np.allclose(tr[:, :nb], rs, rtol=1e-9, atol=0)
    assert rel(x, ref["x"]) <= 1e-10
    c2 = W.small_2d(n=(40, 36), seed=3)
    opts = dict(max_iter=2000, adapt=1, gamma0=1.5, stop=1, exec=mode)
    ref2 = oracle_run(c2["m"], c2["grid"], c2["sets"][::2], {k: v for k, v in opts.items() if k != "exec"})
    x2, info2, _ = run_gpu(c2["m"], c2["grid"], c2["sets"][::2], "f64", opts)
    assert info2["iters"] == ref2["iters"] and rel(x2, ref2["x"]) <= 1e-10


def test_adapt_rho_and_gamma_full_algorithm():
    c = layered_small((40, 56))
    opts = dict(c["opts"], adapt=2, max_iter=40)
    ref = oracle_run(c["m"], c["grid"], c["sets"], opts)
    x, info, tr = run_gpu(c["m"], c["grid"], c["sets"], "f64", opts, trace=True)
    rs, gs = schedules(ref)
    nb = len(c["sets"]) + 1
    assert np.allclose(tr[:, :nb], rs, rtol=1e-9)
    assert np.allclose(tr[:, nb:2 * nb], gs, rtol=1e-9)
    assert rel(x, ref["x"]) <= 1e-10


def test_direct_form():
    c = layered_small((48, 40))
    opts = dict(c["opts"], form="direct", max_iter=50)
    ref = oracle_run(c["m"], c["grid"], c["sets"], opts)
    x, info, _ = run_gpu(c["m"], c["grid"], c["sets"], "f64", opts)
    assert rel(x, ref["x"]) <= 1e-10


# ---------------------------------------------------------------- 3D and multilevel
def grf3(n=(20, 16, 12)):
    c = W.grf_3d(n=n, seed=33)
    c["opts"] = dict(c["opts"], max_iter=40)
    return c


def test_3d_fp64():
    c = grf3()
    ref = oracle_run(c["m"], c["grid"], c["sets"], c["opts"])
    x, info, _ = run_gpu(c["m"], c["grid"], c["sets"], "f64", c["opts"])
    assert rel(x, ref["x"]) <= 1e-10


@pytest.mark.parametrize("n,levels,adapt", [((24, 16, 12), 2, 1), ((33, 20), 2, 1), ((48, 40, 32), 3, 1),
                                            ((130, 66), 4, 1), ((97, 81), 5, 0), ((33, 20), 4, 0)])
def test_multilevel_fp64(n, levels, adapt):
    """Algorithm ML-PARSDMM over 2..5 levels (odd sizes coarsen to ceil(n/2)).
    With adaptive rho the coarsest grids keep enough samples: on a few
    samples the adapt-rho-gamma branch tests sit on exact ties, where the
    oracle itself moves by far more than 1e-10 under rounding; deeper
    hierarchies run with fixed rho."""
    c = W.grf_3d(n=n, seed=5) if len(n) == 3 else W.small_2d(n=n, seed=5)
    opts = dict(c["opts"], max_iter=30, adapt=adapt, gamma0=1.5)
    ref = P.ml_parsdmm(c["m"], c["grid"], c["sets"], P.options(**opts), levels=levels, coarse_iter=20)
    x, info, _ = run_gpu(c["m"], c["grid"], c["sets"], "f64", dict(opts, levels=levels, coarse_iter=20))
    assert rel(x, ref["x"]) <= 1e-10


# ---------------------------------------------------------------- stopping, edge cases, errors
def test_stopping_rule_iteration_count():
    c = W.small_2d(n=(32, 24), seed=9)
    opts = dict(max_iter=2000, adapt=1, gamma0=1.5, stop=1)
    sets = [c["sets"][0], c["sets"][2]]
    ref = oracle_run(c["m"], c["grid"], sets, opts)
    x, info, _ = run_gpu(c["m"], c["grid"], sets, "f64", opts)
    assert ref["stop_reason"] == 1
    assert info["stop_reason"] == 1 and info["iters"] == ref["iters"]
    assert rel(x, ref["x"]) <= 1e-10


@pytest.mark.parametrize("grid,sets", [
    ({"n": (2, 2)}, [{"op": "TV", "type": "l1", "sigma": 0.1}, {"op": "I", "type": "bounds", "lo": 0.0, "hi": 1.0}]),
    ({"n": (1, 9)}, [{"op": "DX", "type": "card", "k": 2}]),
    ({"n": (5, 1)}, [{"op": "DZ", "type": "l2", "sigma": 0.3}]),
    ({"n": (3, 2, 2)}, [{"op": "TV", "type": "l1", "sigma_rel": 0.2}, {"op": "DY", "type": "bounds", "lo": 0.0, "hi": 9.0}]),
    ({"n": (1031, 3)}, [{"op": "DZ", "type": "card", "k_frac": 0.1}, {"op": "I", "type": "l1", "sigma_rel": 0.5}]),
])
def test_degenerate_and_ragged_grids(grid, sets):
    # On grids this small adapt-rho-gamma's correlation tests sit on exact
    # ties (the oracle itself moves by 1e-3 under a 1e-15 perturbation of m
    # on the 2 x 2 case), so the rho / gamma schedule is replayed.
    g = np.random.default_rng(1)
    m = g.standard_normal(int(np.prod(grid["n"])))
    opts = dict(max_iter=25, adapt=1, gamma0=1.5)
    ref = oracle_run(m, grid, sets, opts)
    rs, gs = schedules(ref)
    x, info, _ = run_gpu(m, grid, sets, "f64", opts, rho_schedule=rs, gamma_schedule=gs)
    assert rel(x, ref["x"]) <= 1e-10


def test_repeat_calls_on_one_handle():
    c = layered_small((32, 48))
    pr = sip.Projector(c["grid"], c["sets"], dtype="f64", **c["opts"])
    m = torch.as_tensor(c["m"], device="cuda")
    x1, _ = pr.project(m)
    x2, _ = pr.project(m)
    m2 = m.flip(0).contiguous()
    x3, _ = pr.project(m2)
    x4, _ = pr.project(m)
    a, b, d = x1.cpu().numpy(), x2.cpu().numpy(), x4.cpu().numpy()
    assert rel(b, a) <= 1e-12 and rel(d, a) <= 1e-12
    ref = oracle_run(c["m"][::-1].copy(), c["grid"], c["sets"], c["opts"])
    assert rel(x3.cpu().numpy(), ref["x"]) <= 1e-10
    pr.close()


def test_nonfinite_model_rejected():
    c = W.small_2d(n=(16, 16))
    m = c["m"].copy()
    m[37] = np.nan
    pr = sip.Projector(c["grid"], c["sets"], dtype="f64", max_iter=10)
    with pytest.raises(sip.SipError) as e:
        pr.project(torch.as_tensor(m, device="cuda"))
    assert e.value.status == 5
    x, info = pr.project(torch.as_tensor(c["m"], device="cuda"))   # handle still usable
    assert info["iters"] == 10
    pr.close()


@pytest.mark.parametrize("n", [(4, 300), (12, 37), (8, 2000), (36, 129), (12, 1001)])
def test_fp32_four_sample_cg_step(n):
    """Binary32 2D grids with n_z % 4 == 0 take the CG step that loads 4
    samples of a column at once; its z neighbours come from adjacent lanes
    or, at warp and work-item edges (here inside columns: n_z = 12, 36),
    from single loads.  n_z = 4 puts every column in one group (both z ends
    missing).  Fixed rho, no selection sets: the result must track the FP64
    oracle as closely as the general step's."""
    g = np.random.default_rng(5)
    m = 3.0 + g.standard_normal(n[0] * n[1])
    grid = {"n": n}
    sets = [{"op": "I", "type": "bounds", "lo": 2.5, "hi": 3.5},
            {"op": "DZ", "type": "l2", "sigma_rel": 0.3},
            {"op": "DX", "type": "bounds", "lo": -0.5, "hi": 0.5}]
    opts = dict(max_iter=30, adapt=0, rho0=1.0, gamma0=1.5)
    m32 = m_as(m, "f32")
    ref = oracle_run(m32, grid, sets, opts)
    x, info, _ = run_gpu(m32, grid, sets, "f32", opts)
    assert info["cg_steps"] == ref["cg_steps"]
    assert rel(x, ref["x"]) <= 5e-5


# ---------------------------------------------------------------- full size 512 x 1024
def test_full_size_layered_first_iterations():
    """The 512 x 1024 five-set workload in the bench launch configuration:
    a few iterations compared whole against the oracle."""
    c = W.layered_2d()
    opts = dict(c["opts"], max_iter=6)
    ref = oracle_run(c["m"], c["grid"], c["sets"], opts)
    x, info, _ = run_gpu(c["m"], c["grid"], c["sets"], "f64", opts)
    assert rel(x, ref["x"]) <= 1e-10
    m32 = m_as(c["m"], "f32")
    ref32 = oracle_run(m32, c["grid"], c["sets"], opts)
    rs, gs = schedules(ref32)
    x, info, _ = run_gpu(m32, c["grid"], c["sets"], "f32", opts, rho_schedule=rs, gamma_schedule=gs)
    assert rel(x, ref32["x"]) <= 1e-4


@pytest.mark.parametrize("hist,every", [(5, 2), (2, 2), (3, 1)])
def test_adapt_k0_quantities_ring_or_copy(hist, every):
    """Algorithm adapt-rho-gamma compares s = A_i x with its value at the
    previous adapt iteration k0.  With adapt_every < evol_hist, s^{k0} is
    recomputed from x^{k0} in the x history ring; otherwise a copy is kept.
    Either way the rho trajectory and x follow the oracle."""
    c = layered_small()
    opts = dict(c["opts"], evol_hist=hist, adapt_every=every)
    ref = oracle_run(c["m"], c["grid"], c["sets"], opts)
    x, info, tr = run_gpu(c["m"], c["grid"], c["sets"], "f64", opts, trace=True)
    rs, _ = schedules(ref)
    nb = len(c["sets"]) + 1
    assert np.ptp(rs) > 0
    assert np.allclose(tr[:, :nb], rs, rtol=1e-9, atol=0)
    assert rel(x, ref["x"]) <= 1e-10


# ---------------------------------------------------------------- Eq. cg_stop (adaptive CG steps)
@pytest.mark.parametrize("case", ["small_fixed_rho", "layered_adaptive_rho"])
def test_adaptive_cg_rule_matches_oracle(case):
    # cg_iters = 0: each x-update stops once ||r_j|| < 0.1 ||r_0|| (the reading
    # of Eq. cg_stop), at most cg_max steps; the per-iteration step counts
    # must equal the oracle's and x must match it in FP64
    if case == "small_fixed_rho":
        c = W.small_2d()
        opts = dict(c["opts"], max_iter=60, cg_iters=0, cg_max=100)
    else:
        c = layered_small((64, 80))
        opts = dict(c["opts"], max_iter=40, cg_iters=0, cg_max=100)
    ref = oracle_run(c["m"], c["grid"], c["sets"], opts)
    x, info, tr = run_gpu(c["m"], c["grid"], c["sets"], "f64", opts, trace=True)
    nb = info["nblocks"] if "nblocks" in info else len(c["sets"]) + 1
    steps_ref = np.array([t["cg_steps"] for t in ref["trace"]])
    steps_gpu = tr[:, 2 * nb].astype(int)
    assert steps_ref.max() > 1 and np.ptp(steps_ref) > 0, "the rule must vary the step count here"
    assert np.array_equal(steps_gpu, steps_ref)
    assert info["cg_steps"] == ref["cg_steps"]
    assert rel(x, ref["x"]) <= 1e-10


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("n", [(36, 64), (37, 20)], ids=["nz4", "nz37"])
@pytest.mark.parametrize("cg", [1, 2, 3])
def test_cg_step_counts(cg, n, dt):
    """The first step launch of an iteration (beta = 0: p and s are not read)
    and the last (only x is formed) are kernels of their own.  With one step
    the last launch is also the first (it takes the right-hand side's and
    w_0's sums); with two the x-only launch follows the first directly.
    n_z = 36 takes the four-sample kernels in binary32, n_z = 37 the general
    ones.  Fixed rho: FP64 within 1e-10 of the oracle, FP32 within the
    four-sample step test's 5e-5, and the same number of CG steps."""
    g = np.random.default_rng(31 + cg)
    m = 3.0 + g.standard_normal(n[0] * n[1])
    grid = {"n": n}
    sets = [{"op": "I", "type": "bounds", "lo": 2.5, "hi": 3.5},
            {"op": "TV", "type": "l1", "sigma_rel": 0.4},
            {"op": "DZ", "type": "bounds", "lo": -0.5, "hi": 0.5}]
    opts = dict(max_iter=30, cg_iters=cg, adapt=0, rho0=1.0, gamma0=1.5)
    mm = m_as(m, dt)
    ref = oracle_run(mm, grid, sets, opts)
    x, info, _ = run_gpu(mm, grid, sets, dt, opts)
    # every iteration takes cg steps but the first (y = v = 0 there, so b and
    # r_0 are zero and no step is taken)
    assert info["cg_steps"] == ref["cg_steps"] == 29 * cg
    assert rel(x, ref["x"]) <= (1e-10 if dt == "f64" else 5e-5)


def test_full_size_fp32_tracks_fp64_while_supports_hold():
    """The 512 x 1024 five-set workload, FP32 against the FP64 GPU loop (each
    with its own adapt-rho-gamma) in the bench launch configuration.  The
    cardinality set's support amplifies binary32-sized perturbations: the two
    stay within 2e-7 for the first 35 iterations and part after about 40
    (measured; the FP64 loop with its state rounded to binary32 after every
    iteration parts the same way later).  Gate: 30 iterations with all five
    sets, and 500 iterations with the four convex sets."""
    c = W.layered_2d()
    for sets, its, bar in ((c["sets"], 30, 1e-5),
                           ([s for s in c["sets"] if s["type"] != "card"], 500, 1e-5)):
        opts = dict(c["opts"], max_iter=its)
        x64, _, _ = run_gpu(c["m"], c["grid"], sets, "f64", opts)
        x32, _, _ = run_gpu(c["m"], c["grid"], sets, "f32", opts)
        assert rel(x32, x64) <= bar, (len(sets), its)


# ---------------------------------------------------------------- cluster execution
@pytest.mark.parametrize("ctas", [1, 4, 16])
def test_cluster_execution_small_fp64(ctas):
    """The 64 x 64 FP64 workload on one thread-block cluster of 1, 4 or 16
    CTAs (all 200 iterations in one launch) against the oracle."""
    c = W.small_2d()
    ref = oracle_run(c["m"], c["grid"], c["sets"], c["opts"])
    x, info, tr = run_gpu(c["m"], c["grid"], c["sets"], "f64", dict(c["opts"], exec="cluster", cluster_ctas=ctas),
                          trace=True)
    assert info["iters"] == 200
    assert rel(x, ref["x"]) <= 1e-10
    assert info["cg_steps"] == ref["cg_steps"]
    for a, b in zip(info["r_feas"], ref["r_feas"]):
        assert a == pytest.approx(b, rel=1e-8, abs=1e-14)


def test_cluster_execution_stopping_rule_and_fp32():
    """Cluster execution with the feasibility stopping rule (each instance
    leaves the loop on its own) and in FP32 with a replayed schedule."""
    c = layered_small((48, 64))
    opts = dict(c["opts"], max_iter=200, stop=2, eps_feas=5e-2, exec="cluster", cluster_ctas=4)
    ref = oracle_run(c["m"], c["grid"], c["sets"], {k: v for k, v in opts.items() if k not in ("exec", "cluster_ctas")})
    x, info, _ = run_gpu(c["m"], c["grid"], c["sets"], "f64", opts)
    assert info["iters"] == ref["iters"] < 200
    assert rel(x, ref["x"]) <= 1e-10
    sets = [s_ for s_ in c["sets"] if s_["type"] != "card"]
    o32 = dict(c["opts"], exec="cluster", cluster_ctas=8)
    m = m_as(c["m"], "f32")
    ref32 = oracle_run(m, c["grid"], sets, c["opts"])
    rs, gs = schedules(ref32)
    x, info, _ = run_gpu(m, c["grid"], sets, "f32", o32, rho_schedule=rs, gamma_schedule=gs)
    assert rel(x, ref32["x"]) <= 1e-4


def test_multilevel_3d_reduced_at_full_iteration_counts():
    """The 3D four-set workload (bounds, 3D TV l1 ball, D_z x >= 0, card(D_x x)
    at 1% of N) on a reduced 48 x 48 x 24 grid with its full iteration counts:
    two levels, 300 coarse + 300 fine iterations, FP64, adaptive rho, against
    the oracle.  The per-set feasibility must be the oracle's, so the r_feas a
    full-size run ends with is the method's at that iteration count."""
    c = W.grf_3d(n=(48, 48, 24), seed=1003)
    opts = dict(c["opts"])
    ref = P.ml_parsdmm(c["m"], c["grid"], c["sets"], P.options(**opts), levels=2, coarse_iter=300)
    x, info, _ = run_gpu(c["m"], c["grid"], c["sets"], "f64", dict(opts, levels=2, coarse_iter=300))
    assert rel(x, ref["x"]) <= 1e-9
    for a, b in zip(info["r_feas"], ref["r_feas"]):
        assert a == pytest.approx(b, rel=1e-6, abs=1e-12)
