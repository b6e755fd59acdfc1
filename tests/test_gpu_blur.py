"""Data-fit sets with a blurring forward operator F through the C ABI,
against the FP64 oracle.

F is a centred symmetric averaging kernel of 2R + 1 samples along one axis
with zero padding (the blur of the paper's data-fit formulation and of its
joint deblurring-denoising-inpainting example).  It enters the x-step's
right-hand side as F^T (rho_F y_F + v_F), the system matrix as
rho_F F^T F (a band of 4R + 1 samples along the axis, Eq. sys_mat) and the
set pass as s = F x.  Bars as in the other loop parity tests: 1e-10 in
FP64, 1e-4 in FP32 with fixed rho.
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run_gpu(m, grid, sets, dt, opts):
    pr = sip.Projector(grid, sets, dtype=dt, **opts)
    x, info = pr.project(torch.as_tensor(m, dtype=TD[dt], device="cuda"))
    out = x.double().cpu().numpy(), info
    pr.close()
    return out


def as_f32(a):
    return torch.as_tensor(a, dtype=torch.float32).double().numpy()


def taps_of(R, seed):
    """Positive, decreasing taps k_0..k_R summing (two-sided) to 1."""
    g = np.random.default_rng(seed)
    t = np.sort(g.uniform(0.2, 1.0, R + 1))[::-1]
    return tuple(t / (t[0] + 2 * t[1:].sum()))


def deblur_case(n, axis, R, seed, frac=0.3, bound=0.05):
    """Layered model, observed data = its blur (the oracle's F, input only)
    at a random fraction of the samples plus noise; data fit
    {-bound <= F x - d <= bound} there, +-inf elsewhere; [1.5, 4.5] bounds
    and a TV ball from the truth."""
    g = np.random.default_rng(seed)
    grid = {"n": n}
    truth = W.layered(n, n_layers=6, seed=seed) if len(n) == 2 and n[0] >= 16 else W.grf(n, seed=seed)
    taps = taps_of(R, seed)
    d = O.apply(grid, O.blur_op(axis, taps), truth) + g.uniform(-0.02, 0.02, truth.size)
    obs = g.uniform(size=truth.size) < frac
    lo = np.where(obs, d - bound, -math.inf)
    hi = np.where(obs, d + bound, math.inf)
    m = np.where(obs, d, float(d[obs].mean())) + 0.1 * g.standard_normal(truth.size)
    tv = float(np.abs(O.apply(grid, "TV", truth)).sum())
    sets = [{"op": "BLUR", "axis": axis, "taps": taps, "type": "bounds", "lo": lo, "hi": hi},
            {"op": "TV", "type": "l1", "sigma": tv},
            {"op": "I", "type": "bounds", "lo": 1.5, "hi": 4.5}]
    return grid, m, sets


CASES = [
    ((37, 29), "z", 2, 31),
    ((37, 29), "x", 3, 32),
    ((64, 52), "x", 12, 33),     # the 25-sample motion blur
    ((24, 16, 12), "y", 2, 34),
    ((5, 40), "z", 4, 35),       # n_z < 2R: every sample meets both ends
    ((130, 9), "x", 6, 36),
    ((20, 40, 6), "x", 3, 37),   # 3D, x blur: blocks over z and x, y neighbours from memory
    ((30, 7, 5), "z", 2, 38),    # 3D, z blur: runs of one z column
]


@pytest.mark.parametrize("n,axis,R,seed", CASES)
def test_blur_data_fit_fp64_matches_oracle(n, axis, R, seed):
    grid, m, sets = deblur_case(n, axis, R, seed)
    opts = dict(max_iter=40, cg_iters=5, adapt=1, rho0=1.0, gamma0=1.5)
    ref = P.parsdmm(m, grid, sets, P.options(**opts))
    x, info = run_gpu(m, grid, sets, "f64", opts)
    assert rel(x, ref["x"]) <= 1e-10
    for a, b in zip(info["r_feas"], ref["r_feas"]):
        assert a == pytest.approx(b, rel=1e-8, abs=1e-13)


BOX_CASES = [
    ((64, 52), "x", 12, 41),     # a 25-sample motion blur
    ((37, 70), "x", 5, 42),      # ragged blocks along z and x
    ((24, 16, 40), "y", 3, 43),
    ((40, 9), "x", 6, 44),       # n_x < 2R
    ((18, 45, 4), "x", 4, 45),   # 3D
]


@pytest.mark.parametrize("dt,bar", [("f64", 1e-10), ("f32", 1e-4)])
@pytest.mark.parametrize("n,axis,R,seed", BOX_CASES)
def test_box_blur_matches_oracle(n, axis, R, seed, dt, bar):
    """Equal taps (a box, the paper's motion blur): the x and y blocks take
    sliding window sums instead of the tap band."""
    grid, m, sets = deblur_case(n, axis, R, seed)
    sets[0]["taps"] = W.motion_blur_taps(2 * R + 1)
    if dt == "f32":
        m = as_f32(m)
    opts = dict(max_iter=40, cg_iters=5, adapt=1 if dt == "f64" else 0, rho0=1.0, gamma0=1.5)
    ref = P.parsdmm(m, grid, sets, P.options(**opts))
    x, _ = run_gpu(m, grid, sets, dt, opts)
    assert rel(x, ref["x"]) <= bar


@pytest.mark.parametrize("n,axis,R,seed", CASES[:4])
def test_blur_data_fit_fp32(n, axis, R, seed):
    grid, m, sets = deblur_case(n, axis, R, seed)
    m = as_f32(m)
    opts = dict(max_iter=40, cg_iters=5, adapt=0, rho0=1.0, gamma0=1.5)
    ref = P.parsdmm(m, grid, sets, P.options(**opts))
    x, _ = run_gpu(m, grid, sets, "f32", opts)
    assert rel(x, ref["x"]) <= 1e-4


@pytest.mark.parametrize("dt,bar", [("f64", 1e-10), ("f32", 1e-4)])
def test_blur_l2_data_ball_and_norm_sets(dt, bar):
    """{||M (F x - d)|| <= sigma} (NaN: unobserved) next to an l2 ball
    with a relative radius and a card set on D_x x."""
    n = (40, 36)
    g = np.random.default_rng(37)
    grid = {"n": n}
    truth = W.layered(n, n_layers=6, seed=37)
    taps = taps_of(3, 37)
    d = O.apply(grid, O.blur_op("z", taps), truth) + 0.03 * g.standard_normal(truth.size)
    d[g.uniform(size=truth.size) < 0.4] = np.nan
    sigma = 0.03 * math.sqrt(np.sum(~np.isnan(d)))
    m = np.where(np.isnan(d), 3.0, d)
    if dt == "f32":
        m = as_f32(m)
    sets = [{"op": "BLUR", "axis": "z", "taps": taps, "type": "l2", "sigma": sigma, "center": d},
            {"op": "I", "type": "l2", "sigma_rel": 0.95},
            {"op": "DX", "type": "card", "k_frac": 0.05},
            {"op": "I", "type": "bounds", "lo": 1.5, "hi": 4.5}]
    opts = dict(max_iter=50, cg_iters=5, adapt=1 if dt == "f64" else 0, rho0=1.0, gamma0=1.5)
    ref = P.parsdmm(m, grid, sets, P.options(**opts))
    x, _ = run_gpu(m, grid, sets, dt, opts)
    assert rel(x, ref["x"]) <= bar


def test_blur_with_relative_radius_on_f_x():
    """sigma_rel on a blur set: the radius resolves against ||F m||_1 on the
    device (the norm kernel applies F)."""
    n = (33, 27)
    grid = {"n": n}
    m = W.layered(n, n_layers=5, seed=38)
    taps = taps_of(2, 38)
    sets = [{"op": "BLUR", "axis": "x", "taps": taps, "type": "l1", "sigma_rel": 0.9},
            {"op": "I", "type": "bounds", "lo": 1.5, "hi": 4.5}]
    opts = dict(max_iter=40, cg_iters=5, adapt=1, rho0=1.0, gamma0=1.5)
    ref = P.parsdmm(m, grid, sets, P.options(**opts))
    x, _ = run_gpu(m, grid, sets, "f64", opts)
    assert rel(x, ref["x"]) <= 1e-10


def test_blur_in_a_batch_and_persistent_request():
    """A batch mixing an instance with a blur and one without (one plan,
    the blur instantiations of the kernels for both), and a persistent
    request, which a blur plan runs on the graph path."""
    g1, m1, s1 = deblur_case((30, 26), "x", 2, 39)
    g2 = {"n": (21, 34)}
    m2 = W.layered(g2["n"], n_layers=5, seed=40)
    s2 = [{"op": "TV", "type": "l1", "sigma_rel": 0.4}, {"op": "I", "type": "bounds", "lo": 2.0, "hi": 4.0}]
    opts = dict(max_iter=40, cg_iters=5, adapt=1, rho0=1.0, gamma0=1.5)
    bp = sip.BatchProjector([(g1, s1), (g2, s2)], dtype="f64", **opts)
    xs, _ = bp.project([m1, m2])
    bp.close()
    for (grid, sets, m), x in zip([(g1, s1, m1), (g2, s2, m2)], xs):
        ref = P.parsdmm(m, grid, sets, P.options(**opts))
        assert rel(x.cpu().numpy(), ref["x"]) <= 1e-10
    x, _ = run_gpu(m1, g1, s1, "f64", dict(opts, exec="persistent"))
    ref = P.parsdmm(m1, g1, s1, P.options(**opts))
    assert rel(x, ref["x"]) <= 1e-10


def test_deblur_workload_full_size_first_iterations():
    """The 1100 x 1100 deblurring-inpainting workload (25-sample motion
    blur) in the bench's configuration (FP32, adaptive rho), two iterations
    against the oracle from the same binary32 model."""
    c = W.deblur_2d()
    m = as_f32(c["m"])
    opts = dict(c["opts"], max_iter=2)
    ref = P.parsdmm(m, c["grid"], c["sets"], P.options(**opts))
    x, info = run_gpu(m, c["grid"], c["sets"], "f32", opts)
    assert info["iters"] == 2
    assert rel(x, ref["x"]) <= 1e-5


def test_blur_sets_validated():
    base = {"op": "BLUR", "axis": "z", "taps": (0.5, 0.25), "type": "bounds", "lo": 0.0, "hi": 9.0}
    bad = [
        dict(base, taps=(1.0,)),                      # R = 0
        dict(base, taps=(1.0 / 27,) * 14),            # R = 13 > SIP_MAX_BLUR_RADIUS
        dict(base, axis="y"),                         # y in 2D
        dict(base, taps=(0.5, float("nan"))),
        dict(base, type="l2", sigma=1.0, scope="z"),  # per-line
    ]
    for s in bad:
        with pytest.raises(sip.SipError):
            sip.Projector({"n": (8, 8)}, [s], dtype="f64")
    with pytest.raises(sip.SipError):                 # two blur sets
        sip.Projector({"n": (8, 8)}, [base, dict(base, axis="x")], dtype="f64")
    with pytest.raises(sip.SipError):                 # multilevel
        sip.Projector({"n": (16, 16)}, [base], dtype="f64", levels=2)
    with pytest.raises(sip.SipError):                 # single-operator entry points carry no taps
        sip.op_norm({"n": (8, 8)}, "BLUR", "l2", torch.zeros(64, dtype=torch.float64, device="cuda"))
