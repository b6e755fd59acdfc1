"""Warm start through the C ABI: sip_get_state returns the final iterates
(x, y_i, v_i) of a projection, and sip_set_state starts the next
projection from a given state, as ML-PARSDMM hands the state from one
level to the next (Sec. "Multilevel PARSDMM").  Checked against the FP64
oracle started from the same state."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import parsdmm as P                   # noqa: E402
from paper_1902_09699_gb300 import sip            # noqa: E402
from paper_1902_09699_gb300 import workloads as W  # noqa: E402

SETS = [{"op": "I", "type": "bounds", "lo": 1.8, "hi": 4.2},
        {"op": "TV", "type": "l1", "sigma_rel": 0.4},
        {"op": "DZ", "type": "bounds", "lo": -0.2, "hi": 0.6}]
OPTS = dict(max_iter=40, cg_iters=5, adapt=1, rho0=1.0, gamma0=1.5)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def split(flat, blocks):
    out, off = [], 0
    for b in blocks:
        out.append(flat[off:off + b["M"]])
        off += b["M"]
    assert off == flat.size
    return out


@pytest.mark.parametrize("form", ["alg1", "direct"])
def test_state_round_trip_and_warm_start(form):
    grid = {"n": (40, 36)}
    m1 = W.layered(grid["n"], n_layers=6, seed=51)
    m2 = m1 + 0.05 * np.random.default_rng(52).standard_normal(m1.size)
    opts = dict(OPTS, form=form)
    pr = sip.Projector(grid, SETS, dtype="f64", **opts)
    x1, _ = pr.project(torch.as_tensor(m1, device="cuda"))
    ref1 = P.parsdmm(m1, grid, SETS, P.options(**opts))
    # get_state: the final iterates, blocks in order (identity block last in alg1)
    xs, ys, vs = (t.cpu().numpy() for t in pr.get_state())
    assert pr.state_rows() == sum(b["M"] for b in ref1["blocks"])
    assert rel(xs, ref1["x"]) <= 1e-10
    assert np.array_equal(xs, x1.cpu().numpy())
    # per block, against the whole vector's size (an inactive set's duals
    # are rounding noise around 0)
    for mine, theirs in ((ys, ref1["y"]), (vs, ref1["v"])):
        scale = np.linalg.norm(np.concatenate(theirs))
        for got, want in zip(split(mine, ref1["blocks"]), theirs):
            assert np.linalg.norm(got - want) <= 1e-9 * scale
    # warm start of the next projection from that state
    pr.set_state(xs, ys, vs)
    x2, _ = pr.project(torch.as_tensor(m2, device="cuda"))
    ref2 = P.parsdmm(m2, grid, SETS, P.options(**opts),
                     init=(xs, split(ys, ref1["blocks"]), split(vs, ref1["blocks"])))
    assert rel(x2.cpu().numpy(), ref2["x"]) <= 1e-10
    # only that projection: the next one starts from zeros again
    x3, _ = pr.project(torch.as_tensor(m2, device="cuda"))
    ref3 = P.parsdmm(m2, grid, SETS, P.options(**opts))
    assert rel(x3.cpu().numpy(), ref3["x"]) <= 1e-10
    pr.close()


def test_set_state_with_x_only_and_fp32():
    grid = {"n": (33, 28)}
    m = W.layered(grid["n"], n_layers=5, seed=53)
    m32 = torch.as_tensor(m, dtype=torch.float32).double().numpy()
    x0 = np.clip(m32, 2.0, 4.0)
    x0 = torch.as_tensor(x0, dtype=torch.float32).double().numpy()
    opts = dict(OPTS, adapt=0)
    pr = sip.Projector(grid, SETS, dtype="f32", **opts)
    pr.set_state(x0)                       # y, v from zeros
    x, _ = pr.project(torch.as_tensor(m32, dtype=torch.float32, device="cuda"))
    blocks = P.parsdmm(m32, grid, SETS, P.options(**dict(opts, max_iter=1)))["blocks"]
    ref = P.parsdmm(m32, grid, SETS, P.options(**opts),
                    init=(x0, [np.zeros(b["M"]) for b in blocks], [np.zeros(b["M"]) for b in blocks]))
    assert rel(x.double().cpu().numpy(), ref["x"]) <= 1e-4
    pr.close()


def test_state_calls_rejected_where_there_is_no_single_state():
    grid = {"n": (32, 32)}
    pr = sip.Projector(grid, SETS[:1], dtype="f64", levels=2)
    assert pr.state_rows() == -1
    with pytest.raises(sip.SipError):
        pr.get_state()
    with pytest.raises(sip.SipError):
        pr.set_state(np.zeros(32 * 32))
    pr.close()


def test_warm_start_carries_rho_and_gamma():
    """The penalties and relaxations adapted in one projection (sip_info)
    start the next one, against the oracle started from the same x, y_i,
    v_i, rho_i and gamma_i."""
    grid = {"n": (36, 30)}
    m1 = W.layered(grid["n"], n_layers=6, seed=54)
    m2 = m1 + 0.05 * np.random.default_rng(55).standard_normal(m1.size)
    opts = dict(OPTS, adapt=2)
    pr = sip.Projector(grid, SETS, dtype="f64", **opts)
    _, info = pr.project(torch.as_tensor(m1, device="cuda"))
    ref1 = P.parsdmm(m1, grid, SETS, P.options(**opts))
    assert np.allclose(info["rho"], ref1["rho"], rtol=1e-9)
    xs, ys, vs = (t.cpu().numpy() for t in pr.get_state())
    pr.set_state(xs, ys, vs, rho=info["rho"], gamma=info["gamma"])
    x2, _ = pr.project(torch.as_tensor(m2, device="cuda"))
    blocks = ref1["blocks"]
    ref2 = P.parsdmm(m2, grid, SETS, P.options(**opts), init=(xs, split(ys, blocks), split(vs, blocks)),
                     init_rho=info["rho"], init_gamma=info["gamma"])
    assert rel(x2.cpu().numpy(), ref2["x"]) <= 1e-10
    with pytest.raises(sip.SipError):
        pr.set_state(xs, rho=[-1.0] * len(blocks))
    pr.close()


@pytest.mark.parametrize("dt", ["f64"])
def test_warm_start_with_adapt_state_continues_the_run(dt):
    """K iterations, then a warm start that carries x, y_i, v_i, rho_i,
    gamma_i and adapt-rho-gamma's saved quantities, for K more: the result of
    2K uninterrupted iterations of the oracle (the oracle's own pin shows the
    same continuity, and that without the saved quantities it is lost)."""
    c = W.layered_2d(n=(48, 64), seed=77)
    sets = [s_ for s_ in c["sets"] if s_["type"] != "card"]
    K = 20
    opts = dict(c["opts"], adapt=2, max_iter=K)
    m = torch.as_tensor(c["m"], device="cuda")
    full = P.parsdmm(c["m"], c["grid"], sets, P.options(**dict(opts, max_iter=2 * K)))
    pr = sip.Projector(c["grid"], sets, dtype=dt, **opts)
    _, info = pr.project(m)
    x, y, v = pr.get_state()
    st = pr.get_adapt_state()
    assert st is not None
    pr.set_state(x, y, v, rho=info["rho"], gamma=info["gamma"])
    pr.set_adapt_state(*st)
    x2, info2 = pr.project(m)
    pr.close()
    ref = full["x"]
    e2 = float(np.linalg.norm(x2.cpu().numpy() - ref) / np.linalg.norm(ref))
    assert e2 <= 1e-10, e2
    np.testing.assert_allclose(info2["rho"], full["rho"], rtol=1e-9)
    np.testing.assert_allclose(info2["gamma"], full["gamma"], rtol=1e-9)


def test_adapt_state_rejected_without_adaptation_or_ring():
    c = W.small_2d(n=(16, 16))
    pr = sip.Projector(c["grid"], c["sets"], dtype="f64", **dict(c["opts"], adapt=0))
    with pytest.raises(sip.SipError):
        pr.get_adapt_state()
    pr.close()
    pr = sip.Projector(c["grid"], c["sets"], dtype="f64", **dict(c["opts"], adapt=1, adapt_every=5, evol_hist=5))
    with pytest.raises(sip.SipError):
        pr.get_adapt_state()
    pr.close()
