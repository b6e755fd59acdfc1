"""The projection server (continuous batching).

Requests of different sizes and set lists are submitted together so that
the worker forms cohorts and runs them concurrently; each result must equal
the result of the same projection run alone through sip_project (FP64:
1e-10, the rounding order of binary64 atomics aside), the budget must be
respected, and over-budget requests must fail cleanly.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1902_09699_gb300 import sip            # noqa: E402
from paper_1902_09699_gb300 import workloads as W  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def requests(count, seed=3):
    g = np.random.default_rng(seed)
    pool = W.small_2d()["sets"]
    out = []
    for i in range(count):
        if i % 4 == 3:
            n = (int(g.integers(8, 20)), int(g.integers(8, 20)), int(g.integers(4, 10)))
        else:
            n = (int(g.integers(16, 96)), int(g.integers(16, 96)))
        sets = [dict(pool[j]) for j in g.integers(0, len(pool), size=int(g.integers(2, 5)))]
        out.append(({"n": n}, sets, W.grf(n, seed=100 + i)))
    return out


def test_results_alone_and_in_the_mix_are_equal():
    opts = dict(max_iter=120, adapt=1, gamma0=1.5, stop=2)
    reqs = requests(14)
    srv = sip.Server(dtype="f64", max_batch=5, max_cohorts=3, max_wait_ms=0.5, **opts)
    ids = [srv.submit(g, s, m) for g, s, m in reqs]
    got = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["p99_ms"] >= st["p50_ms"] > 0
    for (g, s, m), (x, info, lat) in zip(reqs, got):
        pr = sip.Projector(g, s, dtype="f64", **opts)
        x1, info1 = pr.project(torch.as_tensor(m, device="cuda"))
        pr.close()
        assert info["iters"] == info1["iters"]
        assert rel(x, x1.cpu().numpy()) <= 1e-10
        assert lat > 0


def test_budget_is_respected_and_oversize_requests_fail():
    opts = dict(max_iter=40, adapt=1, gamma0=1.5)
    reqs = requests(6, seed=9)
    srv = sip.Server(dtype="f32", budget_bytes=64 << 20, max_batch=8, max_cohorts=2, **opts)
    ids = [srv.submit(g, s, m) for g, s, m in reqs]
    for i in ids:
        x, info, lat = srv.wait(i)
        assert np.isfinite(x).all()
    big = ({"n": (1024, 1024)}, W.small_2d()["sets"], W.grf((1024, 1024), seed=1))
    rid = srv.submit(*big)
    with pytest.raises(sip.SipError) as e:
        srv.wait(rid)
    assert e.value.status == 6
    st = srv.stats()
    srv.close()
    assert 0 < st["hbm_peak"] <= 64 << 20


def test_served_results_match_the_oracle():
    """Every served result against the FP64 oracle run alone on the same
    request (adaptive rho, feasibility stopping rule): the same stopping
    iteration and x within 1e-9 (the GPU's own rho trajectory follows the
    oracle's to 1e-9)."""
    from oracle import parsdmm as P
    opts = dict(max_iter=150, adapt=1, gamma0=1.5, stop=2, eps_feas=1e-2)
    g = np.random.default_rng(21)
    pool = W.small_2d()["sets"]
    reqs = []
    for i in range(8):
        n = (int(g.integers(8, 14)), int(g.integers(8, 14)), 4) if i % 4 == 3 else \
            (int(g.integers(12, 40)), int(g.integers(12, 40)))
        sets = [dict(pool[j]) for j in g.integers(0, len(pool), size=int(g.integers(2, 4)))]
        reqs.append(({"n": n}, sets, W.grf(n, seed=300 + i)))
    srv = sip.Server(dtype="f64", max_batch=4, max_cohorts=2, max_wait_ms=0.5, **opts)
    ids = [srv.submit(gr, s, m) for gr, s, m in reqs]
    got = [srv.wait(i) for i in ids]
    srv.close()
    for (gr, s, m), (x, info, lat) in zip(reqs, got):
        ref = P.parsdmm(m, gr, s, P.options(**opts))
        assert info["iters"] == ref["iters"]
        assert rel(x, ref["x"]) <= 1e-9
