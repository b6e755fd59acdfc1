"""Failure handling without a GPU fault: host-side fault injection through
sip_test_hook.

* A device allocation that fails (made to fail on the host, before
  cudaMalloc is called) returns SIP_ERR_OOM and leaves the library usable.
* A bounded device wait that runs out: the persistent kernel's grid barriers
  are told to wait for one arrival more than the grid makes, with a short
  poll limit, so every CTA gives up within milliseconds and returns;
  sip_project reports SIP_ERR_TIMEOUT and the same handle then projects
  correctly.  Nothing waits without a limit and no kernel faults.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import parsdmm as P                   # noqa: E402
from paper_1902_09699_gb300 import sip            # noqa: E402
from paper_1902_09699_gb300 import workloads as W  # noqa: E402


@pytest.fixture
def hooks():
    yield sip.test_hook
    for name in sip.HOOKS:
        sip.test_hook(name, 0)


def small_case():
    c = W.small_2d(n=(24, 20), seed=5)
    return c, dict(c["opts"], max_iter=20)


def test_arena_allocation_failure_returns_oom(hooks):
    c, opts = small_case()
    hooks("fail_alloc", 1)
    with pytest.raises(sip.SipError) as e:
        sip.Projector(c["grid"], c["sets"], dtype="f64", **opts)
    assert e.value.status == 2 and "allocation" in str(e.value)
    # the hook fired once; the next handle is created and projects correctly
    pr = sip.Projector(c["grid"], c["sets"], dtype="f64", **opts)
    x, info = pr.project(torch.as_tensor(c["m"], device="cuda"))
    pr.close()
    ref = P.parsdmm(c["m"], c["grid"], c["sets"], P.options(**opts))
    assert np.linalg.norm(x.cpu().numpy() - ref["x"]) <= 1e-10 * np.linalg.norm(ref["x"])


def test_second_allocation_fails_in_a_batch(hooks):
    c, opts = small_case()
    inst = [(c["grid"], c["sets"])] * 3
    hooks("fail_alloc", 2)       # the first create passes, the second fails
    bp = sip.BatchProjector(inst, dtype="f64", **opts)
    with pytest.raises(sip.SipError) as e:
        sip.BatchProjector(inst, dtype="f64", **opts)
    assert e.value.status == 2
    xs, _ = bp.project([c["m"]] * 3)
    bp.close()
    ref = P.parsdmm(c["m"], c["grid"], c["sets"], P.options(**opts))
    for xi in xs:
        assert np.linalg.norm(xi.cpu().numpy() - ref["x"]) <= 1e-10 * np.linalg.norm(ref["x"])


def test_persistent_barrier_timeout_then_handle_usable(hooks):
    c, opts = small_case()
    pr = sip.Projector(c["grid"], c["sets"], dtype="f64", exec="persistent", **opts)
    m = torch.as_tensor(c["m"], device="cuda")
    hooks("barrier_spins", 4096)
    hooks("barrier_extra", 1)
    with pytest.raises(sip.SipError) as e:
        pr.project(m)
    assert e.value.status == 4 and "bounded device wait" in str(e.value)
    hooks("barrier_extra", 0)
    hooks("barrier_spins", 0)
    x, info = pr.project(m)
    pr.close()
    assert info["iters"] == opts["max_iter"]
    ref = P.parsdmm(c["m"], c["grid"], c["sets"], P.options(**opts))
    assert np.linalg.norm(x.cpu().numpy() - ref["x"]) <= 1e-10 * np.linalg.norm(ref["x"])
