"""The allocation-free l1-ball projection (sip_project_l1_noalloc).

Some callers cannot allocate device memory while they run, for instance code
inside a fixed memory pool or budget, or a latency-sensitive loop where an
allocation could synchronise the device.  For them the library offers an
l1-ball projection whose scratch is a fixed array compiled into the library.
This test checks, through the C ABI, that it returns the same result as the
regular entry point sip_project_set and as the FP64 oracle's l1-ball
projection on two calls in a row (the second call reuses the array the first
one left behind), and that it rejects sizes above its fixed limit and
non-finite input.  It lives in its own file, collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import prox as oracle_prox     # noqa: E402
from paper_1902_09699_gb300 import sip     # noqa: E402

TD = {"f64": torch.float64, "f32": torch.float32}
# the l1 tolerances of the single-step parity tests (tests/test_gpu_steps.py)
ATOL = {"f64": 1e-12, "f32": 2e-6}


def regular(w, tau):
    return sip.project_set({"type": "l1", "sigma": tau}, w)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_noalloc_matches_regular_entry_point_twice(dt):
    g = np.random.default_rng(2024)
    for call, n in enumerate((300001, 4097)):       # two calls in a row, different sizes
        w = torch.as_tensor(g.standard_normal(n) * 3.0, dtype=TD[dt], device="cuda")
        tau = 0.4 * float(w.abs().sum())
        y_ref, th_ref = regular(w, tau)
        y = torch.full_like(w, float("nan"))
        y, th = sip.project_l1_noalloc(w, tau, y=y)
        scale = float(w.abs().max())
        assert torch.allclose(y, y_ref, rtol=0, atol=ATOL[dt] * scale), (call, n)
        assert th == pytest.approx(th_ref, rel=1e-12)
        # and the FP64 oracle (sort-based threshold) on the same input
        w64 = w.double().cpu().numpy()
        y_or = oracle_prox.proj_l1(w64, tau)
        th_or = oracle_prox.l1_threshold(w64, tau)
        assert np.max(np.abs(y.double().cpu().numpy() - y_or)) <= ATOL[dt] * scale, (call, n)
        assert th == pytest.approx(th_or, rel=1e-10 if dt == "f64" else 1e-5)


def test_noalloc_inside_ball_and_zero_radius():
    w = torch.as_tensor(np.linspace(-1.0, 1.0, 1001), device="cuda")
    y, th = sip.project_l1_noalloc(w, 1e9)
    assert torch.equal(y, w) and th == 0.0
    y, th = sip.project_l1_noalloc(w, 0.0)
    assert torch.count_nonzero(y) == 0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    w = torch.zeros(sip.NOALLOC_MAX_N + 1, dtype=torch.float32, device="cuda")
    with pytest.raises(sip.SipError) as e:
        sip.project_l1_noalloc(w, 1.0)
    assert e.value.status == 1 and "SIP_NOALLOC_MAX_N" in str(e.value)


def test_noalloc_rejects_a_bad_output_tensor_on_the_host():
    w = torch.ones(100, dtype=torch.float64, device="cuda")
    for y in (torch.empty(99, dtype=torch.float64, device="cuda"),
              torch.empty(100, dtype=torch.float32, device="cuda")):
        with pytest.raises(ValueError):
            sip.project_l1_noalloc(w, 1.0, y=y)


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_noalloc_reports_non_finite_input(bad):
    w = torch.linspace(-1.0, 1.0, 5000, dtype=torch.float32, device="cuda")
    w[1234] = bad
    with pytest.raises(sip.SipError) as e:
        sip.project_l1_noalloc(w, 1.0)
    assert e.value.status == 5
    # the array is usable again right after
    w[1234] = 0.0
    y, th = sip.project_l1_noalloc(w, 1.0)
    y_ref, th_ref = regular(w, 1.0)
    assert torch.allclose(y, y_ref, rtol=0, atol=2e-6) and th == pytest.approx(th_ref, rel=1e-12)
