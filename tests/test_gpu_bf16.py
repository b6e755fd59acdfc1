"""BF16 storage trial (sip_options.store_bf16): y_i, v_i (and their adapt
copies) and the model are rounded to bfloat16 at every store, so the
iteration follows exactly the numbers a BF16 storage of them would hold.

* Every stored y_i, v_i is a bfloat16 value (the rounding reaches every
  store: set pass, final pass, multilevel hand-over, warm start).
* Tolerance.  bfloat16 keeps 8 significand bits: one rounding moves a value
  by at most 2^-9 = 2.0e-3 of it.  The stored duals are rounded in every
  iteration, so the iterate carries a perturbation of that order, and on
  convex sets the projection is 1-Lipschitz in its data: the result is held
  to 2e-2 of the FP64 oracle (ten roundings' worth), and the binary32 run
  without the trial to 1e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import parsdmm as P                   # noqa: E402
from paper_1902_09699_gb300 import sip            # noqa: E402
from paper_1902_09699_gb300 import workloads as W  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def is_bf16(t):
    return bool(torch.equal(t, t.to(torch.bfloat16).to(torch.float32)))


def convex_3d():
    c = W.grf_3d(n=(40, 36, 20), seed=11)
    sets = [s for s in c["sets"] if s["type"] != "card"]
    return c, sets, dict(c["opts"], max_iter=120)


def test_bf16_storage_single_level_against_oracle():
    c, sets, opts = convex_3d()
    ref = P.parsdmm(c["m"], c["grid"], sets, P.options(**opts))
    m32 = torch.as_tensor(c["m"], dtype=torch.float32, device="cuda")
    out = {}
    for bf in (0, 1):
        pr = sip.Projector(c["grid"], sets, dtype="f32", store_bf16=bf, **opts)
        x, info = pr.project(m32)
        _, y, v = pr.get_state()
        pr.close()
        out[bf] = x.double().cpu().numpy()
        assert is_bf16(y) == bool(bf) and is_bf16(v) == bool(bf)
    assert rel(out[0], ref["x"]) <= 1e-5
    e = rel(out[1], ref["x"])
    assert 1e-6 < e <= 2e-2, e


def test_bf16_storage_multilevel_and_warm_start():
    c, sets, opts = convex_3d()
    m32 = torch.as_tensor(c["m"], dtype=torch.float32, device="cuda")
    ref = P.ml_parsdmm(c["m"], c["grid"], sets, P.options(**opts), levels=2, coarse_iter=60)
    pr = sip.Projector(c["grid"], sets, dtype="f32", store_bf16=1, levels=2, coarse_iter=60, **opts)
    x, _ = pr.project(m32)
    pr.close()
    assert rel(x.double().cpu().numpy(), ref["x"]) <= 2e-2
    # a warm start from a state that is not bfloat16: the loaded duals are rounded
    pr = sip.Projector(c["grid"], sets, dtype="f32", store_bf16=1, **dict(opts, max_iter=1))
    M = pr.state_rows()
    g = torch.Generator(device="cpu").manual_seed(3)
    y0 = torch.randn(M, generator=g).cuda()
    v0 = torch.randn(M, generator=g).cuda()
    pr.set_state(m32, y0, v0)
    _, y, v = pr.get_state()
    pr.close()
    assert is_bf16(y) and is_bf16(v)


def test_bf16_storage_rejected_where_not_available():
    c = W.small_2d(n=(16, 16))
    for bad in (dict(dtype="f64"),):
        with pytest.raises(sip.SipError) as e:
            sip.Projector(c["grid"], c["sets"], store_bf16=1, **dict(c["opts"], **{}), **bad)
        assert e.value.status == 1
    sets = [dict(c["sets"][0], scope="z")]
    with pytest.raises(sip.SipError):
        sip.Projector(c["grid"], sets, dtype="f32", store_bf16=1, **c["opts"])
