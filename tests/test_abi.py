"""C-ABI checks that need no GPU: the library builds and loads, exports every
function include/sip.h declares, the ctypes structs match the C layout, and
host-side argument validation rejects bad input before any device work."""
import ctypes
import math
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sip.h")


@pytest.fixture(scope="module")
def sip():
    from paper_1902_09699_gb300 import build, sip as S
    if not os.path.exists(S.LIB_PATH):
        build.build()
    S.lib()
    return S


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sip_[a-z_0-9]+)\s*\(", src)))


def test_header_functions_exported_and_bound(sip):
    names = declared_functions()
    assert len(names) >= 15
    L = sip.lib()
    for n in names:
        assert hasattr(L, n), n
        assert n in sip.SIGNATURES, "binding misses " + n
    assert set(sip.SIGNATURES) == set(names)
    out = subprocess.run(["nm", "-D", "--defined-only", sip.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (sip_\w+)", out))
    assert set(names) <= exported


def test_struct_layouts_match_c(sip, tmp_path):
    prog = tmp_path / "sizes.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "sip.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(sip_grid),'
                    ' sizeof(sip_set), sizeof(sip_options), sizeof(sip_info), offsetof(sip_options, rho0),'
                    ' offsetof(sip_options, trace), offsetof(sip_info, ms), sizeof(sip_server_config),'
                    ' sizeof(sip_server_stats), offsetof(sip_server_config, max_points), sizeof(sip_tuning),'
                    ' offsetof(sip_tuning, tuned), offsetof(sip_options, tune)); return 0;}\n')
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(sip.Grid), ctypes.sizeof(sip.Set), ctypes.sizeof(sip.Options), ctypes.sizeof(sip.Info),
            sip.Options.rho0.offset, sip.Options.trace.offset, sip.Info.ms.offset, ctypes.sizeof(sip.ServerConfig),
            ctypes.sizeof(sip.ServerStats), sip.ServerConfig.max_points.offset, ctypes.sizeof(sip.Tuning),
            sip.Tuning.tuned.offset, sip.Options.tune.offset]
    assert got == want


def test_defaults_follow_the_paper(sip):
    o = sip.default_options()
    assert (o.eps_feas, o.eps_evol, o.check_every, o.evol_hist) == (1e-3, 1e-2, 5, 5)
    assert (o.eps_corr, o.adapt_every, o.cg_iters) == (0.3, 2, 5)


def test_op_rows(sip):
    g = {"n": (5, 4), "h": (1.0, 1.0)}
    assert sip.op_rows(g, "I") == 20
    assert sip.op_rows(g, "DZ") == 16
    assert sip.op_rows(g, "DX") == 15
    assert sip.op_rows(g, "TV") == 31
    g3 = {"n": (4, 3, 5)}
    assert sip.op_rows(g3, "DY") == 48
    assert sip.op_rows(g3, "TV") == 3 * 3 * 5 + 4 * 2 * 5 + 48
    assert sip.op_rows(g, "DY") == -1             # 2D grid has no y axis
    assert sip.op_rows(g, "BLUR") == -1           # the single-operator calls carry no taps


BLUR = {"op": "BLUR", "axis": "z", "taps": (0.5, 0.25), "type": "bounds", "lo": 0.0, "hi": 9.0}


@pytest.mark.parametrize("bad", [
    dict(grid={"n": (0, 4)}),
    dict(grid={"n": (4, 4), "h": (0.0, 1.0)}),
    dict(sets=[{"op": "I", "type": "bounds", "lo": 3.0, "hi": 2.0}]),
    dict(sets=[{"op": "TV", "type": "l1", "sigma": -1.0}]),
    dict(sets=[{"op": "DZ", "type": "card", "k": -2}]),
    dict(sets=[{"op": "DY", "type": "bounds", "lo": 0.0, "hi": 1.0}]),
    dict(grid={"n": (1, 8)}, sets=[{"op": "DZ", "type": "bounds", "lo": 0.0, "hi": 1.0}]),
    dict(opts=dict(max_iter=0)),
    dict(opts=dict(evol_hist=9)),
    dict(opts=dict(gamma0=2.0)),
    dict(sets=[{"op": "I", "type": "bounds", "lo": 0.0, "hi": 1.0}] * 17),
    dict(opts=dict(levels=0)),
    dict(opts=dict(levels=9)),
    # 4 -> 2 -> 1 samples along z: D_z has no rows on the third level
    dict(grid={"n": (4, 8)}, sets=[{"op": "DZ", "type": "bounds", "lo": 0.0, "hi": 1.0}], opts=dict(levels=3)),
    dict(opts=dict(select_window=2)),
    dict(sets=[{"op": "TV", "type": "card", "k": 2, "scope": "z"}]),
    dict(sets=[{"op": "I", "type": "l1", "sigma_rel": 0.2, "scope": "x"}]),
    dict(sets=[{"op": "I", "type": "l2", "sigma": 1.0, "scope": "y"}]),
    dict(grid={"n": (4100, 2)}, sets=[{"op": "I", "type": "card", "k": 1, "scope": "z"}]),
    dict(sets=[{"op": "I", "type": "annulus", "lo": -1.0, "hi": 1.0}]),
    dict(sets=[dict(BLUR, taps=(1.0,))]),                      # radius 0
    dict(sets=[dict(BLUR, taps=(1.0 / 27,) * 14)]),            # radius 13
    dict(sets=[dict(BLUR, axis="y")]),                         # y in 2D
    dict(sets=[dict(BLUR, taps=(0.5, math.inf))]),
    dict(sets=[dict(BLUR, type="l2", sigma=1.0, scope="z")]),
    dict(sets=[BLUR, dict(BLUR, axis="x")]),                   # two blur sets
    dict(grid={"n": (16, 16)}, sets=[BLUR], opts=dict(levels=2)),
])
def test_invalid_arguments_rejected_on_host(sip, bad):
    grid = bad.get("grid", {"n": (8, 8)})
    sets = bad.get("sets", [{"op": "I", "type": "bounds", "lo": 0.0, "hi": 1.0}])
    with pytest.raises(sip.SipError) as e:
        sip.Projector(grid, sets, dtype="f64", **bad.get("opts", {}))
    assert e.value.status == 1
    assert str(e.value)


def test_null_arguments(sip):
    L = sip.lib()
    h = ctypes.c_void_p()
    assert L.sip_create(None, None, 0, None, ctypes.byref(h)) == 1
    assert L.sip_project(None, None, None, None, None) == 1
    assert L.sip_destroy(None) == 0
    assert L.sip_last_error(None)
    # warm-start state of a missing handle
    assert L.sip_state_rows(None) == -1
    assert L.sip_get_state(None, None, None, None, None) == 1
    assert L.sip_set_state(None, None, None, None, None, None, None) == 1


def test_test_hook_rejects_bad_arguments(sip):
    L = sip.lib()
    assert L.sip_test_hook(99, 0) == 1
    assert b"unknown hook" in L.sip_last_error(None)
    assert L.sip_test_hook(sip.HOOKS["fail_alloc"], -1) == 1
    assert L.sip_test_hook(sip.HOOKS["barrier_extra"], 1 << 21) == 1
    for h in sip.HOOKS.values():
        assert L.sip_test_hook(h, 0) == 0


def test_guard_macros_compile_away_in_release_and_on_in_debug():
    """The index guards exist only in the debug build: the release kernels
    source compiles the macros to nothing, the guarded one to checks."""
    src = open(os.path.join(ROOT, "paper_1902_09699_gb300", "csrc", "sip_dev.cuh")).read()
    assert "#if defined(__CUDACC__) && defined(SIP_GUARDS)" in src
    k = open(os.path.join(ROOT, "paper_1902_09699_gb300", "csrc", "kernels.cu")).read()
    assert k.count("SIP_GUARD_TILE(") >= 9 and k.count("SIP_GUARD_IDX(") >= 3
