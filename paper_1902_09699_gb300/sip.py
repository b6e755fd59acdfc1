"""Thin ctypes binding of the C ABI in include/sip.h (libsip.so).

Argument marshalling only: every step of a projection runs in the library's
CUDA kernels.  Device memory and streams come from PyTorch tensors.  If the
library has not been built this module raises on first use; there is no
fallback path.
"""
import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SIP_GUARDS=1 selects the debug build whose kernels check their work items
# and indices (a failed check makes the call return SIP_ERR_INTERNAL)
LIB_PATH = os.path.join(_HERE, "libsip_guarded.so" if os.environ.get("SIP_GUARDS") == "1" else "libsip.so")

OPS = {"I": 0, "DZ": 1, "DX": 2, "DY": 3, "TV": 4, "BLUR": 5}
BLUR_AXES = {"z": 0, "x": 1, "y": 2}
SET_TYPES = {"bounds": 0, "l1": 1, "l2": 2, "card": 3, "annulus": 4}
SCOPES = {"all": 0, "z": 1, "x": 2, "y": 3}
F64, F32 = 0, 1
FORMS = {"alg1": 0, "direct": 1}
EXEC = {"auto": 0, "graph": 1, "persistent": 2, "cluster": 3}
STATUS = {0: "SIP_OK", 1: "SIP_ERR_INVALID_ARG", 2: "SIP_ERR_OOM", 3: "SIP_ERR_CUDA", 4: "SIP_ERR_TIMEOUT",
          5: "SIP_ERR_NONFINITE", 6: "SIP_ERR_BUDGET", 7: "SIP_ERR_INTERNAL"}
MAX_SETS = 16

c_int, c_i64, c_dbl, c_vp = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


class Grid(ctypes.Structure):
    _fields_ = [("ndim", c_int), ("n", c_i64 * 3), ("h", c_dbl * 3)]


class Set(ctypes.Structure):
    _fields_ = [("op", c_int), ("type", c_int), ("lo", c_dbl), ("hi", c_dbl), ("sigma", c_dbl),
                ("sigma_rel", c_dbl), ("k", c_i64), ("k_frac", c_dbl), ("scope", c_int),
                ("lo_vec", ctypes.POINTER(c_dbl)), ("hi_vec", ctypes.POINTER(c_dbl)),
                ("center_vec", ctypes.POINTER(c_dbl)),
                ("blur_axis", c_int), ("blur_radius", c_int), ("blur_taps", ctypes.POINTER(c_dbl))]


class Options(ctypes.Structure):
    _fields_ = [("max_iter", c_int), ("cg_iters", c_int), ("cg_max", c_int), ("eps_feas", c_dbl),
                ("eps_evol", c_dbl), ("check_every", c_int), ("evol_hist", c_int), ("stop", c_int),
                ("adapt", c_int), ("adapt_every", c_int), ("rho0", c_dbl), ("gamma0", c_dbl),
                ("eps_corr", c_dbl), ("rho_ratio_max", c_dbl), ("gamma_max", c_dbl), ("form", c_int),
                ("dtype", c_int), ("levels", c_int), ("coarse_iter", c_int),
                ("rho_schedule", ctypes.POINTER(c_dbl)), ("gamma_schedule", ctypes.POINTER(c_dbl)),
                ("trace", ctypes.POINTER(c_dbl)), ("exec", c_int), ("select_window", c_int),
                ("cluster_ctas", c_int), ("tune", c_int), ("store_bf16", c_int)]


class Info(ctypes.Structure):
    _fields_ = [("iters", c_int), ("cg_steps_total", c_int), ("stop_reason", c_int), ("nblocks", c_int),
                ("r_evol", c_dbl), ("r_feas", c_dbl * MAX_SETS), ("rho", c_dbl * (MAX_SETS + 1)),
                ("gamma", c_dbl * (MAX_SETS + 1)), ("sigma", c_dbl * MAX_SETS), ("k", c_i64 * MAX_SETS),
                ("ms", ctypes.c_float), ("window_hits", c_int)]


class Tuning(ctypes.Structure):
    _fields_ = [("scale_n", c_dbl), ("scale_set", c_dbl), ("scale_sel", c_dbl), ("scale_fin", c_dbl),
                ("exec", c_int), ("cluster_ctas", c_int), ("select_window", c_int), ("stage_rhs", c_int),
                ("tuned", c_int), ("from_cache", c_int), ("candidates", c_int), ("ms_default", c_dbl),
                ("ms_best", c_dbl)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("opts", Options), ("budget_bytes", c_i64), ("max_batch", c_int), ("max_cohorts", c_int),
                ("max_wait_ms", c_dbl), ("max_points", c_i64)]


class DykstraInfo(ctypes.Structure):
    _fields_ = [("sweeps", c_int), ("cg_steps", c_i64), ("l1_projections", c_i64), ("ms", ctypes.c_float)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", c_i64), ("failed", c_i64), ("queued", c_i64), ("running_cohorts", c_int),
                ("hbm_in_use", c_i64), ("hbm_peak", c_i64), ("p50_ms", c_dbl), ("p99_ms", c_dbl),
                ("projections_per_s", c_dbl)]


# every function declared in include/sip.h: name -> (restype, argtypes)
SIGNATURES = {
    "sip_options_default": (None, [ctypes.POINTER(Options)]),
    "sip_create": (c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Set), c_int, ctypes.POINTER(Options),
                           ctypes.POINTER(c_vp)]),
    "sip_project": (c_int, [c_vp, c_vp, c_vp, c_vp, ctypes.POINTER(Info)]),
    "sip_destroy": (c_int, [c_vp]),
    "sip_state_rows": (c_i64, [c_vp]),
    "sip_get_state": (c_int, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "sip_set_state": (c_int, [c_vp, c_vp, c_vp, c_vp, ctypes.POINTER(c_dbl), ctypes.POINTER(c_dbl), c_vp]),
    "sip_get_adapt_state": (c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, ctypes.POINTER(c_int), c_vp]),
    "sip_set_adapt_state": (c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "sip_last_error": (ctypes.c_char_p, [c_vp]),
    "sip_device_bytes": (c_i64, [c_vp]),
    "sip_bytes_per_iter": (c_dbl, [c_vp]),
    "sip_set_timing": (c_int, [c_vp, c_int]),
    "sip_kernel_times": (c_int, [c_vp, ctypes.POINTER(c_dbl), ctypes.POINTER(c_i64), ctypes.POINTER(c_dbl)]),
    "sip_kernel_name": (ctypes.c_char_p, [c_int]),
    "sip_apply_op": (c_int, [ctypes.POINTER(Grid), c_int, c_int, c_vp, c_vp, c_vp]),
    "sip_apply_op_t": (c_int, [ctypes.POINTER(Grid), c_int, c_int, c_vp, c_vp, c_vp]),
    "sip_op_rows": (c_i64, [ctypes.POINTER(Grid), c_int]),
    "sip_system_apply": (c_int, [ctypes.POINTER(Grid), ctypes.POINTER(c_int), ctypes.POINTER(c_dbl), c_int, c_dbl,
                                 c_int, c_vp, c_vp, c_vp]),
    "sip_project_set": (c_int, [ctypes.POINTER(Set), c_int, c_vp, c_i64, c_vp, c_vp, ctypes.POINTER(c_dbl)]),
    "sip_op_norm": (c_int, [ctypes.POINTER(Grid), c_int, c_int, c_int, c_vp, c_vp, ctypes.POINTER(c_dbl)]),
    "sip_restrict": (c_int, [ctypes.POINTER(Grid), c_int, c_vp, c_vp, c_vp]),
    "sip_prolong": (c_int, [ctypes.POINTER(Grid), c_int, c_int, c_vp, c_vp, c_vp]),
    "sip_project_l1_noalloc": (c_int, [c_int, c_vp, c_i64, c_dbl, c_vp, c_vp, ctypes.POINTER(c_dbl)]),
    "sip_test_hook": (c_int, [c_int, c_i64]),
    "sip_get_tuning": (c_int, [c_vp, ctypes.POINTER(Tuning)]),
    "sip_set_tuning": (c_int, [c_vp, ctypes.POINTER(Tuning)]),
    "sip_batch_create": (c_int, [c_int, ctypes.POINTER(Grid), ctypes.POINTER(Set), ctypes.POINTER(c_int),
                                 ctypes.POINTER(Options), ctypes.POINTER(c_vp)]),
    "sip_batch_project": (c_int, [c_vp, c_vp, c_vp, c_vp, ctypes.POINTER(Info)]),
    "sip_batch_offset": (c_i64, [c_vp, c_int]),
    "sip_dykstra_create": (c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Set), c_int, ctypes.POINTER(Options),
                                   ctypes.POINTER(c_vp)]),
    "sip_dykstra_project": (c_int, [c_vp, c_vp, c_vp, c_int, c_vp, ctypes.POINTER(DykstraInfo)]),
    "sip_server_config_default": (None, [ctypes.POINTER(ServerConfig)]),
    "sip_server_create": (c_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(c_vp)]),
    "sip_server_submit": (c_int, [c_vp, ctypes.POINTER(Grid), ctypes.POINTER(Set), c_int, c_vp, c_vp,
                                  ctypes.POINTER(c_i64)]),
    "sip_server_wait": (c_int, [c_vp, c_i64, c_dbl, ctypes.POINTER(Info), ctypes.POINTER(c_dbl)]),
    "sip_server_query_stats": (c_int, [c_vp, ctypes.POINTER(ServerStats)]),
    "sip_server_destroy": (c_int, [c_vp]),
}
NOALLOC_MAX_N = 1 << 24
HOOKS = {"fail_alloc": 1, "barrier_extra": 2, "barrier_spins": 3}

_lib = None


class SipError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def lib():
    """Load libsip.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsip.so is not built (run paper_1902_09699_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status, handle=None):
    if status != 0:
        msg = lib().sip_last_error(handle)
        raise SipError(status, msg.decode() if msg else "")


# ---------------------------------------------------------------- marshalling
def make_grid(grid):
    n = tuple(int(v) for v in grid["n"])
    h = tuple(float(v) for v in grid.get("h", (1.0,) * len(n)))
    g = Grid()
    g.ndim = len(n)
    for a in range(3):
        g.n[a] = n[a] if a < len(n) else 1
        g.h[a] = h[a] if a < len(h) else 1.0
    return g


def make_set(s):
    """A sip_set from a set dict; array-valued "lo" / "hi" (bounds) become
    per-entry bound vectors (kept alive on the returned struct).  A "BLUR"
    operator takes "axis" ("z", "x" or "y") and "taps" (k_0..k_R)."""
    c = Set()
    c.op = OPS[s["op"]]
    c.type = SET_TYPES[s["type"]]
    c._keep = []
    for name in ("lo", "hi"):
        v = s.get(name, -math.inf if name == "lo" else math.inf)
        if np.ndim(v):
            a = np.ascontiguousarray(v, dtype=np.float64)
            c._keep.append(a)
            setattr(c, name + "_vec", a.ctypes.data_as(ctypes.POINTER(c_dbl)))
            setattr(c, name, 0.0)
        else:
            setattr(c, name, float(v))
    if s.get("center") is not None:
        a = np.ascontiguousarray(s["center"], dtype=np.float64)
        c._keep.append(a)
        c.center_vec = a.ctypes.data_as(ctypes.POINTER(c_dbl))
    c.sigma = float(s.get("sigma", 0.0))
    c.sigma_rel = float(s.get("sigma_rel", 0.0))
    c.k = int(s.get("k", 0))
    c.k_frac = float(s.get("k_frac", 0.0))
    c.scope = SCOPES[s.get("scope", "all")]
    if s["op"] == "BLUR":
        taps = np.ascontiguousarray(s["taps"], dtype=np.float64).reshape(-1)
        c._keep.append(taps)
        c.blur_axis = BLUR_AXES[s["axis"]]
        c.blur_radius = taps.size - 1
        c.blur_taps = taps.ctypes.data_as(ctypes.POINTER(c_dbl))
    return c


def make_sets(sets):
    arr = (Set * len(sets))()
    keep = []
    for i, s in enumerate(sets):
        c = make_set(s)
        keep.append(c._keep)
        arr[i] = c
    arr._keep = keep  # the per-entry bound vectors the structs point to
    return arr


def default_options():
    o = Options()
    lib().sip_options_default(ctypes.byref(o))
    return o


def _dtype_code(dtype):
    import torch
    if dtype in ("f64", torch.float64, F64):
        return F64
    if dtype in ("f32", torch.float32, F32):
        return F32
    raise ValueError("dtype must be f32 or f64")


def _torch_dtype(code):
    import torch
    return torch.float64 if code == F64 else torch.float32


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return c_vp(stream.cuda_stream)


def _ptr(t):
    return c_vp(t.data_ptr())


def _dev(t, code):
    import torch
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(np.asarray(t))
    return t.to(device="cuda", dtype=_torch_dtype(code)).contiguous()


# ---------------------------------------------------------------- projector
class Projector:
    """One sip_handle: a grid, a list of (A_i, C_i) and options.

    ``opts`` keys follow sip_options (max_iter, cg_iters, adapt, rho0, gamma0,
    form="alg1"|"direct", levels, ...).  ``rho_schedule`` / ``gamma_schedule``
    (arrays [max_iter, nblocks]) replay rho / gamma; ``trace=True`` records
    the per-iteration trace.
    """

    def __init__(self, grid, sets, dtype="f32", rho_schedule=None, gamma_schedule=None, trace=False, **opts):
        L = lib()
        self.grid_dict = dict(grid)
        self.sets = [dict(s) for s in sets]
        self.code = _dtype_code(dtype)
        self.N = int(np.prod(grid["n"]))
        o = default_options()
        for k, v in opts.items():
            if k == "form":
                v = FORMS[v] if isinstance(v, str) else int(v)
            if k == "exec":
                v = EXEC[v] if isinstance(v, str) else int(v)
            if not hasattr(o, k):
                raise KeyError("unknown option %r" % (k,))
            setattr(o, k, v)
        o.dtype = self.code
        self.nblocks = len(sets) + (1 if o.form == FORMS["alg1"] else 0)
        self._keep = []
        if rho_schedule is not None:
            rs = np.ascontiguousarray(rho_schedule, dtype=np.float64)
            assert rs.shape == (o.max_iter, self.nblocks), rs.shape
            self._keep.append(rs)
            o.rho_schedule = rs.ctypes.data_as(ctypes.POINTER(c_dbl))
        if gamma_schedule is not None:
            gs = np.ascontiguousarray(gamma_schedule, dtype=np.float64)
            assert gs.shape == (o.max_iter, self.nblocks), gs.shape
            self._keep.append(gs)
            o.gamma_schedule = gs.ctypes.data_as(ctypes.POINTER(c_dbl))
        self.trace = None
        if trace:
            self.trace_w = 2 * self.nblocks + 2 + len(sets)
            self.trace = np.zeros((o.max_iter, self.trace_w))
            o.trace = self.trace.ctypes.data_as(ctypes.POINTER(c_dbl))
        self.opts = o
        self._grid = make_grid(grid)
        self._sets = make_sets(sets)
        h = c_vp()
        _check(L.sip_create(ctypes.byref(self._grid), self._sets, len(sets), ctypes.byref(o), ctypes.byref(h)))
        self.handle = h

    @property
    def torch_dtype(self):
        return _torch_dtype(self.code)

    def project(self, m, x=None, stream=None, info=True):
        """x = P(m) for a CUDA tensor m (flat, z fastest).  Returns (x, info)
        where info is a dict (or None when info=False: no synchronisation)."""
        import torch
        m = _dev(m, self.code)
        if m.numel() != self.N:
            raise ValueError("m has %d entries, grid has %d" % (m.numel(), self.N))
        if x is None:
            x = torch.empty(self.N, dtype=self.torch_dtype, device=m.device)
        inf = Info() if info else None
        _check(lib().sip_project(self.handle, _ptr(m), _ptr(x), _stream_ptr(stream),
                                 ctypes.byref(inf) if info else None), self.handle)
        if not info:
            return x, None
        p = len(self.sets)
        d = dict(iters=inf.iters, cg_steps=inf.cg_steps_total, stop_reason=inf.stop_reason,
                 r_evol=inf.r_evol, r_feas=list(inf.r_feas[:p]), rho=list(inf.rho[:self.nblocks]),
                 gamma=list(inf.gamma[:self.nblocks]), sigma=list(inf.sigma[:p]), k=list(inf.k[:p]),
                 ms=float(inf.ms), window_hits=inf.window_hits)
        return x, d

    def state_rows(self):
        """M', the entries of y (and of v): every block's rows."""
        return int(lib().sip_state_rows(self.handle))

    def get_state(self, device="cuda", stream=None):
        """(x, y, v) of the handle: after a projection, its final iterates."""
        import torch
        M = self.state_rows()
        if M < 0:  # batched or multilevel: the library reports why
            _check(lib().sip_get_state(self.handle, None, None, None, _stream_ptr(stream)), self.handle)
        x = torch.empty(self.N, dtype=self.torch_dtype, device=device)
        y = torch.empty(M, dtype=self.torch_dtype, device=device)
        v = torch.empty(M, dtype=self.torch_dtype, device=device)
        _check(lib().sip_get_state(self.handle, _ptr(x), _ptr(y), _ptr(v), _stream_ptr(stream)), self.handle)
        return x, y, v

    def set_state(self, x, y=None, v=None, rho=None, gamma=None, stream=None):
        """Start the next projection from (x, y, v) (None: zeros), with
        starting rho_i / gamma_i per block (None: rho0 / gamma0)."""
        x = _dev(x, self.code)
        y = None if y is None else _dev(y, self.code)
        v = None if v is None else _dev(v, self.code)

        def host(a):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64)
            if a.size != self.nblocks:
                raise ValueError("one value per block (%d)" % self.nblocks)
            return a
        rh, gh = host(rho), host(gamma)
        _check(lib().sip_set_state(self.handle, _ptr(x), None if y is None else _ptr(y),
                                   None if v is None else _ptr(v),
                                   None if rh is None else rh.ctypes.data_as(ctypes.POINTER(c_dbl)),
                                   None if gh is None else gh.ctypes.data_as(ctypes.POINTER(c_dbl)),
                                   _stream_ptr(stream)), self.handle)
        self._state_keep = (x, y, v)  # the copies are stream-ordered: keep the sources alive

    def get_adapt_state(self, device="cuda", stream=None):
        """Algorithm adapt-rho-gamma's saved quantities after a projection:
        (vhat, y, v, x_k0) at its last adapt call, or None before any."""
        import torch
        M = self.state_rows()
        vh, y, v = (torch.empty(M, dtype=self.torch_dtype, device=device) for _ in range(3))
        xk0 = torch.empty(self.N, dtype=self.torch_dtype, device=device)
        have = c_int(0)
        _check(lib().sip_get_adapt_state(self.handle, _ptr(vh), _ptr(y), _ptr(v), _ptr(xk0), ctypes.byref(have),
                                         _stream_ptr(stream)), self.handle)
        return (vh, y, v, xk0) if have.value else None

    def set_adapt_state(self, vhat, y, v, xk0, stream=None):
        """Load the saved quantities for the next (warm-started) projection."""
        a = [_dev(t, self.code) for t in (vhat, y, v, xk0)]
        _check(lib().sip_set_adapt_state(self.handle, *[_ptr(t) for t in a], _stream_ptr(stream)), self.handle)
        self._adapt_keep = a

    def device_bytes(self):
        return int(lib().sip_device_bytes(self.handle))

    def tuning(self):
        return get_tuning(self.handle)

    def set_tuning(self, **knobs):
        set_tuning(self.handle, **knobs)

    def bytes_per_iter(self):
        return float(lib().sip_bytes_per_iter(self.handle))

    def set_timing(self, on):
        _check(lib().sip_set_timing(self.handle, 1 if on else 0), self.handle)

    def kernel_times(self):
        n = 9  # SIP_KERNEL_CATEGORIES
        ms = (c_dbl * n)()
        la = (c_i64 * n)()
        by = (c_dbl * n)()
        _check(lib().sip_kernel_times(self.handle, ms, la, by), self.handle)
        return {lib().sip_kernel_name(i).decode(): dict(ms=ms[i], launches=la[i], bytes_per_launch=by[i])
                for i in range(n)}

    def close(self):
        if getattr(self, "handle", None):
            lib().sip_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def get_tuning(handle):
    """The plan's launch-shape knobs and what tuning measured (sip_get_tuning)."""
    t = Tuning()
    _check(lib().sip_get_tuning(handle, ctypes.byref(t)), handle)
    return {k: getattr(t, k) for k, _ in Tuning._fields_}


def set_tuning(handle, **knobs):
    """Rebuild the plan with the given knobs (others keep their values)."""
    t = Tuning()
    _check(lib().sip_get_tuning(handle, ctypes.byref(t)), handle)
    for k, v in knobs.items():
        if k == "exec":
            v = EXEC[v] if isinstance(v, str) else int(v)
        if not hasattr(t, k):
            raise KeyError("unknown knob %r" % (k,))
        setattr(t, k, v)
    _check(lib().sip_set_tuning(handle, ctypes.byref(t)), handle)


def _info_dict(inf, nsets, nblocks):
    return dict(iters=inf.iters, cg_steps=inf.cg_steps_total, stop_reason=inf.stop_reason, r_evol=inf.r_evol,
                r_feas=list(inf.r_feas[:nsets]), rho=list(inf.rho[:nblocks]), gamma=list(inf.gamma[:nblocks]),
                sigma=list(inf.sigma[:nsets]), k=list(inf.k[:nsets]), ms=float(inf.ms), window_hits=inf.window_hits)


class Dykstra:
    """Parallel Dykstra baseline (sip_dykstra_*): ``inner`` options (as for
    Projector; max_iter = iterations of each single-set sub-problem) for the
    sets' projections.  project(m, sweeps) returns (x, info dict)."""

    def __init__(self, grid, sets, dtype="f32", **inner):
        L = lib()
        self.code = _dtype_code(dtype)
        o = default_options()
        for k, v in inner.items():
            if k == "form":
                v = FORMS[v] if isinstance(v, str) else int(v)
            if k == "exec":
                v = EXEC[v] if isinstance(v, str) else int(v)
            setattr(o, k, v)
        o.dtype = self.code
        self.N = int(np.prod(grid["n"]))
        self._grid = make_grid(grid)
        self._sets = make_sets(sets)
        h = c_vp()
        _check(L.sip_dykstra_create(ctypes.byref(self._grid), self._sets, len(sets), ctypes.byref(o), ctypes.byref(h)))
        self.handle = h

    def project(self, m, sweeps, stream=None):
        import torch
        m = _dev(m, self.code)
        x = torch.empty(self.N, dtype=_torch_dtype(self.code), device=m.device)
        inf = DykstraInfo()
        _check(lib().sip_dykstra_project(self.handle, _ptr(m), _ptr(x), int(sweeps), _stream_ptr(stream),
                                         ctypes.byref(inf)), self.handle)
        return x, dict(sweeps=inf.sweeps, cg_steps=inf.cg_steps, l1_projections=inf.l1_projections, ms=float(inf.ms))

    def close(self):
        if getattr(self, "handle", None):
            lib().sip_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchProjector:
    """A batched handle: ``instances`` is a list of (grid, sets); options as
    for Projector.  project() takes the packed models (or a list of
    per-instance tensors) and returns the per-instance results."""

    def __init__(self, instances, dtype="f32", **opts):
        L = lib()
        self.code = _dtype_code(dtype)
        o = default_options()
        for k, v in opts.items():
            if k == "form":
                v = FORMS[v] if isinstance(v, str) else int(v)
            if k == "exec":
                v = EXEC[v] if isinstance(v, str) else int(v)
            setattr(o, k, v)
        o.dtype = self.code
        self.opts = o
        self.count = len(instances)
        self.grids = (Grid * self.count)(*[make_grid(g) for g, _ in instances])
        all_sets = [s for _, ss in instances for s in ss]
        self.sets = make_sets(all_sets)
        self.nsets = (c_int * self.count)(*[len(ss) for _, ss in instances])
        self.nblocks = [len(ss) + (1 if o.form == FORMS["alg1"] else 0) for _, ss in instances]
        h = c_vp()
        _check(L.sip_batch_create(self.count, self.grids, self.sets, self.nsets, ctypes.byref(o), ctypes.byref(h)))
        self.handle = h
        self.offsets = [int(L.sip_batch_offset(h, i)) for i in range(self.count + 1)]

    @property
    def torch_dtype(self):
        return _torch_dtype(self.code)

    def pack(self, models):
        import torch
        return torch.cat([_dev(m, self.code).reshape(-1) for m in models])

    def project(self, m, x=None, stream=None, info=True):
        import torch
        if isinstance(m, (list, tuple)):
            m = self.pack(m)
        m = _dev(m, self.code)
        total = self.offsets[-1]
        if m.numel() != total:
            raise ValueError("packed models hold %d elements, the batch needs %d" % (m.numel(), total))
        if x is None:
            x = torch.empty(total, dtype=self.torch_dtype, device=m.device)
        infos = (Info * self.count)() if info else None
        _check(lib().sip_batch_project(self.handle, _ptr(m), _ptr(x), _stream_ptr(stream), infos), self.handle)
        xs = [x[self.offsets[i]:self.offsets[i + 1]] for i in range(self.count)]
        if not info:
            return xs, None
        nsets = list(self.nsets)
        return xs, [_info_dict(infos[i], nsets[i], self.nblocks[i]) for i in range(self.count)]

    def set_timing(self, on):
        _check(lib().sip_set_timing(self.handle, 1 if on else 0), self.handle)

    def bytes_per_iter(self):
        return float(lib().sip_bytes_per_iter(self.handle))

    def tuning(self):
        return get_tuning(self.handle)

    def set_tuning(self, **knobs):
        set_tuning(self.handle, **knobs)

    def close(self):
        if getattr(self, "handle", None):
            lib().sip_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """A projection server (continuous batching; see sip_server_* in
    include/sip.h).  Models and results are host numpy arrays of the server's
    dtype."""

    def __init__(self, dtype="f32", budget_bytes=120 << 30, max_batch=64, max_cohorts=8, max_wait_ms=2.0, **opts):
        L = lib()
        cfg = ServerConfig()
        L.sip_server_config_default(ctypes.byref(cfg))
        self.code = _dtype_code(dtype)
        self.np_dtype = np.float64 if self.code == F64 else np.float32
        for k, v in opts.items():
            if k == "form":
                v = FORMS[v] if isinstance(v, str) else int(v)
            if k == "exec":
                v = EXEC[v] if isinstance(v, str) else int(v)
            setattr(cfg.opts, k, v)
        cfg.opts.dtype = self.code
        cfg.budget_bytes = int(budget_bytes)
        cfg.max_batch = int(max_batch)
        cfg.max_cohorts = int(max_cohorts)
        cfg.max_wait_ms = float(max_wait_ms)
        h = c_vp()
        _check(L.sip_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h
        self.pending = {}

    def submit(self, grid, sets, m):
        m = np.ascontiguousarray(np.asarray(m, dtype=self.np_dtype).reshape(-1))
        x = np.empty_like(m)
        g = make_grid(grid)
        ss = make_sets(sets)
        rid = c_i64(0)
        _check(lib().sip_server_submit(self.handle, ctypes.byref(g), ss, len(sets), m.ctypes.data_as(c_vp),
                                       x.ctypes.data_as(c_vp), ctypes.byref(rid)))
        self.pending[rid.value] = (x, len(sets), len(sets) + 1)
        return rid.value

    def wait(self, rid, timeout_ms=-1.0):
        inf = Info()
        lat = c_dbl(0.0)
        x, ns, nb = self.pending[rid]
        st = lib().sip_server_wait(self.handle, rid, float(timeout_ms), ctypes.byref(inf), ctypes.byref(lat))
        del self.pending[rid]
        _check(st)
        return x, _info_dict(inf, ns, nb), lat.value

    def stats(self):
        out = ServerStats()
        _check(lib().sip_server_query_stats(self.handle, ctypes.byref(out)))
        return {k: getattr(out, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            lib().sip_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def test_hook(name, value):
    """Host-side fault injection for the failure-handling tests (sip_test_hook)."""
    _check(lib().sip_test_hook(HOOKS[name], int(value)))


# ---------------------------------------------------------------- single steps
def op_rows(grid, op):
    return int(lib().sip_op_rows(ctypes.byref(make_grid(grid)), OPS[op]))


def apply_op(grid, op, x, stream=None):
    import torch
    code = _dtype_code(x.dtype)
    g = make_grid(grid)
    s = torch.empty(op_rows(grid, op), dtype=x.dtype, device=x.device)
    _check(lib().sip_apply_op(ctypes.byref(g), OPS[op], code, _ptr(x), _ptr(s), _stream_ptr(stream)))
    return s


def apply_op_t(grid, op, s, stream=None):
    import torch
    code = _dtype_code(s.dtype)
    g = make_grid(grid)
    x = torch.empty(int(np.prod(grid["n"])), dtype=s.dtype, device=s.device)
    _check(lib().sip_apply_op_t(ctypes.byref(g), OPS[op], code, _ptr(s), _ptr(x), _stream_ptr(stream)))
    return x


def system_apply(grid, ops, rhos, c_identity, x, stream=None):
    import torch
    code = _dtype_code(x.dtype)
    g = make_grid(grid)
    oa = (c_int * len(ops))(*[OPS[o] for o in ops])
    ra = (c_dbl * len(rhos))(*[float(r) for r in rhos])
    out = torch.empty_like(x)
    _check(lib().sip_system_apply(ctypes.byref(g), oa, ra, len(ops), float(c_identity), code, _ptr(x), _ptr(out),
                                  _stream_ptr(stream)))
    return out


def project_set(set_spec, w, stream=None):
    """y = P_C(w) with the loop's kernels; returns (y, scalar)."""
    import torch
    code = _dtype_code(w.dtype)
    s = make_set(dict(set_spec, op="I"))
    y = torch.empty_like(w)
    sc = c_dbl(0.0)
    _check(lib().sip_project_set(ctypes.byref(s), code, _ptr(w), w.numel(), _ptr(y), _stream_ptr(stream),
                                 ctypes.byref(sc)))
    return y, sc.value


def project_l1_noalloc(w, tau, y=None, stream=None):
    """l1-ball projection through the allocation-free entry point; the
    output tensor y may be passed in (nothing is allocated by the library
    either way).  Returns (y, theta)."""
    import torch
    code = _dtype_code(w.dtype)
    if not w.is_cuda or not w.is_contiguous():
        raise ValueError("w must be a contiguous CUDA tensor")
    if y is None:
        y = torch.empty_like(w)
    elif (not isinstance(y, torch.Tensor) or y.device != w.device or y.dtype != w.dtype
          or y.numel() != w.numel() or not y.is_contiguous()):
        raise ValueError("y must be a contiguous tensor on w's device with w's dtype and size")
    th = c_dbl(0.0)
    _check(lib().sip_project_l1_noalloc(code, _ptr(w), w.numel(), float(tau), _ptr(y), _stream_ptr(stream),
                                        ctypes.byref(th)))
    return y, th.value


def op_norm(grid, op, set_type, m, stream=None):
    code = _dtype_code(m.dtype)
    out = c_dbl(0.0)
    _check(lib().sip_op_norm(ctypes.byref(make_grid(grid)), OPS[op], SET_TYPES[set_type], code, _ptr(m),
                             _stream_ptr(stream), ctypes.byref(out)))
    return out.value


def coarse_grid(grid):
    n = tuple((int(v) + 1) // 2 for v in grid["n"])
    h = tuple(2.0 * float(v) for v in grid.get("h", (1.0,) * len(n)))
    return {"n": n, "h": h}


def restrict(grid, m, stream=None):
    import torch
    code = _dtype_code(m.dtype)
    mc = torch.empty(int(np.prod(coarse_grid(grid)["n"])), dtype=m.dtype, device=m.device)
    _check(lib().sip_restrict(ctypes.byref(make_grid(grid)), code, _ptr(m), _ptr(mc), _stream_ptr(stream)))
    return mc


def prolong(grid, op, uc, stream=None):
    import torch
    code = _dtype_code(uc.dtype)
    uf = torch.empty(op_rows(grid, op), dtype=uc.dtype, device=uc.device)
    _check(lib().sip_prolong(ctypes.byref(make_grid(grid)), OPS[op], code, _ptr(uc), _ptr(uf), _stream_ptr(stream)))
    return uf
