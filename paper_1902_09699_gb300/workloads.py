"""Seeded synthetic inputs shaped like the paper's 2D/3D model grids.

This module only makes input data (models m, set lists, option values).  It
holds none of the projection method's arithmetic, so both the CUDA library's
tests/benchmark and the CPU oracle can consume its output.

Models (stand-ins for the paper's geological models and images, which are
not available): smooth Gaussian random fields and layered media with a
Gaussian anomaly, plus Gaussian noise.  All randomness is numpy's Philox
counter-based generator seeded per workload.

Set dicts: {"op": "I"|"DZ"|"DX"|"DY"|"TV"|"BLUR", "type": "bounds"|"l1"|"l2"|
"card", "lo", "hi", "sigma", "sigma_rel", "k", "k_frac"}; ``sigma_rel`` asks
for a radius relative to the projected model's own norm, ``k_frac`` for a
cardinality relative to the grid size; a "BLUR" operator also takes "axis"
and "taps".
"""
import math

import numpy as np

INF = math.inf


def rng(seed):
    return np.random.Generator(np.random.Philox(int(seed)))


def _smooth(noise, corr_len):
    """Periodic convolution of white noise with a Gaussian of standard
    deviation ``corr_len`` cells, via the FFT."""
    F = np.fft.rfftn(noise)
    shape = noise.shape
    g = None
    for ax, n in enumerate(shape):
        if ax == len(shape) - 1:
            f = np.fft.rfftfreq(n)
        else:
            f = np.fft.fftfreq(n)
        k = np.exp(-2.0 * (math.pi * f * corr_len) ** 2)
        sh = [1] * len(shape)
        sh[ax] = k.size
        k = k.reshape(sh)
        g = k if g is None else g * k
    return np.fft.irfftn(F * g, s=shape, axes=tuple(range(len(shape))))


def _to_range(a, lo, hi):
    amin, amax = float(a.min()), float(a.max())
    if amax == amin:
        return np.full_like(a, 0.5 * (lo + hi))
    return lo + (a - amin) * ((hi - lo) / (amax - amin))


def grf(n, corr_len=8.0, lo=1.5, hi=4.5, noise=0.1, seed=0):
    """Smooth random field on a grid n = (nz, nx[, ny]) mapped affinely to
    [lo, hi], plus N(0, noise^2).  Returned flat with z fastest."""
    n = tuple(int(v) for v in n)
    shape = tuple(reversed(n))             # (ny, nx, nz) / (nx, nz), C order
    g = rng(seed)
    f = _smooth(g.standard_normal(shape), corr_len)
    f = _to_range(f, lo, hi)
    f = f + noise * g.standard_normal(shape)
    return np.ascontiguousarray(f.reshape(-1))


def layered(n, n_layers=20, lo=1.5, hi=4.5, blob_amp=0.5, blob_std=40.0,
            noise=0.05, seed=0):
    """2D layered medium: ``n_layers`` flat layers (interfaces uniform over
    depth, values drawn uniformly in [lo, hi] without repetition) plus one
    Gaussian blob (amplitude, standard deviation in cells, random centre)
    plus N(0, noise^2).  n = (nz, nx); flat with z fastest."""
    nz, nx = int(n[0]), int(n[1])
    g = rng(seed)
    cuts = np.sort(g.choice(np.arange(1, nz), size=n_layers - 1, replace=False))
    vals = g.uniform(lo, hi, size=n_layers)
    while len(np.unique(vals)) < n_layers:
        vals = g.uniform(lo, hi, size=n_layers)
    col = np.empty(nz)
    edges = np.concatenate([[0], cuts, [nz]])
    for j in range(n_layers):
        col[edges[j]:edges[j + 1]] = vals[j]
    f = np.tile(col, (nx, 1))               # (nx, nz)
    cz, cx = g.uniform(0, nz), g.uniform(0, nx)
    iz = np.arange(nz)[None, :]
    ix = np.arange(nx)[:, None]
    f = f + blob_amp * np.exp(-((iz - cz) ** 2 + (ix - cx) ** 2) / (2.0 * blob_std ** 2))
    f = f + noise * g.standard_normal(f.shape)
    return np.ascontiguousarray(f.reshape(-1))


# --------------------------------------------------------------------------
# The five workloads
# --------------------------------------------------------------------------
def small_2d(n=(64, 64), seed=1001):
    """2D 64 x 64, FP64, plain loop: bounds [2, 4] on x, anisotropic TV
    l1 ball tau = 0.5 TV(m), D_z x >= 0; 200 iterations, 5 warm-started CG
    steps, fixed rho = 1, gamma = 1."""
    m = grf(n, corr_len=8.0, noise=0.1, seed=seed)
    sets = [
        {"op": "I", "type": "bounds", "lo": 2.0, "hi": 4.0},
        {"op": "TV", "type": "l1", "sigma_rel": 0.5},
        {"op": "DZ", "type": "bounds", "lo": 0.0, "hi": INF},
    ]
    opts = dict(max_iter=200, cg_iters=5, adapt=0, rho0=1.0, gamma0=1.0)
    return dict(name="2d-64x64-f64-bounds-tv-dz", grid={"n": tuple(n), "h": (1.0, 1.0)},
                m=m, sets=sets, opts=opts, dtype="f64")


def layered_2d(n=(512, 1024), seed=1002):
    """2D 512 x 1024 layered model, FP32 bulk with FP64 reductions:
    bounds [2, 4]; TV l1 ball tau = 0.3 TV(m); l2 ball on D_x x with
    sigma = 0.5 ||D_x m||; card(D_z x) <= 2% of N; D_z x in [-0.1, 0.5];
    adaptive rho, gamma = 1.5; 500 iterations, 5 CG steps."""
    m = layered(n, seed=seed)
    sets = [
        {"op": "I", "type": "bounds", "lo": 2.0, "hi": 4.0},
        {"op": "TV", "type": "l1", "sigma_rel": 0.3},
        {"op": "DX", "type": "l2", "sigma_rel": 0.5},
        {"op": "DZ", "type": "card", "k_frac": 0.02},
        {"op": "DZ", "type": "bounds", "lo": -0.1, "hi": 0.5},
    ]
    opts = dict(max_iter=500, cg_iters=5, adapt=1, rho0=1.0, gamma0=1.5)
    return dict(name="2d-%dx%d-layered-5sets" % tuple(n), grid={"n": tuple(n), "h": (1.0, 1.0)},
                m=m, sets=sets, opts=opts, dtype="f32")


def lines_2d(n=(512, 1024), seed=1006):
    """2D 512 x 1024 layered model under the set list of the paper's seismic
    example with per-row and per-column sets (its rank constraint is left
    out): bounds [2, 4]; card(D_z x) <= n_x and card(D_x x) <= n_z over the
    whole model; at most 2 nonzeros of D_x in every row and of D_z in every
    column.  FP32, adaptive rho, gamma = 1.5, 300 iterations, 5 CG steps."""
    m = layered(n, seed=seed)
    nz, nx = int(n[0]), int(n[1])
    sets = [
        {"op": "I", "type": "bounds", "lo": 2.0, "hi": 4.0},
        {"op": "DZ", "type": "card", "k": nx},
        {"op": "DX", "type": "card", "k": nz},
        {"op": "DX", "type": "card", "k": 2, "scope": "x"},
        {"op": "DZ", "type": "card", "k": 2, "scope": "z"},
    ]
    opts = dict(max_iter=300, cg_iters=5, adapt=1, rho0=1.0, gamma0=1.5)
    return dict(name="2d-%dx%d-layered-rowcol-card" % tuple(n), grid={"n": tuple(n), "h": (1.0, 1.0)},
                m=m, sets=sets, opts=opts, dtype="f32")


def motion_blur_taps(length=25):
    """Taps k_0..k_R of a centred box of ``length`` = 2R + 1 samples (a
    straight motion blur of that many pixels), each 1 / length."""
    if length < 3 or length % 2 == 0:
        raise ValueError("an odd length >= 3")
    return tuple([1.0 / length] * (length // 2 + 1))


def deblur_2d(n=(1100, 1100), seed=1007, blur_len=25, frac=0.2, noise=10.0, bound=15.0, axis="x"):
    """Stand-in for the paper's joint deblurring-denoising-inpainting example
    (Sec. "Joint deblurring-denoising-inpainting": 1100 x 1100 grayscale
    patches in [0, 255], a known 25-pixel motion blur, 20% of the pixels
    observed with uniform noise in [-10, 10], data fit with the
    over-estimate [-15, 15]).  The image is a smooth random field mapped to
    [0, 255]; the observed data are its blur (scipy's zero-padded 1D
    convolution with a box of ``blur_len`` samples along ``axis``) at a
    random ``frac`` of the pixels plus uniform noise.  Data-fit set
    {-bound <= F x - d <= bound} on the observed pixels (+-inf elsewhere),
    with the model-property sets [0, 255] bounds, a TV l1 ball and slope
    bounds on D_z x and D_x x whose sizes come from a second training image
    of the same generator.  Initial guess: d at observed pixels, their mean
    elsewhere.  FP32, adaptive rho, gamma = 1.5, 5 CG steps."""
    from scipy import ndimage
    g = rng(seed)
    nz, nx = int(n[0]), int(n[1])
    truth = grf((nz, nx), corr_len=6.0, lo=0.0, hi=255.0, noise=0.0, seed=seed)
    train = grf((nz, nx), corr_len=6.0, lo=0.0, hi=255.0, noise=0.0, seed=seed + 1)
    taps = motion_blur_taps(blur_len)
    kfull = np.array(taps[::-1] + taps[1:])
    ax = {"z": 1, "x": 0}[axis]  # axis of the (n_x, n_z) array
    blurred = ndimage.convolve1d(truth.reshape(nx, nz), kfull, axis=ax, mode="constant", cval=0.0).reshape(-1)
    obs = g.uniform(size=truth.size) < frac
    d = blurred + g.uniform(-noise, noise, truth.size)
    lo = np.where(obs, d - bound, -INF)
    hi = np.where(obs, d + bound, INF)
    m = np.where(obs, d, float(d[obs].mean()))
    T = train.reshape(nx, nz)
    dz, dx = np.diff(T, axis=1), np.diff(T, axis=0)
    tv = float(np.abs(dz).sum() + np.abs(dx).sum())
    sz, sx = float(np.abs(dz).max()), float(np.abs(dx).max())
    sets = [
        {"op": "BLUR", "axis": axis, "taps": taps, "type": "bounds", "lo": lo, "hi": hi},
        {"op": "I", "type": "bounds", "lo": 0.0, "hi": 255.0},
        {"op": "TV", "type": "l1", "sigma": tv},
        {"op": "DZ", "type": "bounds", "lo": -sz, "hi": sz},
        {"op": "DX", "type": "bounds", "lo": -sx, "hi": sx},
    ]
    opts = dict(max_iter=300, cg_iters=5, adapt=1, rho0=1.0, gamma0=1.5)
    return dict(name="2d-%dx%d-deblur-inpaint-blur%d" % (nz, nx, blur_len), grid={"n": (nz, nx), "h": (1.0, 1.0)},
                m=m, sets=sets, opts=opts, dtype="f32", truth=truth, obs=obs)


def grf_3d(n=(256, 256, 128), seed=1003):
    """3D 256 x 256 x 128 (n_z, n_x, n_y) random field, FP32: bounds [2, 4];
    3D TV l1 ball tau = 0.4 TV(m); D_z x >= 0; card(D_x x) <= 1% of N;
    two-level multilevel, 300 iterations per level."""
    m = grf(n, corr_len=8.0, noise=0.1, seed=seed)
    sets = [
        {"op": "I", "type": "bounds", "lo": 2.0, "hi": 4.0},
        {"op": "TV", "type": "l1", "sigma_rel": 0.4},
        {"op": "DZ", "type": "bounds", "lo": 0.0, "hi": INF},
        {"op": "DX", "type": "card", "k_frac": 0.01},
    ]
    opts = dict(max_iter=300, cg_iters=5, adapt=1, rho0=1.0, gamma0=1.5)
    return dict(name="3d-%dx%dx%d-grf-4sets-ml2" % tuple(n), grid={"n": tuple(n), "h": (1.0, 1.0, 1.0)},
                m=m, sets=sets, opts=opts, dtype="f32", levels=2)


_BATCH_SET_POOL = [
    {"op": "I", "type": "bounds", "lo": 2.0, "hi": 4.0},
    {"op": "TV", "type": "l1", "sigma_rel": 0.5},
    {"op": "DZ", "type": "bounds", "lo": -0.1, "hi": 0.5},
    {"op": "DZ", "type": "card", "k_frac": 0.02},
]


def ragged_batch(count=512, lo=32, hi=512, seed=1004):
    """``count`` independent 2D instances with n_z, n_x uniform in
    [lo, hi]; each has 2-5 sets drawn with replacement from {bounds, TV l1
    ball, D_z bounds, card(D_z x) 2%}; models as in ``small_2d``; FP32 with
    FP64 reductions, 300 iterations each."""
    g = rng(seed)
    out = []
    for i in range(count):
        nz, nx = int(g.integers(lo, hi + 1)), int(g.integers(lo, hi + 1))
        ns = int(g.integers(2, 6))
        pick = g.integers(0, len(_BATCH_SET_POOL), size=ns)
        sets = [dict(_BATCH_SET_POOL[j]) for j in pick]
        m = grf((nz, nx), corr_len=8.0, noise=0.1, seed=seed * 100000 + i)
        out.append(dict(grid={"n": (nz, nx), "h": (1.0, 1.0)}, m=m, sets=sets))
    opts = dict(max_iter=300, cg_iters=5, adapt=1, rho0=1.0, gamma0=1.5)
    return dict(name="ragged-%d-2d-%d..%d" % (count, lo, hi), instances=out, opts=opts, dtype="f32")


def request_stream(rate=2000.0, seconds=60.0, seed=1005, max_requests=None):
    """Poisson arrivals (mean ``rate`` per second); sizes log-uniform: 2D
    64^2..1024^2 and 3D 64^3..192^3 (half each); 2-6 sets drawn from the
    small_2d set types; stop at relative feasibility 1e-3 or 500
    iterations.  Returns a list of (arrival_s, request dict); models are
    generated lazily by ``request_model``."""
    g = rng(seed)
    t = 0.0
    reqs = []
    while True:
        t += float(g.exponential(1.0 / rate))
        if t > seconds or (max_requests is not None and len(reqs) >= max_requests):
            break
        is3d = bool(g.integers(0, 2))
        if is3d:
            n = int(round(math.exp(g.uniform(math.log(64), math.log(192)))))
            dims = (n, n, n)
        else:
            n = int(round(math.exp(g.uniform(math.log(64), math.log(1024)))))
            dims = (n, n)
        ns = int(g.integers(2, 7))
        pool = small_2d()["sets"]
        pick = g.integers(0, len(pool), size=ns)
        sets = [dict(pool[j]) for j in pick]
        reqs.append((t, dict(grid={"n": dims, "h": (1.0,) * len(dims)}, sets=sets,
                             seed=int(g.integers(0, 2 ** 31)))))
    return reqs


def request_model(req):
    return grf(req["grid"]["n"], corr_len=8.0, noise=0.1, seed=req["seed"])
