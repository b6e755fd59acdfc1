"""Pins for oracle/operators.py against the paper's matrix definitions.

Eq. FD_mat defines D_z as the (n_z-1) x n_z bidiagonal matrix with -1 on the
diagonal and +1 above it, scaled by 1/h_z; the x and y derivatives are the
same matrix along their axis; TV stacks them (Sec. "Parallel Dykstra versus
PARSDMM").  These tests build those matrices entry by entry with index loops
and compare, plus adjoint and closed-form checks.
"""
import itertools

import numpy as np
import pytest

from oracle import operators as ops

GRIDS = [
    {"n": (5, 4), "h": (1.0, 1.0)},
    {"n": (6, 3), "h": (0.5, 2.0)},
    {"n": (4, 3, 5), "h": (1.0, 1.0, 1.0)},
    {"n": (3, 5, 2), "h": (2.0, 0.25, 3.0)},
    {"n": (1, 7), "h": (1.0, 1.0)},
]


def lin(iz, ix, iy, n):
    return iz + n[0] * (ix + n[1] * iy)


def explicit_diff_matrix(grid, axis):
    """Rows: every (iz, ix, iy) of the output grid (z fastest); entries -1/h
    at the sample, +1/h at its successor along ``axis``."""
    n = tuple(grid["n"]) + ((1,) if len(grid["n"]) == 2 else ())
    h = tuple(grid["h"]) + ((1.0,) if len(grid["h"]) == 2 else ())
    out_n = list(n)
    out_n[axis] -= 1
    N = n[0] * n[1] * n[2]
    rows = []
    for iy in range(out_n[2]):
        for ix in range(out_n[1]):
            for iz in range(out_n[0]):
                r = np.zeros(N)
                src = [iz, ix, iy]
                dst = list(src)
                dst[axis] += 1
                r[lin(*src, n)] -= 1.0 / h[axis]
                r[lin(*dst, n)] += 1.0 / h[axis]
                rows.append(r)
    return np.array(rows).reshape(-1, N)


def dense(grid, op):
    N = ops.grid_size(grid)
    return np.stack([ops.apply(grid, op, e) for e in np.eye(N)], axis=1)


@pytest.mark.parametrize("grid", GRIDS)
def test_difference_matrices_match_eq_fd_mat(grid):
    for name, axis in (("DZ", 0), ("DX", 1), ("DY", 2)):
        if axis >= len(grid["n"]):
            continue
        E = explicit_diff_matrix(grid, axis)
        A = dense(grid, name)
        assert A.shape == E.shape
        assert np.array_equal(A, E)


@pytest.mark.parametrize("grid", GRIDS)
def test_tv_is_stack_of_differences(grid):
    parts = [explicit_diff_matrix(grid, a) for a in range(len(grid["n"]))]
    E = np.vstack(parts)
    assert np.array_equal(dense(grid, "TV"), E)
    assert ops.out_size(grid, "TV") == E.shape[0]


@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("op", ["I", "DZ", "DX", "DY", "TV"])
def test_adjoint_dot_product(grid, op):
    if op == "DY" and len(grid["n"]) == 2:
        pytest.skip("2D grid has no y axis")
    g = np.random.default_rng(7)
    x = g.standard_normal(ops.grid_size(grid))
    y = g.standard_normal(ops.out_size(grid, op))
    lhs = float(ops.apply(grid, op, x) @ y)
    rhs = float(x @ ops.apply_t(grid, op, y))
    assert abs(lhs - rhs) <= 1e-12 * (1 + abs(lhs))
    # and the adjoint equals the transpose of the explicit matrix
    A = dense(grid, op)
    assert np.allclose(ops.apply_t(grid, op, y), A.T @ y, rtol=0, atol=1e-13)


def test_dz_normal_matrix_is_neumann_tridiagonal():
    # D_z^T D_z for one column: diag (1, 2, ..., 2, 1), off-diagonals -1, / h^2
    for nz, h in ((2, 1.0), (5, 1.0), (7, 0.5)):
        grid = {"n": (nz, 1), "h": (h, 1.0)}
        T = np.zeros((nz, nz))
        for i in range(nz):
            T[i, i] = 2.0
            if i > 0:
                T[i, i - 1] = -1.0
            if i < nz - 1:
                T[i, i + 1] = -1.0
        T[0, 0] = T[-1, -1] = 1.0
        T /= h * h
        A = dense(grid, "DZ")
        assert np.allclose(A.T @ A, T, atol=1e-14)


def test_tv_of_linear_ramp_closed_form():
    # m = a*z + b*x (+ c*y): every D_z entry is a/h_z, etc.
    nz, nx, ny = 9, 7, 4
    a, b, c = 0.3, -1.7, 0.6
    for dim in (2, 3):
        n = (nz, nx) if dim == 2 else (nz, nx, ny)
        h = (0.5, 2.0) if dim == 2 else (0.5, 2.0, 1.5)
        grid = {"n": n, "h": h}
        iy, ix, iz = np.meshgrid(np.arange(ny if dim == 3 else 1), np.arange(nx), np.arange(nz), indexing="ij")
        m = (a * iz * h[0] + b * ix * h[1] + (c * iy * h[2] if dim == 3 else 0.0)).reshape(-1)
        tv = ops.norm_of(grid, "TV", "l1", m)
        expect = abs(a) * (nz - 1) * nx + abs(b) * nz * (nx - 1)
        if dim == 3:
            expect = expect * ny + abs(c) * nz * nx * (ny - 1)
        assert tv == pytest.approx(expect, rel=1e-13)


@pytest.mark.parametrize("grid", GRIDS[:4])
def test_system_matrix_against_explicit_blocks(grid):
    ops_list = ["I", "TV", "DZ", "DX"]
    rhos = [0.7, 1.3, 2.1, 0.4]
    c_id = 1.9
    N = ops.grid_size(grid)
    C = c_id * np.eye(N)
    for op, r in zip(ops_list, rhos):
        if op == "I":
            A = np.eye(N)
        elif op == "TV":
            A = np.vstack([explicit_diff_matrix(grid, a) for a in range(len(grid["n"]))])
        else:
            A = explicit_diff_matrix(grid, {"DZ": 0, "DX": 1}[op])
        C += r * A.T @ A
    x = np.random.default_rng(3).standard_normal(N)
    assert np.allclose(ops.system_apply(grid, ops_list, rhos, c_id, x), C @ x, atol=1e-12)
    # Eq. sys_mat: C is symmetric positive definite
    assert np.allclose(C, C.T)
    assert np.linalg.eigvalsh(C).min() > 0


def test_layout_is_z_fastest():
    grid = {"n": (3, 4, 2), "h": (1.0, 1.0, 1.0)}
    m = np.zeros(24)
    for iz, ix, iy in itertools.product(range(3), range(4), range(2)):
        m[iz + 3 * (ix + 4 * iy)] = iz  # depends on z only
    assert np.all(ops.apply(grid, "DX", m) == 0)
    assert np.all(ops.apply(grid, "DY", m) == 0)
    assert np.all(ops.apply(grid, "DZ", m) == 1)


# --------------------------------------------------------------------------
# Blurring forward operator F of the data-fit set (Sec. "Introduction",
# data-fit formulation; Sec. "Joint deblurring-denoising-inpainting").
# --------------------------------------------------------------------------
BLUR_CASES = [
    ({"n": (9, 6)}, "z", (0.5, 0.25)),
    ({"n": (9, 6)}, "x", (0.4, 0.2, 0.1)),
    ({"n": (5, 4, 6)}, "y", (0.3, 0.2, 0.1, 0.05)),
    ({"n": (3, 8)}, "z", (0.2,) * 5),      # R = 4 > n_z: every sample sees both ends
    ({"n": (30, 2)}, "z", (1.0 / 25,) * 13),  # the 25-sample motion blur
]
_AX = {"z": 0, "x": 1, "y": 2}


def convolve_matrix(grid, axis, taps):
    """F from scipy's 1D convolution with zero padding ("constant" mode),
    applied to every unit vector: column i of F is the blur of e_i."""
    nd = pytest.importorskip("scipy.ndimage")
    shape = ops.grid_shape(grid)
    kfull = np.array(taps[::-1] + taps[1:])
    N = ops.grid_size(grid)
    cols = []
    for e in np.eye(N):
        E = e.reshape(shape)
        cols.append(nd.convolve1d(E, kfull, axis=2 - _AX[axis], mode="constant", cval=0.0).reshape(-1))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("grid,axis,taps", BLUR_CASES)
def test_blur_matches_scipy_convolution(grid, axis, taps):
    op = ops.blur_op(axis, taps)
    F = convolve_matrix(grid, axis, taps)
    x = np.random.default_rng(11).standard_normal(F.shape[1])
    assert np.allclose(ops.apply(grid, op, x), F @ x, rtol=0, atol=1e-14)
    assert np.allclose(ops.apply_t(grid, op, x), F.T @ x, rtol=0, atol=1e-14)
    assert ops.out_size(grid, op) == F.shape[0] == F.shape[1]
    # a centred symmetric kernel: F is symmetric
    assert np.array_equal(F, F.T)


@pytest.mark.parametrize("grid,axis,taps", BLUR_CASES)
def test_blur_adjoint_dot_product(grid, axis, taps):
    op = ops.blur_op(axis, taps)
    g = np.random.default_rng(12)
    N = ops.grid_size(grid)
    x, u = g.standard_normal(N), g.standard_normal(N)
    lhs = float(np.dot(ops.apply(grid, op, x), u))
    rhs = float(np.dot(x, ops.apply_t(grid, op, u)))
    assert lhs == pytest.approx(rhs, rel=1e-13, abs=1e-13)


def test_box_blur_of_a_constant_closed_form():
    """A normalised box of 2R+1 samples keeps a constant c in the interior
    and gives c (samples inside the grid) / (2R+1) within R of an edge."""
    R, n, c = 3, 11, 2.5
    grid = {"n": (n, 2)}
    op = ops.blur_op("z", (1.0 / (2 * R + 1),) * (R + 1))
    y = ops.apply(grid, op, np.full(2 * n, c)).reshape(2, n)
    for j in range(n):
        inside = min(n - 1, j + R) - max(0, j - R) + 1
        assert y[0, j] == pytest.approx(c * inside / (2 * R + 1), rel=1e-14)
        assert y[1, j] == y[0, j]


def test_blur_normal_matrix_interior_is_autocorrelation():
    """Rows of F^T F at least 2R samples from both ends hold the kernel's
    autocorrelation a_d = sum_t k_t k_{t+d} at offset d (|d| <= 2R)."""
    taps = (0.35, 0.2, 0.1, 0.025)
    R, n = len(taps) - 1, 20
    grid = {"n": (n, 1)}
    op = ops.blur_op("z", taps)
    kfull = np.array(taps[::-1] + taps[1:])
    auto = np.correlate(kfull, kfull, mode="full")   # offsets -2R..2R
    FtF = np.stack([ops.apply_t(grid, op, ops.apply(grid, op, e)) for e in np.eye(n)], axis=1)
    for i in range(2 * R, n - 2 * R):
        row = np.zeros(n)
        row[i - 2 * R:i + 2 * R + 1] = auto
        assert np.allclose(FtF[i], row, rtol=0, atol=1e-15)
    # near an end some products are missing: the diagonal is smaller there
    assert FtF[0, 0] < auto[2 * R] - 1e-3


@pytest.mark.parametrize("grid,axis,taps", BLUR_CASES[:3])
def test_system_matrix_with_a_blur(grid, axis, taps):
    """Eq. sys_mat with a blur block: C = c I + rho_D D_z^T D_z + rho_F F^T F."""
    op = ops.blur_op(axis, taps)
    F = convolve_matrix(grid, axis, taps)
    N = F.shape[0]
    D = explicit_diff_matrix(dict(grid, h=(1.0,) * len(grid["n"])), 0)
    C = 1.3 * np.eye(N) + 0.7 * D.T @ D + 2.2 * F.T @ F
    x = np.random.default_rng(13).standard_normal(N)
    got = ops.system_apply(dict(grid, h=(1.0,) * len(grid["n"])), ["DZ", op], [0.7, 2.2], 1.3, x)
    assert np.allclose(got, C @ x, rtol=0, atol=1e-12)


def test_blur_op_rejects_bad_arguments():
    with pytest.raises(ValueError):
        ops.blur_op("w", (0.5, 0.25))
    with pytest.raises(ValueError):
        ops.blur_op("z", (1.0,))
    with pytest.raises(ValueError):
        ops.apply({"n": (4, 4)}, ops.blur_op("y", (0.5, 0.25)), np.zeros(16))
