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
