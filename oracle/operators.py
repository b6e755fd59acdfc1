"""Grid layout, the linear operators A_i and the system matrix C (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Layout (Sec. "Notation"): the model m in R^N is the vectorised n_z x n_x
(x n_y) array with z the fastest index, i.e. linear index
``iz + n_z*(ix + n_x*iy)``.  Here every vector is reshaped to a C-ordered
numpy array of shape (n_y, n_x, n_z) (n_y = 1 in 2D), so axis -1 is z,
axis -2 is x and axis -3 is y.

A grid is a dict ``{"n": (nz, nx[, ny]), "h": (hz, hx[, hy])}``.
An operator is one of the names "I", "DZ", "DX", "DY", "TV", or a blur
``("BLUR", axis, taps)`` made by ``blur_op``.
"""
import numpy as np

_AXIS = {"DZ": -1, "DX": -2, "DY": -3}
_HIDX = {"DZ": 0, "DX": 1, "DY": 2}
_BLUR_AXIS = {"z": -1, "x": -2, "y": -3}


def blur_op(axis, taps):
    """The blurring forward operator F of the data-fit formulation (Sec.
    "Introduction", the feasibility / projection problem with a data-fit
    set; the motion blur of Sec. "Joint deblurring-denoising-inpainting")
    as an operator value: a symmetric averaging kernel of 2R+1 samples along
    one grid axis, taps = (k_0, ..., k_R) with weight k_|t| on the sample t
    steps away.  Reading: the kernel is centred and symmetric (a 25-pixel
    motion blur is R = 12, k_t = 1/25) and samples outside the grid count as
    zero, so F is N x N and banded."""
    if axis not in _BLUR_AXIS:
        raise ValueError("blur axis must be 'z', 'x' or 'y'")
    taps = tuple(float(t) for t in taps)
    if len(taps) < 2:
        raise ValueError("a blur needs taps k_0..k_R with R >= 1")
    return ("BLUR", axis, taps)


def is_blur(op):
    return isinstance(op, tuple) and op[0] == "BLUR"


def _along(grid, op, v):
    """v as a grid array with the blur axis moved last."""
    X = np.asarray(v, dtype=np.float64).reshape(grid_shape(grid))
    return np.moveaxis(X, _BLUR_AXIS[op[1]], -1)


def _back(grid, op, Y):
    return np.moveaxis(Y, -1, _BLUR_AXIS[op[1]]).reshape(-1)


def blur_apply(grid, op, x):
    """(F x)[j] = sum over |t| <= R of k_|t| x[j + t] along the axis, the
    terms whose sample j + t falls outside the grid left out: row j of F
    gathers the samples around j."""
    if len(grid["n"]) < 3 and op[1] == "y":
        raise ValueError("no y axis in 2D")
    taps = op[2]
    X = _along(grid, op, x)
    n = X.shape[-1]
    Y = taps[0] * X
    for t in range(1, len(taps)):
        if t >= n:
            break
        Y[..., :n - t] += taps[t] * X[..., t:]   # sample j + t
        Y[..., t:] += taps[t] * X[..., :n - t]   # sample j - t
    return _back(grid, op, Y)


def blur_apply_t(grid, op, u):
    """(F^T u)[i] = sum over rows j of F[j, i] u[j]: every row j scatters
    k_|i - j| u[j] to the samples i within R of it (the columns of F)."""
    taps = op[2]
    U = _along(grid, op, u)
    n = U.shape[-1]
    Z = np.zeros_like(U)
    R = len(taps) - 1
    for j in range(n):
        for i in range(max(0, j - R), min(n, j + R + 1)):
            Z[..., i] += taps[abs(i - j)] * U[..., j]
    return _back(grid, op, Z)


def grid_shape(grid):
    """(ny, nx, nz) array shape of a 2D or 3D grid (Sec. "Notation")."""
    n = tuple(int(v) for v in grid["n"])
    nz, nx = n[0], n[1]
    ny = n[2] if len(n) > 2 else 1
    return (ny, nx, nz)


def grid_h(grid):
    h = tuple(float(v) for v in grid.get("h", (1.0,) * len(grid["n"])))
    return h + (1.0,) * (3 - len(h))


def grid_size(grid):
    s = grid_shape(grid)
    return s[0] * s[1] * s[2]


def tv_parts(grid):
    """Difference operators stacked by the anisotropic TV operator.

    In 2D the paper stacks the vertical and the horizontal derivative
    (Sec. "Parallel Dykstra versus PARSDMM", TV operator A); in 3D the y
    derivative is appended.  Order: D_z, D_x, (D_y).
    """
    return ["DZ", "DX"] + (["DY"] if len(grid["n"]) > 2 else [])


def diff_shape(grid, name):
    """Output array shape of a forward difference: one fewer sample along
    the differenced axis, no boundary rows (Eq. FD_mat)."""
    s = list(grid_shape(grid))
    s[_AXIS[name]] -= 1
    return tuple(s)


def out_size(grid, op):
    """M_i, the number of rows of A_i."""
    if op == "I" or is_blur(op):
        return grid_size(grid)
    if op == "TV":
        return sum(out_size(grid, d) for d in tv_parts(grid))
    return int(np.prod(diff_shape(grid, op)))


def forward_diff(grid, name, x):
    """(D x)[i] = (x[i+1] - x[i]) / h along one axis (Eq. FD_mat): the
    bidiagonal [-1, 1] matrix scaled by 1/h, applied along z, x or y."""
    a = _AXIS[name]
    h = grid_h(grid)[_HIDX[name]]
    X = np.asarray(x, dtype=np.float64).reshape(grid_shape(grid))
    n = X.shape[a]
    hi = [slice(None)] * 3
    lo = [slice(None)] * 3
    hi[a] = slice(1, n)
    lo[a] = slice(0, n - 1)
    return ((X[tuple(hi)] - X[tuple(lo)]) / h).reshape(-1)


def adjoint_diff(grid, name, u):
    """Transpose of ``forward_diff``: (D^T u)[i] = (u[i-1] - u[i]) / h with
    u[-1] = u[n-1] = 0 (the columns of the bidiagonal matrix of Eq. FD_mat)."""
    a = _AXIS[name]
    h = grid_h(grid)[_HIDX[name]]
    U = np.asarray(u, dtype=np.float64).reshape(diff_shape(grid, name))
    out = np.zeros(grid_shape(grid))
    n = out.shape[a]
    hi = [slice(None)] * 3
    lo = [slice(None)] * 3
    hi[a] = slice(1, n)
    lo[a] = slice(0, n - 1)
    out[tuple(lo)] -= U
    out[tuple(hi)] += U
    return (out / h).reshape(-1)


def apply(grid, op, x):
    """s = A x for A in {I, D_z, D_x, D_y, TV} (set table, Sec. "Software")
    or a blur F (``blur_op``)."""
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    if is_blur(op):
        return blur_apply(grid, op, x)
    if op == "I":
        return x.copy()
    if op == "TV":
        return np.concatenate([forward_diff(grid, d, x) for d in tv_parts(grid)])
    return forward_diff(grid, op, x)


def apply_t(grid, op, y):
    """A^T y, the adjoint of ``apply``."""
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    if is_blur(op):
        return blur_apply_t(grid, op, y)
    if op == "I":
        return y.copy()
    if op == "TV":
        out = np.zeros(grid_size(grid))
        off = 0
        for d in tv_parts(grid):
            m = out_size(grid, d)
            out += adjoint_diff(grid, d, y[off:off + m])
            off += m
        return out
    return adjoint_diff(grid, op, y)


def system_apply(grid, ops, rhos, c_identity, x):
    """C x with C = sum_i rho_i A_i^T A_i + c_identity * I (Eq. sys_mat).

    In the paper's form the identity term is the extra block A_{p+1} = I_N
    with weight rho_{p+1}; in the direct form it is the 1 from the distance
    term.  Written from the definition: each A_i^T A_i x is formed by
    applying A_i and then A_i^T.
    """
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    out = c_identity * x
    for op, rho in zip(ops, rhos):
        out = out + rho * apply_t(grid, op, apply(grid, op, x))
    return out


def norm_of(grid, op, set_type, m):
    """Norm of A m matching a set's norm: the l1 norm for l1 sets and the
    l2 norm for l2 sets.  Used to resolve set radii given relative to the
    model, e.g. tau = 0.5 * TV(m) where TV(m) = ||TV m||_1 (anisotropic TV,
    Sec. "Parallel Dykstra versus PARSDMM")."""
    s = apply(grid, op, m)
    if set_type == "l1":
        return float(np.sum(np.abs(s)))
    if set_type == "l2":
        return float(np.sqrt(np.sum(s * s)))
    raise ValueError("norm_of: set type %r has no radius" % (set_type,))
