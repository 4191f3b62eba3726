"""Spatial grid and second-order one-sided stencils (oracle; test infrastructure only).

Sec. 3.3.2 of the paper: cells idx(i,j,k) = (k-1) n_x n_y + (j-1) n_x + i (x fastest)
and the stencils D^{+,-}_d in R^{n x n} with, for d = x,
  D^+ : diagonal +3/(2 dx), (i+1) -4/(2 dx), (i+2) +1/(2 dx)
  D^- : diagonal -3/(2 dx), (i-1) +4/(2 dx), (i-2) -1/(2 dx)
and likewise along y and z. Both approximate -d/dx: D^+ one-sided forward,
D^- one-sided backward.

Reading of the boundary (the paper states none): two ghost layers of zero on
every face, i.e. vacuum inflow; the collided flux has no external source.

Pins (tests/test_oracle_grid.py): the explicit sparse matrices assembled entry by
entry from the paper's coefficients; second-order convergence on a smooth
function; telescoping of the cell sum of the upwind operator to the boundary
flux (3 u_n - u_{n-1})/2. The transposed application ``apply_DT`` (used by the
discrete adjoint) is pinned against the transpose of the assembled matrix
(tests/test_oracle_adjoint.py).
"""
from __future__ import annotations

import numpy as np

AXIS_OF = {0: 2, 1: 1, 2: 0}  # direction d (x,y,z) -> axis of the (nz, ny, nx, c) view


def apply_D(Y: np.ndarray, dims, d: int, sign: int, delta: float) -> np.ndarray:
    """(D^{sign}_d Y) for Y of shape (n, c) on a grid dims = (nx, ny, nz)."""
    nx, ny, nz = dims
    c = Y.shape[1]
    V = Y.reshape(nz, ny, nx, c)
    ax = AXIS_OF[d]
    pad = [(0, 0)] * 4
    pad[ax] = (2, 2)
    P = np.pad(V, pad)
    L = V.shape[ax]

    def shifted(s):
        sl = [slice(None)] * 4
        sl[ax] = slice(2 + s, 2 + s + L)
        return P[tuple(sl)]

    if sign > 0:
        out = (3.0 * V - 4.0 * shifted(+1) + shifted(+2)) / (2.0 * delta)
    else:
        out = (-3.0 * V + 4.0 * shifted(-1) - shifted(-2)) / (2.0 * delta)
    return out.reshape(-1, c)


def apply_DT(Y: np.ndarray, dims, d: int, sign: int, delta: float) -> np.ndarray:
    """((D^{sign}_d)^T Y): row i of D^{sign}_d holds coef_o / (2 delta) at column i + sign*o
    (o = 0, 1, 2; coef = sign * (3, -4, 1)), so column j of D^T Y gathers coef_o Y[j - sign*o]
    over the rows j - sign*o inside the grid (zero ghost layers, as in apply_D)."""
    nx, ny, nz = dims
    c = Y.shape[1]
    V = Y.reshape(nz, ny, nx, c)
    ax = AXIS_OF[d]
    pad = [(0, 0)] * 4
    pad[ax] = (2, 2)
    P = np.pad(V, pad)
    L = V.shape[ax]

    def shifted(s):
        sl = [slice(None)] * 4
        sl[ax] = slice(2 + s, 2 + s + L)
        return P[tuple(sl)]

    out = np.zeros_like(V)
    for o, coef in ((0, 3.0), (1, -4.0), (2, 1.0)):
        out = out + sign * coef / (2.0 * delta) * shifted(-sign * o)
    return out.reshape(-1, c)


def stencil_matrix(dims, d: int, sign: int, delta: float) -> np.ndarray:
    """Dense D^{sign}_d assembled entry by entry (small grids only)."""
    nx, ny, nz = dims
    n = nx * ny * nz
    D = np.zeros((n, n))

    def idx(i, j, k):
        return (k * ny + j) * nx + i

    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                row = idx(i, j, k)
                for off, coef in ((0, 3.0), (1, -4.0), (2, 1.0)):
                    s = off * sign
                    ii, jj, kk = i, j, k
                    if d == 0:
                        ii = i + s
                    elif d == 1:
                        jj = j + s
                    else:
                        kk = k + s
                    if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz:
                        D[row, idx(ii, jj, kk)] += sign * coef / (2.0 * delta)
    return D
