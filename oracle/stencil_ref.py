"""Thermal 2-D stencil (the hotspot-like second component) — TEST INFRASTRUCTURE ONLY.

The paper evaluates its framework on Rodinia's Hotspot among other
applications (Table 2: CUDA and OpenMP variants, square grids 64 - 8192) but
does not state the computation; the reading used here is the explicit
finite-difference step of the 2-D heat equation on a chip grid with a power
source and a leak to ambient, written from that physics:

    T'[i, j] = T[i, j] + c * ( P[i, j]
                               + (T[i-1, j] + T[i+1, j] - 2 T[i, j]) * gy
                               + (T[i, j-1] + T[i, j+1] - 2 T[i, j]) * gx
                               + (amb - T[i, j]) * gz )

with c = dt / heat capacity and gx, gy, gz the conductances (1/R) to the
column neighbours, row neighbours and ambient.  The grid edge is insulated:
a neighbour outside the grid is replaced by the cell itself, so no heat
flows across the edge.  ``iters`` steps are applied; the result is T after
the last step (``iters == 0``: T unchanged).  The explicit scheme is stable
when c * (2 gx + 2 gy + gz) <= 1.

Two statements of the same step are given, so that each pins the other:
:func:`step` (array form, edge replication by padding) and
:func:`step_loops` (one cell at a time, explicit edge tests) for tiny grids.
Everything is float64.
"""
import numpy as np


def step(T, P, c, gx, gy, gz, amb):
    """One explicit step on the whole grid (float64 arrays, rows x cols)."""
    T = np.asarray(T, dtype=np.float64)
    P = np.asarray(P, dtype=np.float64)
    Tp = np.pad(T, 1, mode="edge")            # insulated edge: neighbour = cell
    north, south = Tp[:-2, 1:-1], Tp[2:, 1:-1]
    west, east = Tp[1:-1, :-2], Tp[1:-1, 2:]
    flux = (P + (north + south - 2.0 * T) * gy + (west + east - 2.0 * T) * gx
            + (amb - T) * gz)
    return T + c * flux


def run(T0, P, iters, c, gx, gy, gz, amb):
    """T after ``iters`` steps (float64)."""
    T = np.asarray(T0, dtype=np.float64).copy()
    for _ in range(int(iters)):
        T = step(T, P, c, gx, gy, gz, amb)
    return T


def step_loops(T, P, c, gx, gy, gz, amb):
    """The same step one cell at a time (pure Python; tiny grids only)."""
    rows, cols = len(T), len(T[0])
    out = [[0.0] * cols for _ in range(rows)]
    for i in range(rows):
        for j in range(cols):
            t = float(T[i][j])
            n = float(T[i - 1][j]) if i > 0 else t
            s = float(T[i + 1][j]) if i < rows - 1 else t
            w = float(T[i][j - 1]) if j > 0 else t
            e = float(T[i][j + 1]) if j < cols - 1 else t
            out[i][j] = t + c * (float(P[i][j]) + (n + s - 2.0 * t) * gy
                                 + (w + e - 2.0 * t) * gx + (amb - t) * gz)
    return np.array(out, dtype=np.float64)


def stable(c, gx, gy, gz):
    """Whether the explicit step is stable for these coefficients."""
    return c * (2.0 * gx + 2.0 * gy + gz) <= 1.0
