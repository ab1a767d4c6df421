"""Hilbert-curve receiver reordering (Receivers re-ordering section, eq. 10-14).

The paper reorders the receivers (the columns of D and U, and both the rows
and columns of X) along a Hilbert space-filling curve so that receivers close
on the ground are close in the matrix.  It does not fix the curve's variant,
orientation or how a non-square grid is embedded; this oracle uses the
classic iterative distance map of the curve on the smallest power-of-two
square that holds the grid, with the base cell order (0,0), (0,1), (1,1),
(1,0).  Receiver r of an nx x ny grid sits at x = r mod nx, y = r div nx.
Keys are distinct, so sorting by key gives a unique permutation.
"""
from __future__ import annotations

import numpy as np


def side_pow2(nx: int, ny: int) -> int:
    """Smallest power of two n with n >= max(nx, ny) (n >= 1)."""
    n = 1
    while n < max(nx, ny):
        n *= 2
    return n


def xy2d(n: int, x: int, y: int) -> int:
    """Distance along the Hilbert curve of cell (x, y) in an n x n grid.

    Walks the quadrants from the coarsest level down: at level s the cell's
    quadrant (rx, ry) contributes s*s*((3*rx) xor ry) cells that the curve
    visits first, then the coordinates are reflected/transposed so the
    sub-square is traversed in the canonical orientation.
    """
    d = 0
    s = n // 2
    while s > 0:
        rx = 1 if (x & s) else 0
        ry = 1 if (y & s) else 0
        d += s * s * ((3 * rx) ^ ry)
        if ry == 0:
            if rx == 1:
                x = n - 1 - x
                y = n - 1 - y
            x, y = y, x
        s //= 2
    return d


def keys(nx: int, ny: int) -> np.ndarray:
    """Hilbert key of every receiver in natural order r = y*nx + x."""
    n = side_pow2(nx, ny)
    out = np.empty(nx * ny, dtype=np.int64)
    for y in range(ny):
        for x in range(nx):
            out[y * nx + x] = xy2d(n, x, y)
    return out


def perm(nx: int, ny: int) -> np.ndarray:
    """perm[a] = natural index of the receiver at Hilbert position a.

    This is the column selection of S in eq. (10): (D S)[:, a] = D[:, perm[a]].
    """
    k = keys(nx, ny)
    return np.argsort(k, kind="stable").astype(np.int32)


def hilbert_matrix(p: np.ndarray) -> np.ndarray:
    """The permutation matrix S of eq. (10): S[perm[a], a] = 1."""
    n = len(p)
    s = np.zeros((n, n))
    s[p, np.arange(n)] = 1.0
    return s
