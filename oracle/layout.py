"""Stacked unknowns of the TLR parametrisation (Tile Low-rank MDD section).

X (n_r x n_r, Hilbert order) is cut into N x N tiles of equal size b = n_r/N
(the paper partitions uniformly, "not a necessary constraint").  The unknowns
are stacked as the paper's three vectors, in this order:

* Z-bar: one entry per diagonal tile i = 0..N-1, either Q_ii (b x k_ii,
  low-rank diagonal, X_ii = Q_ii Q_ii^T, eq. 6) or Z_ii (b x b, dense
  diagonal, X_ii = P Z_ii, eq. 7);
* L-bar: L_ij (b x k_ij) for every sub-diagonal tile i > j, in the paper's
  order L_21, L_31, ..., L_N,N-1 -- tile column j ascending, then row i;
* R-bar: R_ij in the same pair order.

Each block is stored row-major.  R_ij is stored as the b x k matrix whose
transpose is the paper's k x d_j factor, so that X_ij = L_ij R_ij^T (eq. 8)
and X_ji = R_ij L_ij^T (eq. 9).

0-based pair index of tile (i, j), i > j:  p(i, j) = j N - j(j+1)/2 + (i-j-1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def pair_index(i: int, j: int, n: int) -> int:
    """Closed form of the position of tile (i, j), i > j, in L-bar / R-bar."""
    return j * n - j * (j + 1) // 2 + (i - j - 1)


def pairs(n: int) -> list:
    """Sub-diagonal tiles in stacking order (column j outer, row i inner)."""
    return [(i, j) for j in range(n) for i in range(j + 1, n)]


@dataclass
class Layout:
    nr: int
    b: int
    n: int                       # tiles per side
    k_diag: list                 # rank of each diagonal tile (ignored if dense)
    dense: list                  # diagonal tile i is dense Z_ii
    k_pair: list                 # rank of each sub-diagonal pair, stacking order
    pair_list: list = field(default_factory=list)
    off_diag: list = field(default_factory=list)
    off_l: list = field(default_factory=list)
    off_r: list = field(default_factory=list)
    size: int = 0

    def diag_shape(self, i):
        return (self.b, self.b) if self.dense[i] else (self.b, self.k_diag[i])

    def diag_block(self, theta, i):
        r, c = self.diag_shape(i)
        o = self.off_diag[i]
        return theta[o:o + r * c].reshape(r, c)

    def l_block(self, theta, p):
        o = self.off_l[p]
        return theta[o:o + self.b * self.k_pair[p]].reshape(self.b, self.k_pair[p])

    def r_block(self, theta, p):
        o = self.off_r[p]
        return theta[o:o + self.b * self.k_pair[p]].reshape(self.b, self.k_pair[p])

    def rows(self, i):
        return slice(i * self.b, (i + 1) * self.b)


def make_layout(nr: int, b: int, ranks, diag_mode="rule") -> Layout:
    """Build the stacking for tile size ``b`` and ranks.

    ``ranks``: int (uniform) or N diagonal ranks followed by N(N-1)/2 pair
    ranks in stacking order.  ``diag_mode``: "rule" (dense iff k_ii >= b/4,
    the workload configurations' rule), "lowrank", "dense", or a sequence of
    N booleans (True = dense).
    """
    if b <= 0 or nr % b != 0:
        raise ValueError("tile size must divide n_r")
    n = nr // b
    pl = pairs(n)
    if isinstance(ranks, (int, np.integer)):
        kd = [int(ranks)] * n
        kp = [int(ranks)] * len(pl)
    else:
        ranks = [int(r) for r in ranks]
        if len(ranks) != n + len(pl):
            raise ValueError("need N + N(N-1)/2 ranks")
        kd, kp = ranks[:n], ranks[n:]
    for k in kd + kp:
        if k < 0 or k > b:
            raise ValueError("ranks must lie in [0, b]")
    if isinstance(diag_mode, str):
        if diag_mode == "rule":
            dense = [4 * k >= b for k in kd]
        elif diag_mode == "lowrank":
            dense = [False] * n
        elif diag_mode == "dense":
            dense = [True] * n
        else:
            raise ValueError(diag_mode)
    else:
        dense = [bool(x) for x in diag_mode]
    lay = Layout(nr, b, n, kd, dense, kp, pl)
    o = 0
    for i in range(n):
        lay.off_diag.append(o)
        r, c = lay.diag_shape(i)
        o += r * c
    for p in range(len(pl)):
        lay.off_l.append(o)
        o += b * kp[p]
    for p in range(len(pl)):
        lay.off_r.append(o)
        o += b * kp[p]
    lay.size = o
    return lay
