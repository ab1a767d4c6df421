"""Stacked unknowns of the TLR parametrisation (Tile Low-rank MDD section).

X (n_r x n_r, Hilbert order) is cut into N x N tiles: tile (i, j) covers
rows of block i and columns of block j, block i holding d_i consecutive
receivers.  The paper's experiments partition uniformly (d_i = b = n_r/N) and
note that equal tiles are not a necessary constraint; both are supported here
(``tiles``: the list of d_i).  The unknowns are stacked as the paper's three
vectors, in this order:

* Z-bar: one entry per diagonal tile i = 0..N-1, either Q_ii (d_i x k_ii,
  low-rank diagonal, X_ii = Q_ii Q_ii^T, eq. 6) or Z_ii (d_i x d_i, dense
  diagonal, X_ii = P Z_ii, eq. 7);
* L-bar: L_ij (d_i x k_ij) for every sub-diagonal tile i > j, in the paper's
  order L_21, L_31, ..., L_N,N-1 -- tile column j ascending, then row i;
* R-bar: R_ij (d_j x k_ij) in the same pair order.

Each block is stored row-major.  R_ij is stored as the d_j x k matrix whose
transpose is the paper's k x d_j factor, so that X_ij = L_ij R_ij^T (eq. 8)
and X_ji = R_ij L_ij^T (eq. 9).  A tile's rank is at most min(d_i, d_j).

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
    b: int | None                # the tile size of a uniform partition, else None
    n: int                       # tiles per side
    k_diag: list                 # rank of each diagonal tile (ignored if dense)
    dense: list                  # diagonal tile i is dense Z_ii
    k_pair: list                 # rank of each sub-diagonal pair, stacking order
    pair_list: list = field(default_factory=list)
    off_diag: list = field(default_factory=list)
    off_l: list = field(default_factory=list)
    off_r: list = field(default_factory=list)
    size: int = 0
    d: list = field(default_factory=list)      # tile sizes d_i
    roff: list = field(default_factory=list)   # first row of block i

    def diag_shape(self, i):
        return (self.d[i], self.d[i]) if self.dense[i] else (self.d[i], self.k_diag[i])

    def diag_block(self, theta, i):
        r, c = self.diag_shape(i)
        o = self.off_diag[i]
        return theta[o:o + r * c].reshape(r, c)

    def l_block(self, theta, p):
        i, k = self.pair_list[p][0], self.k_pair[p]
        o = self.off_l[p]
        return theta[o:o + self.d[i] * k].reshape(self.d[i], k)

    def r_block(self, theta, p):
        j, k = self.pair_list[p][1], self.k_pair[p]
        o = self.off_r[p]
        return theta[o:o + self.d[j] * k].reshape(self.d[j], k)

    def rows(self, i):
        return slice(self.roff[i], self.roff[i] + self.d[i])


def partition(nr: int, b, tiles=None):
    """Tile sizes d_i and block offsets: ``tiles`` (a list of d_i >= 1 summing
    to n_r) or, when it is None, N = n_r / b equal tiles of size b."""
    if tiles is None:
        if b is None or b <= 0 or nr % b != 0:
            raise ValueError("tile size must divide n_r")
        d = [int(b)] * (nr // b)
    else:
        d = [int(t) for t in tiles]
        if not d or min(d) <= 0 or sum(d) != nr:
            raise ValueError("tile sizes must be positive and sum to n_r")
    roff = [0]
    for t in d[:-1]:
        roff.append(roff[-1] + t)
    return d, roff


def make_layout(nr: int, b, ranks, diag_mode="rule", tiles=None) -> Layout:
    """Build the stacking for tile size ``b`` (or the tile sizes ``tiles``)
    and ranks.

    ``ranks``: int (uniform) or N diagonal ranks followed by N(N-1)/2 pair
    ranks in stacking order.  ``diag_mode``: "rule" (dense iff k_ii >= d_i/4,
    the workload configurations' rule), "lowrank", "dense", or a sequence of
    N booleans (True = dense).
    """
    d, roff = partition(nr, b, tiles)
    n = len(d)
    pl = pairs(n)
    if isinstance(ranks, (int, np.integer)):
        kd = [int(ranks)] * n
        kp = [int(ranks)] * len(pl)
    else:
        ranks = [int(r) for r in ranks]
        if len(ranks) != n + len(pl):
            raise ValueError("need N + N(N-1)/2 ranks")
        kd, kp = ranks[:n], ranks[n:]
    for i in range(n):
        if kd[i] < 0 or kd[i] > d[i]:
            raise ValueError("diagonal ranks must lie in [0, d_i]")
    for p, (i, j) in enumerate(pl):
        if kp[p] < 0 or kp[p] > min(d[i], d[j]):
            raise ValueError("pair ranks must lie in [0, min(d_i, d_j)]")
    if isinstance(diag_mode, str):
        if diag_mode == "rule":
            dense = [4 * kd[i] >= d[i] for i in range(n)]
        elif diag_mode == "lowrank":
            dense = [False] * n
        elif diag_mode == "dense":
            dense = [True] * n
        else:
            raise ValueError(diag_mode)
    else:
        dense = [bool(x) for x in diag_mode]
    uniform = b if tiles is None else (d[0] if len(set(d)) == 1 else None)
    lay = Layout(nr, uniform, n, kd, dense, kp, pl, d=d, roff=roff)
    o = 0
    for i in range(n):
        lay.off_diag.append(o)
        r, c = lay.diag_shape(i)
        o += r * c
    for p, (i, j) in enumerate(pl):
        lay.off_l.append(o)
        o += d[i] * kp[p]
    for p, (i, j) in enumerate(pl):
        lay.off_r.append(o)
        o += d[j] * kp[p]
    lay.size = o
    return lay
