"""Hyper-parameter selection and warm start (TEST INFRASTRUCTURE ONLY).

Restates the paper's hyper-parameter selection and initialisation section and
the three steps of the Examples section that determine tile ranks:

* for a tile size b the solution X-bar is cut into tiles and every tile's
  singular values are computed; v0 is the largest over all tiles; a tile's
  numerical rank is the number of its singular values not below eps v0
  (eps = 0.01 in the paper; a tile with none below is numerically full rank);
* the entry count of a choice is the number of factor entries,
  sum over pairs of k_ij (d_i + d_j) plus, per diagonal tile, d_i k_ii or d_i^2
  (dense where k_ii >= b/4, the configurations' rule); the tile size with the
  fewest entries (largest entry count ratio nr^2 / entries) is chosen;
* warm start: off-diagonal tiles from the truncated SVD, L = U_k Sigma_k^1/2,
  R = Sigma_k^1/2 V_k (stored transposed here: X_ij = L R^T, so
  R = conj(V_k) Sigma_k^1/2 with V the right singular vectors); diagonal tiles
  Q with Q Q^T = X_ii (Takagi form, from the SVD of the symmetric tile:
  U = conj(V) D with D diagonal unitary, Q = conj(V_k) D_k^1/2 Sigma_k^1/2);
  dense diagonal tiles Z = X_ii.

Plain numpy SVDs in FP64; tiles are visited one by one.
"""
from __future__ import annotations

import numpy as np

from . import layout as lay_mod


def lower_tiles(nr: int, b: int) -> list:
    """(i, j) of the diagonal tiles, then of the pairs in stacking order."""
    n = nr // b
    return [(i, i) for i in range(n)] + list(lay_mod.pairs(n))


def tile_svdvals(X, b: int) -> list:
    X = np.asarray(X, np.complex128)
    out = []
    for i, j in lower_tiles(X.shape[0], b):
        out.append(np.linalg.svd(X[i * b:(i + 1) * b, j * b:(j + 1) * b], compute_uv=False))
    return out


def tile_ranks(X, b: int, eps: float = 0.01):
    """(ranks in descriptor order, entry count, v0) by the rank rule."""
    X = np.asarray(X, np.complex128)
    nr = X.shape[0]
    n = nr // b
    sv = tile_svdvals(X, b)
    v0 = max(float(s[0]) for s in sv)
    ranks = [int(np.count_nonzero(s >= eps * v0)) for s in sv]
    entries = 0
    for i in range(n):
        k = ranks[i]
        entries += b * b if 4 * k >= b else b * k
    for p in range(n * (n - 1) // 2):
        entries += 2 * b * ranks[n + p]
    return ranks, entries, v0


def choose_tile(X, candidates, eps: float = 0.01):
    """The candidate tile size with the fewest factor entries (first on ties)."""
    nr = np.asarray(X).shape[0]
    best = None
    for b in candidates:
        if b <= 0 or nr % b != 0:
            continue
        _, e, _ = tile_ranks(X, b, eps)
        if best is None or e < best[1]:
            best = (b, e)
    return best


def takagi(S, k: int):
    """Q (b x k) with Q Q^T the rank-k truncation of the complex symmetric S,
    from its SVD S = U Sigma V^H: U = conj(V) D, D diagonal unitary."""
    U, s, Vh = np.linalg.svd(S)
    V = Vh.conj().T
    d = np.einsum("rq,rq->q", V, U)          # diag(V^T U)
    E = np.sqrt(d / np.abs(d))
    return (V.conj() * E)[:, :k] * np.sqrt(s[:k])


def warm_start(X, lay: lay_mod.Layout) -> np.ndarray:
    """theta of ``lay`` initialised from X (Hilbert order)."""
    X = np.asarray(X, np.complex128)
    th = np.zeros(lay.size, np.complex128)
    for i in range(lay.n):
        T = X[lay.rows(i), lay.rows(i)]
        o = lay.off_diag[i]
        if lay.dense[i]:
            th[o:o + T.size] = T.ravel()
        elif lay.k_diag[i] > 0:
            Q = takagi(T, lay.k_diag[i])
            th[o:o + Q.size] = Q.ravel()
    for p, (i, j) in enumerate(lay.pair_list):
        k = lay.k_pair[p]
        if k == 0:
            continue
        U, s, Vh = np.linalg.svd(X[lay.rows(i), lay.rows(j)])
        rs = np.sqrt(s[:k])
        L = U[:, :k] * rs
        R = Vh[:k, :].T * rs                  # conj(V_k) Sigma_k^1/2
        th[lay.off_l[p]:lay.off_l[p] + L.size] = L.ravel()
        th[lay.off_r[p]:lay.off_r[p] + R.size] = R.ravel()
    return th
